"""Accuracy of extracted creases against known centre lines (Sec. 5: the
average Euclidean distance E and the detected fraction p).

Host-side evaluation of crease segments (from fd4_extract_creases); it is a
measurement of results, not a step of the filter.  The paper describes the
protocol in words; the readings taken here:

  * the ground truth is a set of line segments (the generator's centre-line
    pieces), each sampled every `step` pixels;
  * the reconstruction's "segments" are its polygonal chains: the
    marching-squares segments joined where they share an endpoint;
  * for a ground-truth segment, each chain is restricted to its vertices
    within `neighbourhood` pixels of the segment (six for synthetic data, ten
    for real data in the paper); the chain (restricted) with the smallest
    symmetric Hausdorff distance to the sampled segment is its match;
  * E is the mean, over matched segments, of the mean distance from the
    segment's samples to the matched chain's restricted vertices joined as a
    polyline; p is the matched fraction of the ground truth's length.
"""
from __future__ import annotations

import numpy as np


def chains(segs: np.ndarray, tol: float = 1e-6):
    """Polygonal chains of segments (n, 4) joined at shared endpoints: a list of
    index arrays into segs (connected components)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    n = len(segs)
    if n == 0:
        return []
    pts = np.concatenate([segs[:, 0:2], segs[:, 2:4]])  # endpoint k belongs to segment k % n
    key = np.round(pts / tol).astype(np.int64)
    order = np.lexsort((key[:, 1], key[:, 0]))
    same = np.all(key[order[1:]] == key[order[:-1]], axis=1)
    a, b = order[:-1][same] % n, order[1:][same] % n
    graph = coo_matrix((np.ones(a.size), (a, b)), shape=(n, n))
    _, label = connected_components(graph, directed=False)
    srt = np.argsort(label, kind="stable")
    bounds = np.flatnonzero(np.diff(label[srt])) + 1
    return np.split(srt, bounds)


def _point_segment_dist(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distance of points p (m, 2) to each segment a_k b_k (k rows): (m, k)."""
    ab = b - a
    den = np.maximum((ab * ab).sum(axis=1), 1e-300)
    t = ((p[:, None, :] - a[None, :, :]) * ab[None, :, :]).sum(axis=2) / den[None, :]
    t = np.clip(t, 0.0, 1.0)
    q = a[None, :, :] + t[:, :, None] * ab[None, :, :]
    return np.sqrt(((p[:, None, :] - q) ** 2).sum(axis=2))


def evaluate(segs: np.ndarray, truth, neighbourhood: float = 6.0, step: float = 0.5):
    """E and p of crease segments (n, 4) = (x0, y0, x1, y1) against ground-truth
    segments [(ax, ay, bx, by, ...), ...].  Returns (E or nan, p)."""
    segs = np.asarray(segs, dtype=np.float64).reshape(-1, 4)
    chain_of = np.full(len(segs), -1, dtype=np.int64)
    for c, idx in enumerate(chains(segs)):
        chain_of[idx] = c
    dists, lengths, matched = [], [], []
    for g in truth:
        a = np.array(g[0:2], dtype=np.float64)
        b = np.array(g[2:4], dtype=np.float64)
        L = float(np.hypot(*(b - a)))
        if L <= 0.0:
            continue
        k = max(int(np.ceil(L / step)), 1)
        samples = a[None, :] + np.linspace(0.0, 1.0, k + 1)[:, None] * (b - a)[None, :]
        best = None
        if len(segs):
            # the segments whose endpoints both lie in the neighbourhood, by chain
            d0 = _point_segment_dist(segs[:, 0:2], a[None, :], b[None, :])[:, 0]
            d1 = _point_segment_dist(segs[:, 2:4], a[None, :], b[None, :])[:, 0]
            idx = np.flatnonzero((d0 <= neighbourhood) & (d1 <= neighbourhood))
            idx = idx[np.argsort(chain_of[idx], kind="stable")]
            groups = np.split(idx, np.flatnonzero(np.diff(chain_of[idx])) + 1) if idx.size else []
            for sel in groups:
                s = segs[sel]
                to_chain = _point_segment_dist(samples, s[:, 0:2], s[:, 2:4]).min(axis=1)
                to_truth = np.maximum(d0[sel], d1[sel])
                haus = max(float(to_chain.max()), float(to_truth.max()))
                if best is None or haus < best[0]:
                    best = (haus, float(to_chain.mean()))
        lengths.append(L)
        matched.append(best is not None)
        if best is not None:
            dists.append(best[1])
    total = float(np.sum(lengths))
    p = float(np.sum(np.array(lengths)[np.array(matched, dtype=bool)])) / total if total > 0 else 0.0
    return (float(np.mean(dists)) if dists else float("nan")), p
