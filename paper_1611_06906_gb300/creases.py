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
    n = len(segs)
    if n == 0:
        return []
    parent = np.arange(n)

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    pts = np.concatenate([segs[:, 0:2], segs[:, 2:4]])  # endpoint k of segment k % n
    key = np.round(pts / tol).astype(np.int64)
    order = np.lexsort((key[:, 1], key[:, 0]))
    for a, b in zip(order[:-1], order[1:]):
        if key[a, 0] == key[b, 0] and key[a, 1] == key[b, 1]:
            ra, rb = find(a % n), find(b % n)
            if ra != rb:
                parent[ra] = rb
    roots = np.array([find(i) for i in range(n)])
    return [np.nonzero(roots == r)[0] for r in np.unique(roots)]


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
    groups = chains(segs)
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
        for idx in groups:
            s = segs[idx]
            # keep the chain's segments whose endpoints both lie in the neighbourhood
            d0 = _point_segment_dist(s[:, 0:2], a[None, :], b[None, :])[:, 0]
            d1 = _point_segment_dist(s[:, 2:4], a[None, :], b[None, :])[:, 0]
            keep = (d0 <= neighbourhood) & (d1 <= neighbourhood)
            if not keep.any():
                continue
            s = s[keep]
            to_chain = _point_segment_dist(samples, s[:, 0:2], s[:, 2:4]).min(axis=1)
            to_truth = np.maximum(d0[keep], d1[keep])
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
