"""Training and evaluation driver of the learned scale selector.

Every arithmetic step runs in libfd4 (forward and backward passes on the
tensor cores, Adam on the device); this module only generates the seeded
inputs, moves them to the device and loops.

Training set: 256 x 256 crops of seeded source images, labelled with the
scale index the plain vesselness selection picks on the whole source image
(so the labels see the same image-wide Frangi c as inference on full images).
Sources: "fundus" -- the `batch64_fundus` generator at side 2048 (64 crops
each); "tree16" -- the full-size workload's 4096^2 trees (256 crops each).
The seeds (from 900000 on) are disjoint from the benchmark's images.  A
network that re-selects the scales before every FED cycle is trained on the
images of every cycle instead (`cycles`).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import fd4, synth

CROP = 256
SOURCES = {"fundus": 2048, "tree16": 4096}


def _render(args):
    kind, seed = args
    if kind == "tree16":
        return synth.tree16(seed)
    return synth.fundus_like(seed, SOURCES["fundus"])


def source_images(n_sources: int, kind: str = "fundus", seed0: int = 900000, procs: int = 16):
    """Seeded source images (host float32), rendered in a spawn pool (so the
    calling script must guard its entry point with if __name__ == "__main__")."""
    args = [(kind, seed0 + i) for i in range(n_sources)]
    with mp.get_context("spawn").Pool(max(1, min(procs, os.cpu_count() or 1))) as pool:
        return pool.map(_render, args)


def make_training_set(n_crops: int, sigmas, mode: int, kind: str = "fundus", seed0: int = 900000, device="cuda",
                      cycles=None):
    """(crops (n, 256, 256) float32, labels (n, 256, 256) uint8) on the device.

    cycles = (T, M, n): the crops come from every cycle of the re-selecting
    schedule instead of the source images alone: before cycle c the current
    image u^c is labelled by the plain selection on it, then one FED cycle
    (T / M, n steps) runs with those scales -- the (u^c, sigma*_c) pairs a
    network that re-selects before every cycle sees."""
    import torch
    side = SOURCES[kind]
    per = (side // CROP) ** 2
    n_cyc = 1 if cycles is None else int(cycles[1])
    n_src = -(-n_crops // (per * n_cyc))
    srcs = source_images(n_src, kind, seed0)
    crops = torch.empty((n_crops, CROP, CROP), dtype=torch.float32, device=device)
    labels = torch.empty((n_crops, CROP, CROP), dtype=torch.uint8, device=device)
    prm = fd4.params(mode=mode)
    ws = fd4.workspace(fd4.OP_SELECT_SCALES, side, side, len(sigmas), device)
    wsf = fd4.workspace(fd4.OP_FILTER, side, side, len(sigmas), device) if cycles is not None else None
    k = 0
    for img in srcs:
        u = fd4.to_device(img, device)
        for c in range(n_cyc):
            idx, _ = fd4.select_scales(u, side, sigmas, prm, ws=ws)
            for cy in range(0, side, CROP):
                for cx in range(0, side, CROP):
                    if k == n_crops:
                        break
                    crops[k] = u[cy:cy + CROP, cx:cx + CROP]
                    labels[k] = idx[cy:cy + CROP, cx:cx + CROP]
                    k += 1
            if cycles is not None and c + 1 < n_cyc:
                T, M, n = cycles
                u, _ = fd4.filter_image(u, side, sigmas, T / M, 1, n, prm, sigma_idx=idx, ws=wsf)
    return crops[:k], labels[:k]


def train(sel: "fd4.Selector", crops, labels, n_bins: int, epochs: int = 1, batch: int = 32, lr: float = 2e-3,
          seed: int = 1, log_every: int = 0):
    """Adam over shuffled mini-batches.  Returns the per-step mean losses."""
    import torch
    n = crops.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    ws = fd4.Selector.workspace(batch, CROP, CROP, CROP, crops.device)
    loss = torch.zeros(1, dtype=torch.float32, device=crops.device)
    losses = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g)
        for b0 in range(0, n - batch + 1, batch):
            sel_idx = perm[b0:b0 + batch].to(crops.device)
            xb = crops.index_select(0, sel_idx).contiguous()
            yb = labels.index_select(0, sel_idx).contiguous()
            loss.zero_()
            sel.grad(xb, yb, CROP, loss, n_bins=n_bins, ws=ws)
            step += 1
            # cosine decay of the step size over the run
            frac = step / max(1, epochs * (n // batch))
            sel.update(lr * (0.1 + 0.9 * 0.5 * (1 + np.cos(np.pi * frac))), step)
            losses.append(loss)
            loss = torch.zeros(1, dtype=torch.float32, device=crops.device)
            if log_every and step % log_every == 0:
                print("step %d loss %.4f" % (step, float(losses[-1].item())), flush=True)
    return [float(x.item()) for x in losses]


def evaluate(sel: "fd4.Selector", images, widths, sigmas, mode: int, thresholds=(0.0, 0.5, 0.9)):
    """Agreement of the learned selection with the plain selection per threshold.

    images: list of device (h, pitch) tensors.  Returns a dict per threshold with
    the pixel agreement and the fraction of 32 x 64 tiles that fell back."""
    import torch
    prm = fd4.params(mode=mode)
    out = {}
    plain = []
    for u, w in zip(images, widths):
        idx, _ = fd4.select_scales(u, w, sigmas, prm)
        plain.append(idx)
    for thr in thresholds:
        agree = tot = fb = tiles = 0
        for u, w, ref in zip(images, widths, plain):
            h = u.shape[0]
            idx, conf, nfb = sel.select_learned(u, w, sigmas, prm, conf_threshold=thr)
            agree += int((idx[:, :w] == ref[:, :w]).sum().item())
            tot += h * w
            fb += int(nfb.item())
            tiles += ((w + 31) // 32) * ((h + 63) // 64)
        out[thr] = {"agreement": agree / tot, "fallback_tiles": fb / tiles}
    return out
