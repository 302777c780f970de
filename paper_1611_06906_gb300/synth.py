"""Seeded synthetic inputs for the MAFOD filter.

This module only draws pseudo-random numbers and renders test images; it holds
none of the filter's arithmetic, so both the CUDA path and the FP64 oracle can
consume its outputs.  Everything is generated on the host in float64 and
rounded to float32 once; the oracle then reads the same float32 values
(upcast).

Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) with uniform doubles from the top 53 bits and
normals from the Box-Muller transform, so the streams are identical on every
platform and numpy version.

Workloads (they stand in for the paper's synthetic test images and the infrared
fundus data, which are not available; widths are Gaussian standard deviations):
  ridges_128          128x128, two straight ridges and one circular arc of widths
                      1.5, 2.5, 4 px, amplitude 1 on 0, noise sd 0.1
  vessel_tree         dark branching tree (depth d, radius r0 * (r1/r0)^(level/(d-1)))
                      of valleys on a bright background with a linear gradient
  fundus_like         vessel_tree inside a circular field of view with radial
                      vignetting (1 - 0.4 rho^2)
  batch_uneven        64 fundus_like images with sides drawn from 512..2048
  tree16              4096x4096 depth-8 tree, radii 12 -> 0.75 px, mixed polarity,
                      noise sd 0.15 (16 of them form the full-size workload)
"""
from __future__ import annotations

import math

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & _M64)

    def next_u64(self, n: int) -> np.ndarray:
        gamma = np.uint64(0x9E3779B97F4A7C15)
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + idx * gamma
            self.state = self.state + np.uint64(n) * gamma
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (two uniforms per pair)."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
        z = np.concatenate([rad * np.cos(2.0 * math.pi * u2), rad * np.sin(2.0 * math.pi * u2)])
        return z[:n]

    def scalar(self) -> float:
        return float(self.uniform(1)[0])


def _seg_dist(X, Y, ax, ay, bx, by):
    dx, dy = bx - ax, by - ay
    L2 = dx * dx + dy * dy
    t = np.clip(((X - ax) * dx + (Y - ay) * dy) / max(L2, 1e-12), 0.0, 1.0)
    px, py = ax + t * dx, ay + t * dy
    return np.hypot(X - px, Y - py)


def _stamp_segment(acc, ax, ay, bx, by, width, amp, combine):
    """Gaussian cross-section exp(-d^2 / 2 w^2) around a segment, combined by max/min."""
    h, w = acc.shape
    pad = 4.0 * width + 2.0
    x0 = max(int(math.floor(min(ax, bx) - pad)), 0)
    x1 = min(int(math.ceil(max(ax, bx) + pad)) + 1, w)
    y0 = max(int(math.floor(min(ay, by) - pad)), 0)
    y1 = min(int(math.ceil(max(ay, by) + pad)) + 1, h)
    if x0 >= x1 or y0 >= y1:
        return
    Y, X = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    d = _seg_dist(X, Y, ax, ay, bx, by)
    prof = amp * np.exp(-d * d / (2.0 * width * width))
    sub = acc[y0:y1, x0:x1]
    acc[y0:y1, x0:x1] = combine(sub, prof)


def ridges_128(seed: int = 1000, size: int = 128, widths=(1.5, 2.5, 4.0), noise=0.1):
    """Two straight ridges and one circular arc, amplitude 1 on 0, max-combined, plus noise.

    Returns (float32 image, list of (kind, params, width))."""
    rng = SplitMix64(seed)
    img = np.zeros((size, size))
    Y, X = np.mgrid[0:size, 0:size].astype(np.float64)
    parts = []
    # two straight ridges: random angle, offsets keep them apart (>= 6 w)
    ang = math.pi * rng.scalar()
    nx, ny = -math.sin(ang), math.cos(ang)
    c = size / 2.0
    offs = (-0.25 * size, 0.02 * size)
    for wdt, off in zip(widths[:2], offs):
        d = np.abs((X - c) * nx + (Y - c) * ny - off)
        img = np.maximum(img, np.exp(-d * d / (2.0 * wdt * wdt)))
        parts.append(("line", (ang, off), wdt))
    # circular arc in the remaining half
    wdt = widths[2]
    cx = c + 0.28 * size * nx + 0.1 * size * (rng.scalar() - 0.5)
    cy = c + 0.28 * size * ny + 0.1 * size * (rng.scalar() - 0.5)
    R = 0.22 * size
    a0 = math.atan2(ny, nx) - 0.5 * math.pi
    phi = np.arctan2(Y - cy, X - cx)
    dphi = np.mod(phi - a0, 2.0 * math.pi)
    on_arc = dphi <= math.pi
    rr = np.hypot(X - cx, Y - cy)
    d_arc = np.abs(rr - R)
    ex = np.stack([cx + R * np.cos(a0), cy + R * np.sin(a0)]), np.stack([cx + R * np.cos(a0 + math.pi), cy + R * np.sin(a0 + math.pi)])
    d_end = np.minimum(np.hypot(X - ex[0][0], Y - ex[0][1]), np.hypot(X - ex[1][0], Y - ex[1][1]))
    d = np.where(on_arc, d_arc, d_end)
    img = np.maximum(img, np.exp(-d * d / (2.0 * wdt * wdt)))
    parts.append(("arc", (cx, cy, R, a0), wdt))
    img = img + noise * rng.normal(size * size).reshape(size, size)
    return img.astype(np.float32), parts


def ridge_profile(size_x: int, size_y: int, width: float, amp: float = 1.0, angle: float = 0.0):
    """Noise-free straight ridge amp * exp(-d^2 / 2 w^2) through the centre (float64)."""
    Y, X = np.mgrid[0:size_y, 0:size_x].astype(np.float64)
    cx, cy = (size_x - 1) / 2.0, (size_y - 1) / 2.0
    nx, ny = -math.sin(angle), math.cos(angle)
    d = (X - cx) * nx + (Y - cy) * ny
    return amp * np.exp(-d * d / (2.0 * width * width))


def _tree_segments(rng: SplitMix64, w: int, h: int, depth: int, r0: float, r1: float):
    """Random binary branching tree: list of (ax, ay, bx, by, radius)."""
    segs = []
    # root enters from a random border side, heading roughly inward
    side = int(rng.scalar() * 4) % 4
    t = 0.3 + 0.4 * rng.scalar()
    if side == 0:
        x, y, ang = t * w, 0.0, 0.5 * math.pi
    elif side == 1:
        x, y, ang = w - 1.0, t * h, math.pi
    elif side == 2:
        x, y, ang = t * w, h - 1.0, -0.5 * math.pi
    else:
        x, y, ang = 0.0, t * h, 0.0
    ang += (rng.scalar() - 0.5) * 0.5
    L0 = 0.32 * min(w, h)
    stack = [(x, y, ang, 0)]
    while stack:
        x, y, a, lvl = stack.pop()
        rad = r0 * (r1 / r0) ** (lvl / max(depth - 1, 1))
        L = L0 * (0.72 ** lvl) * (0.8 + 0.4 * rng.scalar())
        # a gently bending vessel: three sub-segments
        cx, cy, ca = x, y, a
        bend = (rng.scalar() - 0.5) * 0.6
        for _ in range(3):
            nx_, ny_ = cx + L / 3.0 * math.cos(ca), cy + L / 3.0 * math.sin(ca)
            segs.append((cx, cy, nx_, ny_, rad))
            cx, cy, ca = nx_, ny_, ca + bend / 3.0
        if lvl + 1 < depth:
            for sgn in (-1.0, 1.0):
                da = math.radians(20.0 + 20.0 * rng.scalar())
                stack.append((cx, cy, ca + sgn * da, lvl + 1))
    return segs


def vessel_tree(seed: int, w: int = 1024, h: int = 1024, depth: int = 6, r0: float = 8.0,
                r1: float = 1.0, amp: float = -0.4, background: float = 0.6, gradient: float = 0.2,
                noise=None, polarity_mix: bool = False):
    """Dark vessel tree (valleys of depth |amp|) on a bright background with a linear gradient.

    noise=None draws sd ~ U[0.05, 0.2] from the stream.  polarity_mix=True gives each
    branch a random sign (ridges and valleys).  Returns float32 (h, w)."""
    rng = SplitMix64(seed)
    if noise is None:
        noise = 0.05 + 0.15 * rng.scalar()
    ga = 2.0 * math.pi * rng.scalar()
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    base = background + gradient * (((X / max(w - 1, 1)) - 0.5) * math.cos(ga) + ((Y / max(h - 1, 1)) - 0.5) * math.sin(ga))
    dark = np.zeros((h, w))
    bright = np.zeros((h, w))
    for (ax, ay, bx, by, rad) in _tree_segments(rng, w, h, depth, r0, r1):
        sgn = -1.0 if (polarity_mix and rng.scalar() < 0.5) else 1.0
        a = abs(amp)
        if (amp < 0) == (sgn > 0):
            _stamp_segment(dark, ax, ay, bx, by, rad, a, np.maximum)
        else:
            _stamp_segment(bright, ax, ay, bx, by, rad, a, np.maximum)
    img = base - dark + bright + noise * rng.normal(w * h).reshape(h, w)
    return img.astype(np.float32)


def vessel_tree_centrelines(seed: int, w: int = 1024, h: int = 1024, depth: int = 6, r0: float = 8.0,
                            r1: float = 1.0, noise=None):
    """The centre-line segments (ax, ay, bx, by, radius) of vessel_tree with the same
    arguments: the generator's draws replayed up to the tree (the ground truth of the
    crease evaluation)."""
    rng = SplitMix64(seed)
    if noise is None:
        rng.scalar()
    rng.scalar()  # gradient angle
    return _tree_segments(rng, w, h, depth, r0, r1)


def fundus_like(seed: int, side: int, depth: int = 6, noise: float = 0.1):
    """Fundus-like square image: circular field of view, radial vignetting, dark tree."""
    tree = vessel_tree(seed, side, side, depth=depth, noise=0.0).astype(np.float64)
    rng = SplitMix64(seed ^ 0x5EED)
    Y, X = np.mgrid[0:side, 0:side].astype(np.float64)
    c = (side - 1) / 2.0
    rho = np.hypot(X - c, Y - c) / (0.48 * side)
    vign = 1.0 - 0.4 * np.minimum(rho, 1.0) ** 2
    fov = 1.0 / (1.0 + np.exp((rho - 1.0) * side / 8.0))  # soft circular mask
    img = tree * vign * fov + noise * rng.normal(side * side).reshape(side, side)
    return img.astype(np.float32)


def tree16(seed: int, side: int = 4096):
    """One image of the full-size workload: a depth-8 tree with radii 12 -> 0.75 px,
    each branch a ridge or a valley at random, noise sd 0.15, side x side."""
    return vessel_tree(seed, side, side, depth=8, r0=12.0, r1=0.75, noise=0.15, polarity_mix=True)


def batch_sides(seed: int = 3000, count: int = 64, lo: int = 512, hi: int = 2048):
    rng = SplitMix64(seed)
    return [int(lo + math.floor(rng.scalar() * (hi - lo + 1))) for _ in range(count)]


def log_sigmas(lo: float, hi: float, k: int):
    """k scales log-spaced between lo and hi (inclusive)."""
    if k == 1:
        return np.array([lo])
    return np.array([lo * (hi / lo) ** (i / (k - 1)) for i in range(k)])


# Workload descriptions.  lambda = 0.005, rho = 0.5, beta = 0.5 and tau_max = 0.05 are
# the paper's settings; T is chosen so that n steps per cycle sit at tau_max.
WORKLOADS = {
    "ridges_128": dict(sigmas=[1.0, 1.5, 2.0, 3.0, 4.0], mode="ridge", M=2, n=10, T=11.0 / 3.0),
    "tree_1024": dict(sigmas=list(log_sigmas(1.0, 8.0, 8)), mode="valley", M=5, n=20, T=35.0),
    "batch64_fundus": dict(sigmas=list(log_sigmas(1.0, 8.0, 8)), mode="valley", M=5, n=20, T=35.0),
    "tree16_4096": dict(sigmas=list(log_sigmas(0.75, 12.0, 12)), mode="both", M=10, n=25,
                        T=325.0 / 3.0),
}
