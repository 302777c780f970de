"""Pins of the oracle's crease extraction (Sec. 4: marching squares on the zero
contour of d = det(g | Hg)).

  * d and the strongest eigenvalue in closed form on quadratic images (the
    derivative kernels are exact on quadratics away from the border);
  * the segments of a linear field lie exactly on its zero line, one per cell;
  * both resolutions of a saddle cell, their segments worked out by hand;
  * the crease-type filter keeps ridges (negative strongest eigenvalue) or
    valleys (positive) only;
  * an elongated Gaussian blob: d is odd in y about the blob's (half-integer)
    centre row, so the zero crossings next to that row lie exactly on it.
"""
import numpy as np
import pytest


def test_field_on_quadratics(oracle):
    h, w = 40, 46
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    a, b, c, p, q = 0.03, -0.02, 0.05, 0.4, -0.7
    u = 0.5 * a * X * X + b * X * Y + 0.5 * c * Y * Y + p * X + q * Y + 2.0
    d, nu = oracle.crease_field(u, sigma=1.0)
    ux, uy = a * X + b * Y + p, b * X + c * Y + q
    want = ux * (b * ux + c * uy) - uy * (a * ux + b * uy)
    m, r = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
    inner = (slice(6, h - 6), slice(6, w - 6))
    assert np.abs(d[inner] - want[inner]).max() < 1e-10
    assert np.abs(nu[inner] - (m + r if m > 0 else m - r)).max() < 1e-12


def test_linear_field_zero_line(oracle):
    h, w = 6, 8
    X = np.mgrid[0:h, 0:w][1].astype(np.float64)
    d = X - 3.3
    segs, keys = oracle.marching_squares(d, -np.ones((h, w)), oracle.RIDGE)
    assert len(segs) == h - 1
    assert np.array_equal(keys, [2 * (j * (w - 1) + 3) for j in range(h - 1)])
    for j, s in enumerate(segs):  # right edge of cell 3 is not crossed: the top and bottom edges are
        assert np.allclose(s, [3.3, j, 3.3, j + 1], rtol=0, atol=1e-12)
    assert len(oracle.marching_squares(d, -np.ones((h, w)), oracle.VALLEY)[0]) == 0
    assert len(oracle.marching_squares(d, -np.ones((h, w)), oracle.BOTH)[0]) == h - 1


def test_saddle_cells(oracle):
    nu = -np.ones((2, 2))
    # corners TL, TR / BL, BR = 1, -1 / -1, 1: mean 0, the inside corners TL and BR are cut off
    segs, keys = oracle.marching_squares(np.array([[1.0, -1.0], [-1.0, 1.0]]), nu, oracle.RIDGE)
    assert np.array_equal(keys, [0, 1])
    assert np.allclose(segs, [[0.5, 0.0, 0.0, 0.5], [1.0, 0.5, 0.5, 1.0]], rtol=0, atol=1e-15)
    # TL raised to 1.5: mean 0.125 > 0, TL and BR connected, the outside corners TR and BL cut off
    segs, keys = oracle.marching_squares(np.array([[1.5, -1.0], [-1.0, 1.0]]), nu, oracle.RIDGE)
    assert np.allclose(segs, [[0.6, 0.0, 1.0, 0.5], [0.5, 1.0, 0.0, 0.6]], rtol=0, atol=1e-15)


def test_elongated_blob_ridge_line(oracle):
    h, w = 40, 61
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0  # cy = 19.5: between two rows
    u = np.exp(-(X - cx) ** 2 / (2 * 12.0 ** 2) - (Y - cy) ** 2 / (2 * 3.0 ** 2))
    segs, _ = oracle.extract_creases(u, sigma=1.0, mode=oracle.RIDGE)
    near = [s for s in segs if abs(s[1] - cy) < 0.5 and abs(s[3] - cy) < 0.5 and abs(0.5 * (s[0] + s[2]) - cx) < 15]
    assert len(near) >= 20
    for s in near:
        assert abs(s[1] - cy) < 1e-9 and abs(s[3] - cy) < 1e-9
    # a valley filter rejects this bright ridge near the centre
    vsegs, _ = oracle.extract_creases(u, sigma=1.0, mode=oracle.VALLEY)
    assert not any(abs(s[1] - cy) < 0.5 and abs(0.5 * (s[0] + s[2]) - cx) < 10 for s in vsegs)
