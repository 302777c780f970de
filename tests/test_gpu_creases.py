"""Crease extraction on the GPU (fd4_extract_creases) against the FP64 oracle:
the same cells and segment end points on a noisy vessel tree (the decisions
d > 0 and the crease-type filter are taken from FP32 values here and FP64
values in the oracle, so cells whose decision values are within rounding of
zero may differ: the test checks that every differing cell is one of them),
the exact ridge line of an elongated blob, and argument checks."""
import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4, synth

pytestmark = pytest.mark.gpu


def _fp32_bounds(oracle, img, sigma):
    """The FP64 field d = det(g | Hg), the eigenvalue field nu, and bounds on
    the FP32 rounding of both at every pixel.  A derivative computed in FP32 by
    the separable sums is off by at most about n eps sum|w u| (n the taps, eps
    2^-24); the bound takes 1e-6 of the kernels' L1 norm times max |u| (a
    margin of about 16 over eps for the tap counts here) and carries it
    through d = u_x (Hg)_y - u_y (Hg)_x to first order."""
    g0, g1, g2 = oracle.gauss_kernels(sigma)
    L0, L1, L2 = (float(np.abs(k).sum()) for k in (g0, g1, g2))
    umax = float(np.abs(img).max())
    e1 = 1e-6 * L1 * L0 * umax            # u_x, u_y
    e2 = 1e-6 * max(L2 * L0, L1 * L1) * umax  # u_xx, u_xy, u_yy
    ux, uy, hxx, hxy, hyy = oracle.derivatives(img.astype(np.float64), sigma)
    hgx, hgy = hxx * ux + hxy * uy, hxy * ux + hyy * uy
    G = np.abs(ux) + np.abs(uy)
    Hn = np.abs(hxx) + 2 * np.abs(hxy) + np.abs(hyy)
    bd = e1 * (np.abs(hgx) + np.abs(hgy)) + G * (Hn * e1 + G * e2)
    d, nu = oracle.crease_field(img, sigma)
    return d, nu, bd, 2.0 * e2


def _cell(a, cell, w):
    j, i = divmod(int(cell), w - 1)
    return np.array([a[j, i], a[j, i + 1], a[j + 1, i + 1], a[j + 1, i]])  # corners 0..3, as the cell walk


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("sigma", [1.0, 2.0])
def test_segments_match_oracle(oracle, mode, sigma):
    """Cells and end points against the oracle's FP64 field, with the FP32
    rounding bounded per pixel (_fp32_bounds, times a margin K = 4):
    * a cell kept by one side only, or kept by both with other end points,
      has a decision within rounding of zero: a corner of d, the mean of nu
      (crease-type filter) or a saddle's mean of d;
    * every other cell kept by both has its end points t = c0 / (c0 - c1)
      along each crossed edge within the propagated bound
      (|c1| b0 + |c0| b1) / (c0 - c1)^2 of a pixel, plus 1e-5."""
    K = 4.0
    h, w = 160, 200
    img = synth.vessel_tree(5300, w, h, depth=5, r0=4.0)
    d, nu, bd, bnu = _fp32_bounds(oracle, img, sigma)
    want, wkeys = oracle.marching_squares(d, nu, mode)
    got, gkeys = fd4.extract_creases(fd4.to_device(img), w, sigma=sigma, mode=mode)
    assert len(want) > 100

    def degenerate(cell):
        c, b = _cell(d, cell, w), _cell(bd, cell, w)
        nm = 0.25 * _cell(nu, cell, w).sum()
        saddle = ((c > 0).sum() == 2) and (c[0] > 0) == (c[2] > 0)
        return bool((np.abs(c) <= K * b).any() or abs(nm) <= K * bnu
                    or (saddle and abs(c.mean()) <= K * b.mean()))

    only = np.setxor1d(wkeys, gkeys)
    assert only.size <= 0.02 * max(wkeys.size, gkeys.size)
    for cell in np.unique(only // 2):
        assert degenerate(cell), ("cell kept by one side only", cell)
    common, wi, gi = np.intersect1d(wkeys, gkeys, return_indices=True)
    err = np.abs(got[gi] - want[wi]).max(axis=1)
    edges = ((0, 1), (1, 2), (3, 2), (0, 3))
    n_exact = 0
    for k, e in zip(common, err):
        cell = k // 2
        if degenerate(cell):
            assert e <= 1.0
            continue
        c, b = _cell(d, cell, w), _cell(bd, cell, w)
        bound = max(((abs(c[q]) * b[p] + abs(c[p]) * b[q]) / (c[p] - c[q]) ** 2
                     for p, q in edges if (c[p] > 0) != (c[q] > 0)), default=0.0)
        assert e <= K * bound + 1e-5, (cell, e, bound)
        n_exact += 1
    assert n_exact >= 0.9 * common.size


def test_elongated_blob_ridge_line():
    h, w = 40, 61
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    img = np.exp(-(X - cx) ** 2 / (2 * 12.0 ** 2) - (Y - cy) ** 2 / (2 * 3.0 ** 2)).astype(np.float32)
    segs, _ = fd4.extract_creases(fd4.to_device(img), w, sigma=1.0, mode=fd4.RIDGE)
    near = [s for s in segs if abs(s[1] - cy) < 0.5 and abs(s[3] - cy) < 0.5 and abs(0.5 * (s[0] + s[2]) - cx) < 15]
    assert len(near) >= 20
    assert max(max(abs(s[1] - cy), abs(s[3] - cy)) for s in near) < 1e-3


def test_arguments_are_checked():
    u = fd4.to_device(synth.vessel_tree(5301, 32, 32, depth=3, r0=3.0))
    for kw in (dict(sigma=5.0), dict(sigma=0.0), dict(mode=3)):
        with pytest.raises(fd4.Fd4Error):
            fd4.extract_creases(u, 32, **kw)
