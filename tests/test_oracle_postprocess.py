"""Pins of the oracle's scale-image post-processing (Sec. 3.3, the paragraphs
after Eq. 9: each vessel pixel takes the scale nearest to the mean scale of
its cross-section, traced along the Hessian's strongest eigenvector).

  * the strongest eigenvector in closed form (diagonal Hessians, a rotated
    diagonal one, the tie of equal magnitudes, the isotropic case);
  * hand-built fields whose cross-sections are the rows, the columns and the
    diagonals of a masked band: every mask pixel takes the scale nearest to
    the mean over its row / column / diagonal segment (numpy means, not walks);
  * the walk cap as a clipped moving window along a row; the digital line of
    slope 1/3, its pixels listed by hand;
  * an empty mask and isotropic Hessians leave the scale image unchanged;
  * a straight ridge: one scale per cross-section, the one nearest to the
    mean of the selected scales over the column's vessel pixels;
  * the filter with post-processing equals its composition from the pinned
    primitives.
"""
import math

import numpy as np
import pytest

from paper_1611_06906_gb300 import synth

SIG = np.array([1.0, 2.0, 3.0, 5.0])


def _nearest(mean):
    d = np.abs(SIG - mean)
    return int(np.argmin(d))  # first minimum: ties to the smaller sigma


def test_strong_direction_closed_forms(oracle):
    ex, ey = oracle.strong_direction(-2.0, 0.0, 1.0)
    assert abs(abs(ex) - 1.0) < 1e-15 and ey == 0.0
    ex, ey = oracle.strong_direction(1.0, 0.0, 3.0)
    assert abs(abs(ey) - 1.0) < 1e-15 and ex == 0.0
    ex, ey = oracle.strong_direction(0.0, -1.0, 0.0)  # eigenvalues +-1: the negative one, along (1, 1)
    assert abs(ex - ey) < 1e-15 and abs(abs(ex) - math.sqrt(0.5)) < 1e-15
    for phi in np.linspace(0.0, math.pi, 13):
        c, s = math.cos(phi), math.sin(phi)
        R = np.array([[c, -s], [s, c]])
        H = R @ np.diag([-5.0, 1.0]) @ R.T
        ex, ey = oracle.strong_direction(H[0, 0], H[0, 1], H[1, 1])
        assert abs(abs(ex * c + ey * s) - 1.0) < 1e-12
    assert oracle.strong_direction(2.0, 0.0, 2.0) is None


def _fields(h, w, a, b, d):
    return np.full((h, w), float(a)), np.full((h, w), float(b)), np.full((h, w), float(d))


def test_rows_columns_and_diagonals(oracle):
    rng = np.random.default_rng(5)
    h, w = 9, 11
    idx = rng.integers(0, SIG.size, size=(h, w)).astype(np.uint8)
    # cross-sections along x (strong eigenvalue of Hxx): rows of the band 3..8
    vmax = np.zeros((h, w))
    vmax[:, 3:9] = 1.0
    out = oracle.postprocess_core(idx, vmax, *_fields(h, w, -1, 0, 0), SIG, 0.2, 100)
    exp = idx.copy()
    for r in range(h):
        exp[r, 3:9] = _nearest(SIG[idx[r, 3:9]].mean())
    assert np.array_equal(out, exp)
    # along y: columns of the band of rows 2..6
    vmax = np.zeros((h, w))
    vmax[2:7, :] = 1.0
    out = oracle.postprocess_core(idx, vmax, *_fields(h, w, 0, 0, 4), SIG, 0.2, 100)
    exp = idx.copy()
    for c in range(w):
        exp[2:7, c] = _nearest(SIG[idx[2:7, c]].mean())
    assert np.array_equal(out, exp)
    # along (1, 1) (Hxy < 0 with a zero diagonal): the main-direction diagonals
    # of the anti-diagonal band 6 <= x + y <= 12
    yy, xx = np.mgrid[0:h, 0:w]
    band = (xx + yy >= 6) & (xx + yy <= 12)
    vmax = band.astype(np.float64)
    out = oracle.postprocess_core(idx, vmax, *_fields(h, w, 0, -1, 0), SIG, 0.5, 100)
    exp = idx.copy()
    for off in range(-h + 1, w):
        cells = [(y, y + off) for y in range(h) if 0 <= y + off < w and band[y, y + off]]
        if cells:
            m = np.mean([SIG[idx[y, x]] for y, x in cells])
            for y, x in cells:
                exp[y, x] = _nearest(m)
    assert np.array_equal(out, exp)


def test_walk_cap_is_a_clipped_window(oracle):
    rng = np.random.default_rng(6)
    h, w, cap = 3, 17, 2
    idx = rng.integers(0, SIG.size, size=(h, w)).astype(np.uint8)
    vmax = np.ones((h, w))
    out = oracle.postprocess_core(idx, vmax, *_fields(h, w, 3, 0, 0), SIG, 0.2, cap)
    exp = idx.copy()
    for r in range(h):
        for c in range(w):
            exp[r, c] = _nearest(SIG[idx[r, max(0, c - cap):c + cap + 1]].mean())
    assert np.array_equal(out, exp)


def test_empty_mask_and_isotropic_hessian_keep_the_scales(oracle):
    rng = np.random.default_rng(7)
    idx = rng.integers(0, SIG.size, size=(8, 8)).astype(np.uint8)
    vmax = rng.random((8, 8))
    assert np.array_equal(oracle.postprocess_core(idx, vmax, *_fields(8, 8, -1, 0, 0), SIG, 1.0, 50), idx)
    assert np.array_equal(oracle.postprocess_core(idx, vmax, *_fields(8, 8, -1, 0, -1), SIG, 0.0, 50), idx)


def test_straight_ridge_gets_one_scale_per_cross_section(oracle):
    sig = [1.0, 1.5, 2.0, 3.0, 4.0, 6.0]
    img = 0.2 + synth.ridge_profile(64, 48, 3.0)
    idx, vmax, _, _ = oracle.select_scales(img, sig, oracle.RIDGE)
    out = oracle.postprocess_scales(img, idx, vmax, sig, 0.2)
    mask = vmax > 0.2
    sig = np.array(sig)
    for c in range(16, 48):
        rows = np.nonzero(mask[:, c])[0]
        assert rows.size > 0 and rows.size == rows[-1] - rows[0] + 1  # one band per column
        want = int(np.argmin(np.abs(sig - sig[idx[rows, c]].mean())))
        assert np.all(out[rows, c] == want)
    assert np.array_equal(out[~mask], idx[~mask])


@pytest.mark.parametrize("reselect", [False, True])
def test_filter_with_postprocess_equals_composition(oracle, reselect):
    sig = [1.0, 1.6, 2.5, 4.0]
    img = synth.vessel_tree(4400, 48, 40, depth=4, r0=3.0).astype(np.float64)
    M, n = 2, 10
    tau, _, _ = oracle.fed_taus(M * n * (n + 1) * 0.05 / 3, M, 0.05, n=n)
    out, idx = oracle.filter_image(img, sig, tau, M, mode=oracle.VALLEY, reselect=reselect,
                                   postprocess=True, theta=0.2)
    u = img.copy()
    for k in range(M):
        if k == 0 or reselect:
            sel, vmax, _, _ = oracle.select_scales(u, sig, oracle.VALLEY)
            sel = oracle.postprocess_scales(u, sel, vmax, sig, 0.2)
        tensor, _ = oracle.build_tensor(u, sel, sig, mode=oracle.VALLEY)
        u = oracle.fed_cycle(u, tensor, tau)
    assert np.array_equal(out, u) and np.array_equal(idx, sel)


def test_digital_line_of_slope_one_third(oracle):
    """Strongest eigenvector along (3, 1): from p = (x 5, y 4) with cap 3 the
    cross-section is (2,3) (3,3) (4,4) (5,4) (6,4) (7,5) (8,5) (minor
    coordinate k/3 rounded half up), listed here by hand."""
    rng = np.random.default_rng(8)
    h, w = 9, 12
    idx = rng.integers(0, SIG.size, size=(h, w)).astype(np.uint8)
    v = np.array([3.0, 1.0]) / math.sqrt(10.0)
    H = -np.outer(v, v)
    out = oracle.postprocess_core(idx, np.ones((h, w)), *_fields(h, w, H[0, 0], H[0, 1], H[1, 1]), SIG, 0.2, 3)
    cells = [(3, 2), (3, 3), (4, 4), (4, 5), (4, 6), (5, 7), (5, 8)]  # (y, x)
    assert out[4, 5] == _nearest(np.mean([SIG[idx[y, x]] for y, x in cells]))


def test_index_outside_the_set_ends_the_walk(oracle):
    h, w = 3, 9
    idx = np.full((h, w), 1, dtype=np.uint8)
    idx[:, 0:3] = 3
    idx[:, 4] = 7  # not a scale of the set: kept, and it cuts the rows at x = 4
    out = oracle.postprocess_core(idx, np.ones((h, w)), *_fields(h, w, -1, 0, 0), SIG, 0.2, 100)
    assert np.all(out[:, 4] == 7)
    assert np.all(out[:, 0:4] == _nearest(SIG[[3, 3, 3, 1]].mean()))
    assert np.all(out[:, 5:] == 1)
