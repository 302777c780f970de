"""Pins of the oracle's vesselness scale selection (Sec. 3.3, Eq. 9).

Closed forms used:
  * a Gaussian ridge exp(-d^2/2w^2) blurred by G_sigma has centre curvature
    -w / (w^2 + sigma^2)^(3/2); with R_B = 0 there, V is monotone in
    S = sigma^2 w / (w^2 + sigma^2)^(3/2), so the selected scale is the argmax of
    that function over the scale set (maximum at sigma = sqrt(2) w);
  * an isotropic Gaussian blob has nu1 = nu2 at its centre, so R_B = 1 and
    V = exp(-1/(2 beta^2)) (1 - exp(-S^2/(2 c^2))) with S = sqrt(2) sigma^2 |u_xx|.
"""
import math

import numpy as np
import pytest

from paper_1611_06906_gb300 import synth


def _width_scale(w_r, sigmas):
    s = np.asarray(sigmas, dtype=np.float64)
    return s * s * w_r / (w_r * w_r + s * s) ** 1.5


@pytest.mark.parametrize("w_r,expect", [(1.5, 2.0), (4.0, 4.0)])
def test_width_scale_relation_paper_scale_set(oracle, w_r, expect):
    sig = [1.0, 1.5, 2.0, 3.0, 4.0]
    f = _width_scale(w_r, sig)
    assert sig[int(np.argmax(f))] == expect
    u = synth.ridge_profile(161, 81, w_r)
    idx, vmax, vall, c = oracle.select_scales(u, sig, oracle.RIDGE)
    centre = idx[40, 40:120]
    assert np.all(centre == sig.index(expect))


def test_width_scale_relation_dense_scale_set(oracle):
    """On a fine scale grid the centre-line scale sits at the analytic optimum sqrt(2) w."""
    w_r = 2.0
    sig = list(np.arange(1.0, 6.01, 0.25))
    f = _width_scale(w_r, sig)
    ok = {i for i, v in enumerate(f) if v >= f.max() * (1 - 2e-3)}
    u = synth.ridge_profile(161, 101, w_r, angle=0.3)
    idx, _, _, _ = oracle.select_scales(u, sig, oracle.RIDGE)
    assert int(idx[50, 80]) in ok
    assert abs(sig[int(idx[50, 80])] - math.sqrt(2) * w_r) <= 0.25


def test_polarity(oracle):
    sig = [1.0, 2.0, 3.0]
    ridge = synth.ridge_profile(81, 61, 2.0)
    valley = -ridge
    for img, good, bad in ((ridge, oracle.RIDGE, oracle.VALLEY), (valley, oracle.VALLEY, oracle.RIDGE)):
        _, vg, _, _ = oracle.select_scales(img, sig, good)
        _, vb, _, _ = oracle.select_scales(img, sig, bad)
        _, vboth, _, _ = oracle.select_scales(img, sig, oracle.BOTH)
        assert vg[30, 40] > 0.5
        assert vb[30, 40] == 0.0
        assert abs(vboth[30, 40] - vg[30, 40]) < 1e-15


def test_isotropic_blob_closed_form(oracle):
    w_b, sigma, c = 3.0, 2.0, 0.05
    n = 81
    y, x = np.mgrid[0:n, 0:n].astype(np.float64) - 40
    u = np.exp(-(x * x + y * y) / (2 * w_b * w_b))
    idx, vmax, vall, c_used = oracle.select_scales(u, [sigma], oracle.RIDGE, beta=0.5, c=c)
    assert c_used == c
    s2 = w_b * w_b + sigma * sigma
    S = math.sqrt(2) * sigma * sigma * w_b * w_b / (s2 * s2)
    V = math.exp(-1 / (2 * 0.25)) * (1 - math.exp(-S * S / (2 * c * c)))
    assert abs(vall[0, 40, 40] - V) < 1e-2 * V


def test_auto_c_is_half_the_global_maximum_of_S(oracle):
    """c = max(S)/2 over all scales and pixels; S^2 = sigma^4 ||H||_F^2."""
    img, _ = synth.ridges_128(1000)
    sig = [1.0, 2.0, 4.0]
    _, _, vall, c_used = oracle.select_scales(img, sig, oracle.RIDGE)
    smax = 0.0
    for s in sig:
        _, _, uxx, uxy, uyy = oracle.derivatives(img.astype(np.float64), s)
        S = s * s * np.sqrt(uxx ** 2 + 2 * uxy ** 2 + uyy ** 2)
        smax = max(smax, S.max())
    assert abs(c_used - 0.5 * smax) < 1e-12 * smax
    # passing that c explicitly reproduces the selection
    _, _, vall2, _ = oracle.select_scales(img, sig, oracle.RIDGE, c=c_used)
    assert np.array_equal(vall, vall2)


def test_range_and_transpose_invariance(oracle):
    img, _ = synth.ridges_128(1001)
    sig = [1.0, 1.5, 2.0, 3.0, 4.0]
    idx, vmax, vall, _ = oracle.select_scales(img, sig, oracle.RIDGE)
    assert vall.min() >= 0.0 and vall.max() < 1.0
    assert np.array_equal(vmax, vall.max(axis=0))
    idx_t, vmax_t, _, _ = oracle.select_scales(img.T.copy(), sig, oracle.RIDGE)
    idx_r, vmax_r, _, _ = oracle.select_scales(np.rot90(img).copy(), sig, oracle.RIDGE)
    assert np.abs(vmax_t - vmax.T).max() < 1e-12
    assert np.abs(vmax_r - np.rot90(vmax)).max() < 1e-12
    # the argmax may only move between scales whose V agree to rounding
    for got, ref in ((idx_t, idx.T), (idx_r, np.rot90(idx))):
        diff = got != ref
        assert diff.mean() < 1e-3


def test_ties_go_to_the_smallest_scale(oracle):
    u = np.zeros((20, 20))
    idx, vmax, _, c = oracle.select_scales(u, [1.0, 2.0, 3.0], oracle.BOTH)
    assert c == 0.0 and np.all(idx == 0) and np.all(vmax == 0.0)
    # equal V at two scales (two copies of one scale) -> the first one
    img, _ = synth.ridges_128(1002)
    idx2, _, vall, _ = oracle.select_scales(img, [2.0, 2.0, 3.0], oracle.BOTH)
    assert np.array_equal(vall[0], vall[1]) and not np.any(idx2 == 1)
