"""Pins of the oracle's Gaussian-derivative scale space (Sec. 3.1, Eq. 6).

The paper fixes u_sigma = u * G_sigma and its derivatives; it leaves the
discretisation open.  These tests pin the oracle to what the mathematics fixes:
the continuum kernels, exactness on polynomials, separability, the analytic
Gaussian-profile ridge under Gaussian blur, and symmetry under transposition."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("sigma", [0.75, 1.0, 2.5, 6.0])
def test_kernel_moments(oracle, sigma):
    w0, w1, w2 = oracle.gauss_kernels(sigma)
    r = oracle.gauss_radius(sigma)
    assert r == math.ceil(4 * sigma)
    k = np.arange(-r, r + 1, dtype=np.float64)
    assert abs(w0.sum() - 1) < 1e-14
    assert np.allclose(w0, w0[::-1], atol=0) and np.allclose(w2, w2[::-1], atol=1e-18)
    assert np.allclose(w1, -w1[::-1], atol=1e-18)
    # a ramp differentiates to 1, a parabola x^2/2 to 1 (correlation weights)
    assert abs((w1 * k).sum() - 1) < 1e-13
    assert abs(w2.sum()) < 1e-13
    assert abs((w2 * k * k / 2).sum() - 1) < 1e-12
    # smoothing kernel variance is sigma^2 up to the truncation at 4 sigma
    assert abs((w0 * k * k).sum() - sigma ** 2) < 2e-3 * sigma ** 2 + 1e-3


def test_kernels_match_continuum_for_large_sigma(oracle):
    sigma = 6.0
    w0, w1, w2 = oracle.gauss_kernels(sigma)
    r = oracle.gauss_radius(sigma)
    k = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-k * k / (2 * sigma ** 2)) / (math.sqrt(2 * math.pi) * sigma)
    # correlation with +k g(k)/sigma^2 equals convolution with G'
    g1 = k / sigma ** 2 * g
    g2 = (k * k / sigma ** 4 - 1 / sigma ** 2) * g
    assert np.abs(w0 - g).max() < 1e-4 * g.max()
    # the moment normalisation (exactness on x and x^2/2) absorbs the 4-sigma
    # truncation, which moves the derivative kernels by well under 1 %
    assert np.abs(w1 - g1).max() < 1e-2 * np.abs(g1).max()
    assert np.abs(w2 - g2).max() < 1e-2 * np.abs(g2).max()


@pytest.mark.parametrize("sigma", [1.0, 2.0, 3.3])
def test_polynomials_differentiate_exactly(oracle, sigma):
    h, w = 70, 90
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    a, b, c, d, e, f = 0.3, -0.02, 0.013, 0.0021, -0.0017, 0.0009
    u = a + b * x + c * y + d * x * x + e * x * y + f * y * y
    ux, uy, uxx, uxy, uyy = oracle.derivatives(u, sigma)
    r = oracle.gauss_radius(sigma)
    sl = (slice(r, h - r), slice(r, w - r))
    assert np.abs(ux[sl] - (b + 2 * d * x + e * y)[sl]).max() < 1e-11
    assert np.abs(uy[sl] - (c + e * x + 2 * f * y)[sl]).max() < 1e-11
    assert np.abs(uxx[sl] - 2 * d).max() < 1e-12
    assert np.abs(uxy[sl] - e).max() < 1e-12
    assert np.abs(uyy[sl] - 2 * f).max() < 1e-12


@pytest.mark.parametrize("shape,sigma", [((13, 17), 1.5), ((5, 7), 2.0)])
def test_separable_equals_direct_2d_sum(oracle, shape, sigma):
    """Separable evaluation == direct double sum, including mirror folding when r > size."""
    rng = np.random.default_rng(7)
    u = rng.random(shape)
    outs = oracle.derivatives(u, sigma)
    orders = [(1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    for o, (ox, oy) in zip(outs, orders):
        ref = oracle.derivative_direct(u, sigma, ox, oy)
        assert np.abs(o - ref).max() < 1e-13


def test_transpose_swaps_derivatives(oracle):
    rng = np.random.default_rng(3)
    u = rng.random((31, 23))
    ux, uy, uxx, uxy, uyy = oracle.derivatives(u, 1.7)
    tx, ty, txx, txy, tyy = oracle.derivatives(u.T.copy(), 1.7)
    for a, b in ((ux, ty), (uy, tx), (uxx, tyy), (uxy, txy), (uyy, txx)):
        assert np.abs(a.T - b).max() < 1e-13


@pytest.mark.parametrize("w_r,sigma", [(2.0, 3.0), (4.0, 2.0)])
def test_analytic_gaussian_ridge(oracle, w_r, sigma):
    """A ridge exp(-d^2/2w^2) blurred by G_sigma is w/s exp(-d^2/2s^2), s^2 = w^2 + sigma^2.

    Its second derivative across the ridge at the centre line is -w/s^3."""
    from paper_1611_06906_gb300 import synth

    u = synth.ridge_profile(121, 61, w_r)  # ridge along x, centred at row 30
    ux, uy, uxx, uxy, uyy = oracle.derivatives(u, sigma)
    s = math.sqrt(w_r ** 2 + sigma ** 2)
    c = 30
    yy = np.arange(61, dtype=np.float64) - c
    prof = w_r / s * np.exp(-yy ** 2 / (2 * s * s))
    dprof = -yy / s ** 2 * prof
    d2prof = (yy ** 2 / s ** 4 - 1 / s ** 2) * prof
    col = 60  # far from the left/right borders: the ridge is x-invariant there
    inner = slice(c - 8, c + 9)
    # sampled, 4-sigma-truncated kernels: within 1 % of the continuum
    assert np.abs(uyy[inner, col] - d2prof[inner]).max() < 1e-2 * abs(d2prof[c])
    assert np.abs(uy[inner, col] - dprof[inner]).max() < 1e-2 * np.abs(dprof).max()
    assert np.abs(uxx[inner, col]).max() < 1e-12
    assert np.abs(uxy[inner, col]).max() < 1e-12
    assert abs(uyy[c, col] + w_r / s ** 3) < 1e-2 * w_r / s ** 3
