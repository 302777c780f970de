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


# --- the border extension of every Gaussian sum ------------------------------
# Sec. 3.1 only writes u_sigma = u * G_sigma; the oracle extends the image by
# the half-sample symmetric fold (u[-1-i] = u[i], u[n+i] = u[n-1-i], period 2n
# for any offset).  These pins check that fold against two library routines
# that implement it independently and against values worked out by hand, so
# that a whole-sample fold (u[-1] = u[1]) or a wrong period fails.

def _separable_lib(u, wx, wy, mode):
    import scipy.ndimage as ndi
    a = ndi.correlate1d(u, wx, axis=1, mode=mode)
    return ndi.correlate1d(a, wy, axis=0, mode=mode)


def _direct_padded(u, wx, wy, r):
    """Direct 2-D correlation on numpy's 'symmetric' padding (edge value repeated)."""
    p = np.pad(u, r, mode="symmetric")
    h, w = u.shape
    out = np.empty((h, w))
    k2 = wy[:, None] * wx[None, :]
    for y in range(h):
        for x in range(w):
            out[y, x] = (k2 * p[y:y + 2 * r + 1, x:x + 2 * r + 1]).sum()
    return out


@pytest.mark.parametrize("shape,sigma", [((5, 7), 2.0), ((13, 17), 1.5), ((4, 4), 1.25), ((3, 9), 3.0)])
def test_border_fold_matches_library_reflect(oracle, shape, sigma):
    """All five derivatives on random images equal scipy.ndimage's 'reflect'
    mode (d c b a | a b c d) and numpy's 'symmetric' padding, including radii
    larger than the image (the fold repeats with period 2n)."""
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    u = rng.random(shape)
    w0, w1, w2 = oracle.gauss_kernels(sigma)
    r = oracle.gauss_radius(sigma)
    pairs = [(w1, w0), (w0, w1), (w2, w0), (w1, w1), (w0, w2)]
    outs = oracle.derivatives(u, sigma)
    for o, (wx, wy) in zip(outs, pairs):
        assert np.abs(o - _separable_lib(u, wx, wy, "reflect")).max() < 1e-14
        assert np.abs(o - _direct_padded(u, wx, wy, r)).max() < 1e-14
    # the whole-sample fold (scipy's 'mirror': c b | a b c) is a different
    # extension and must not match at the border
    worst = max(np.abs(o - _separable_lib(u, wx, wy, "mirror")).max() for o, (wx, wy) in zip(outs, pairs))
    assert worst > 1e-3


def test_border_fold_hand_worked_4_pixels(oracle):
    """sigma = 1/4 gives radius 1, where the normalised kernels are exactly the
    central differences (-1/2, 0, 1/2) and (1, -2, 1).  On rows [0, 1, 3, 7]
    (constant down the columns) the half-sample fold u[-1] = u[0], u[4] = u[3]
    gives u_x = [1/2, 3/2, 3, 2] and u_xx = [1, 1, 2, -4]; a whole-sample fold
    would give u_x[0] = 0, u_xx[0] = 2."""
    w0, w1, w2 = oracle.gauss_kernels(0.25)
    assert np.allclose(w1, [-0.5, 0.0, 0.5], atol=1e-15)
    assert np.allclose(w2, [1.0, -2.0, 1.0], atol=1e-12)
    u = np.tile(np.array([0.0, 1.0, 3.0, 7.0]), (4, 1))
    ux, uy, uxx, uxy, uyy = oracle.derivatives(u, 0.25)
    for row in range(4):
        assert np.allclose(ux[row], [0.5, 1.5, 3.0, 2.0], atol=1e-12)
        assert np.allclose(uxx[row], [1.0, 1.0, 2.0, -4.0], atol=1e-11)
    assert np.abs(uy).max() < 1e-15 and np.abs(uxy).max() < 1e-15 and np.abs(uyy).max() < 1e-11
    # the same along y: rows y = 0..3 hold 0, 1, 3, 7 (a 4 x 3 image)
    v = np.tile(np.array([[0.0], [1.0], [3.0], [7.0]]), (1, 3))
    vx, vy, vxx, vxy, vyy = oracle.derivatives(v, 0.25)
    for col in range(3):
        assert np.allclose(vy[:, col], [0.5, 1.5, 3.0, 2.0], atol=1e-12)
        assert np.allclose(vyy[:, col], [1.0, 1.0, 2.0, -4.0], atol=1e-11)
