"""Pins of the oracle's isotropic fourth-order comparator (IFOD, Eq. 2):

  * g = 1 on a constant image, and in closed form on a quadratic one (the
    derivative kernels are exact on quadratics away from the border:
    ||H||_F^2 = a^2 + 2 b^2 + c^2 for u = a x^2/2 + b x y + c y^2/2);
  * with a huge lambda g -> 1, and the IFOD cycle equals the cycle with the
    identity tensor (the biharmonic cycle pinned in the FED tests);
  * the IFOD filter conserves the mean grey value and leaves constants alone;
  * the filter equals its composition (tensor from u^k, then the cycle).
"""
import numpy as np
import pytest

from paper_1611_06906_gb300 import synth


def test_constant_and_quadratic_images(oracle):
    t = oracle.build_tensor_ifod(np.full((20, 24), 0.3), sigma=1.0, lam=0.005)
    assert np.all(t[0] == 1.0) and np.all(t[1] == 0.0)
    assert np.allclose(t[2], 1.0, rtol=0, atol=1e-12) and np.array_equal(t[2], t[3])
    h, w = 40, 44
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    a, b, c, lam = 0.004, -0.003, 0.002, 0.005
    u = 0.5 * a * X * X + b * X * Y + 0.5 * c * Y * Y
    t = oracle.build_tensor_ifod(u, sigma=1.0, lam=lam)
    g = 1.0 / (1.0 + (a * a + 2 * b * b + c * c) / lam ** 2)
    inner = (slice(8, h - 8), slice(8, w - 8))
    assert np.abs(t[2][inner] - g).max() < 1e-9


def test_large_lambda_is_the_biharmonic_cycle(oracle):
    img = synth.vessel_tree(4900, 40, 36, depth=4, r0=3.0).astype(np.float64)
    tau, _, _ = oracle.fed_taus(10 * 11 * 0.05 / 3, 1, 0.05, n=10)
    t = oracle.build_tensor_ifod(img, sigma=1.0, lam=1e12)
    ident = np.zeros_like(t)
    ident[0] = 1.0
    ident[2] = ident[3] = 1.0
    assert np.abs(t - ident).max() < 1e-12
    a = oracle.fed_cycle(img, t, tau)
    b = oracle.fed_cycle(img, ident, tau)
    assert np.abs(a - b).max() < 1e-12


@pytest.mark.parametrize("boundary", [0, 1])
def test_filter_conserves_the_mean_and_equals_composition(oracle, boundary):
    img = synth.vessel_tree(4901, 48, 40, depth=4, r0=3.0).astype(np.float64)
    M, n = 3, 10
    tau, _, _ = oracle.fed_taus(M * n * (n + 1) * 0.05 / 3, M, 0.05, n=n)
    out = oracle.filter_ifod(img, tau, M, sigma=1.0, lam=0.005, boundary=boundary)
    assert abs(out.mean() - img.mean()) < 1e-12
    u = img.copy()
    for _ in range(M):
        u = oracle.fed_cycle(u, oracle.build_tensor_ifod(u, 1.0, 0.005), tau, boundary=boundary)
    assert np.array_equal(out, u)
    const = oracle.filter_ifod(np.full((16, 18), 0.7), tau, M)
    assert np.abs(const - 0.7).max() < 1e-13
