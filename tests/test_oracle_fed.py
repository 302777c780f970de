"""Pins of the oracle's discrete operator and FED schedule (Sec. 3.4 Eq. 10-20,
Sec. 3.5 Eq. 21-23).

  * the cycle lengths the paper's own parameter sets imply (tests/golden);
  * sum_i tau_i = T / M, and the cycle polynomial stays within [-1, 1] on the
    stable range (the defining property of FED);
  * P = L^T D L built densely from the oracle on tiny grids: symmetric, positive
    semi-definite, P 1 = 0 (constants stay constant), 1^T P = 0 (the mean is
    conserved), ||P|| <= ||L||^2 <= 34;
  * with D the identity on a periodic grid P is the discrete biharmonic operator,
    whose Fourier symbol is 16 sin^4(kx/2) + 2 sin^2 kx sin^2 ky + 16 sin^4(ky/2);
    a FED cycle multiplies each mode by prod_i (1 - tau_i p(k)), and low modes
    decay like exp(-t |k|^4);
  * a FED cycle equals its own step-by-step product of (I - tau_i P) in any order.
"""
import math
import os

import numpy as np
import pytest

from paper_1611_06906_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fed_cycle_lengths.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        T, M, tmax, n = line.split()[:4]
        rows.append((float(T), int(M), float(tmax), int(n)))
    return rows


@pytest.mark.parametrize("T,M,tmax,n", _golden_rows())
def test_cycle_length_from_paper_parameters(oracle, T, M, tmax, n):
    tau, kappa, amp = oracle.fed_taus(T, M, tmax)
    assert tau.size == n
    assert abs(tau.sum() - T / M) < 1e-12 * T / M


@pytest.mark.parametrize("n,M", [(10, 2), (20, 5), (25, 10), (7, 1)])
def test_tau_sum_order_and_stability(oracle, n, M):
    T = M * n * (n + 1) * 0.05 / 3
    tau_nat, k1, _ = oracle.fed_taus(T, M, 0.05, n=n, kappa=1)
    tau, kappa, amp = oracle.fed_taus(T, M, 0.05, n=n, kappa=0)
    assert k1 == 1 and np.all(np.diff(tau_nat) > 0)
    assert abs(tau.sum() - T / M) < 1e-12 * T / M
    assert np.allclose(np.sort(tau), tau_nat, rtol=0, atol=0)
    assert math.gcd(kappa, n) == 1
    # stable range of the cycle: p in [0, 2 / tau'] with tau' = 3T / (M (n^2 + n)) = tau_max
    p = np.linspace(0.0, 2.0 / 0.05, 20001)
    poly = np.prod(1.0 - np.outer(tau, p), axis=0)
    assert np.abs(poly).max() <= 1.0 + 1e-9
    assert amp >= 1.0


def test_unstable_schedule_is_rejected(oracle):
    with pytest.raises(oracle.UnstableTau):
        oracle.fed_taus(35.0, 5, 0.05, n=10)


def _dense_P(oracle, tensor, boundary):
    _, h, w = tensor.shape
    P = np.zeros((h * w, h * w))
    for j in range(h * w):
        e = np.zeros(h * w)
        e[j] = 1.0
        P[:, j] = oracle.apply_P(e.reshape(h, w), tensor, boundary).ravel()
    return P


def _random_tensor(rng, h, w):
    th = rng.uniform(-math.pi, math.pi, size=(h, w))
    mu = rng.uniform(0.0, 1.0, size=(2, h, w))
    return np.stack([np.cos(2 * th), np.sin(2 * th), mu[0], mu[1]])


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_dense_operator_invariants(oracle, boundary, seed):
    rng = np.random.default_rng(seed)
    h, w = 5, 6
    P = _dense_P(oracle, _random_tensor(rng, h, w), boundary)
    assert np.abs(P - P.T).max() < 1e-14
    ev = np.linalg.eigvalsh(P)
    assert ev.min() > -1e-12
    assert ev.max() <= 34.0
    one = np.ones(h * w)
    assert np.abs(P @ one).max() < 1e-14
    assert np.abs(one @ P).max() < 1e-14
    # one explicit step with tau <= 1/17 does not increase the l2 norm
    u = rng.normal(size=h * w)
    assert np.linalg.norm(u - P @ u / 17.0) <= np.linalg.norm(u) * (1 + 1e-14)


def test_identity_tensor_norm_bound_is_reached_periodic(oracle):
    """With D = identity on a periodic grid the spectrum is the symbol p(k), max 32."""
    h, w = 6, 8
    t = np.stack([np.ones((h, w)), np.zeros((h, w)), np.ones((h, w)), np.ones((h, w))])
    P = _dense_P(oracle, t, 1)
    ky = 2 * math.pi * np.arange(h) / h
    kx = 2 * math.pi * np.arange(w) / w
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    sym = 16 * np.sin(KX / 2) ** 4 + 2 * np.sin(KX) ** 2 * np.sin(KY) ** 2 + 16 * np.sin(KY / 2) ** 4
    assert np.abs(np.sort(np.linalg.eigvalsh(P)) - np.sort(sym.ravel())).max() < 1e-12
    assert abs(sym.max() - 32.0) < 1e-12


def test_biharmonic_fourier_decay(oracle):
    h, w = 32, 40
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    ident = np.stack([np.ones((h, w)), np.zeros((h, w)), np.ones((h, w)), np.ones((h, w))])
    n, M = 10, 1
    T = n * (n + 1) * 0.05 / 3
    tau, _, _ = oracle.fed_taus(T, M, 0.05, n=n)
    for mx, my in ((1, 0), (0, 1), (1, 1), (2, 1), (3, 2), (7, 5), (20, 16)):
        kx, ky = 2 * math.pi * mx / w, 2 * math.pi * my / h
        mode = np.cos(kx * x + ky * y + 0.3)
        p = 16 * math.sin(kx / 2) ** 4 + 2 * math.sin(kx) ** 2 * math.sin(ky) ** 2 + 16 * math.sin(ky / 2) ** 4
        assert np.abs(oracle.apply_P(mode, ident, 1) - p * mode).max() < 1e-12
        mult = float(np.prod(1.0 - tau * p))
        out = oracle.fed_cycle(mode, ident, tau, 1)
        assert np.abs(out - mult * mode).max() < 1e-11
        k2 = kx * kx + ky * ky
        if k2 <= 0.09:
            # p = |k|^4 + O(|k|^6); the cycle polynomial is 1 - t p + O((sum tau_i^2) p^2)
            bound = T * k2 ** 3 + (tau ** 2).sum() * k2 ** 4 + (T * k2 * k2) ** 2
            assert abs(mult - math.exp(-T * k2 * k2)) <= bound


def test_cycle_equals_step_by_step_product(oracle):
    rng = np.random.default_rng(5)
    h, w = 6, 7
    t = _random_tensor(rng, h, w)
    P = _dense_P(oracle, t, 0)
    u = rng.random((h, w))
    tau, kappa, _ = oracle.fed_taus(20 * 21 * 0.05 / 3, 1, 0.05, n=20)
    tau_nat, _, _ = oracle.fed_taus(20 * 21 * 0.05 / 3, 1, 0.05, n=20, kappa=1)
    assert kappa != 1
    v = u.ravel().copy()
    for ti in tau_nat:  # natural order, dense matrix products
        v = v - ti * (P @ v)
    out = oracle.fed_cycle(u, t, tau, 0)
    assert np.abs(out.ravel() - v).max() < 1e-9


def test_mean_and_constants_on_a_real_workload(oracle):
    img, _ = synth.ridges_128(1000)
    wl = synth.WORKLOADS["ridges_128"]
    sig = wl["sigmas"]
    idx, _, _, _ = oracle.select_scales(img, sig, oracle.RIDGE)
    t, _ = oracle.build_tensor(img, idx, sig, mode=oracle.RIDGE)
    tau, _, _ = oracle.fed_taus(wl["T"], wl["M"], 0.05, n=wl["n"])
    u = img.astype(np.float64)
    out = oracle.fed_cycle(u, t, tau)
    assert abs(out.mean() - u.mean()) < 1e-12
    assert np.linalg.norm(out) <= np.linalg.norm(u)
    c = np.full_like(u, 0.37)
    assert np.abs(oracle.fed_cycle(c, t, tau) - 0.37).max() < 1e-13


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_operator_on_quartics_equals_continuum(oracle, seed):
    """Constant D, u a quartic: the stencils are exact, so in the interior
    P u = sum_{ij,kl} D_ijkl d_i d_j d_k d_l u (Eq. 4-5).  Terms with an odd number
    of x-derivatives change sign with the mixed stencil, so this fixes its sign
    and the coupling of D's orientation to the grid axes."""
    rng = np.random.default_rng(seed)
    h, w = 11, 13
    th = rng.uniform(-math.pi, math.pi)
    mu1, mu2 = rng.uniform(0.05, 1.0, size=2)
    D = oracle.tensor_matrix(math.cos(2 * th), math.sin(2 * th), mu1, mu2)
    t = np.stack([np.full((h, w), v) for v in (math.cos(2 * th), math.sin(2 * th), mu1, mu2)])
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    x -= 6.0
    y -= 5.0
    c = rng.normal(size=5)  # c[p] = d^p/dx^p d^(4-p)/dy^(4-p) u
    u = sum(c[p] * x ** p * y ** (4 - p) / (math.factorial(p) * math.factorial(4 - p)) for p in range(5))
    nx = [2, 1, 1, 0]  # x-derivatives in component xx, xy, yx, yy
    expect = sum(D[a, b] * c[nx[a] + nx[b]] for a in range(4) for b in range(4))
    Pu = oracle.apply_P(u, t, 0)
    assert np.abs(Pu[2:-2, 2:-2] - expect).max() < 1e-9 * max(1.0, abs(expect))
