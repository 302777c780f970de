"""Pins of the oracle's fourth-order diffusion tensor (Sec. 3.1 Eq. 6, Sec. 3.2 Eq. 7-8,
Sec. 3.4 D_i = E M E^T).

  * D_i has the eigentensors of Eq. 8 with eigenvalues mu1, mu2, (mu1+mu2)/2, 0;
    it is symmetric with norm <= 1 (Sec. 3.4);
  * on symmetric matrices D_i equals rotate-into-eigenframe, scale, rotate back
    (an independent derivation of the same map);
  * on u = g x + q (y - y0)^2 / 2 the normalised Hessian at row y0 is exactly
    diag(0, q) / sqrt(1 + g) (gradient (g, 0), Hessian diag(0, q)), which fixes
    the eigenvector, both eigenvalues and the diffusivities in every mode;
  * transposing the image maps (cos 2t, sin 2t) to (-cos 2t, sin 2t);
  * the closed form D_i H = mu3 H + q (z I + tr H R) that the FED kernel
    evaluates equals the oracle's D_i on random symmetric H.
"""
import math

import numpy as np
import pytest

from paper_1611_06906_gb300 import synth


def _vec(A):
    return np.array([A[0, 0], A[0, 1], A[1, 0], A[1, 1]])


@pytest.mark.parametrize("seed", range(6))
def test_D_eigentensors_and_norm(oracle, seed):
    rng = np.random.default_rng(seed)
    th = rng.uniform(-math.pi, math.pi)
    mu1, mu2 = rng.uniform(0.01, 1.0, size=2)
    D = oracle.tensor_matrix(math.cos(2 * th), math.sin(2 * th), mu1, mu2)
    e1 = np.array([math.cos(th), math.sin(th)])
    e2 = np.array([-math.sin(th), math.cos(th)])
    assert np.abs(D - D.T).max() < 1e-15
    for E, mu in ((np.outer(e1, e1), mu1), (np.outer(e2, e2), mu2),
                  ((np.outer(e1, e2) + np.outer(e2, e1)) / math.sqrt(2), 0.5 * (mu1 + mu2)),
                  ((np.outer(e1, e2) - np.outer(e2, e1)) / math.sqrt(2), 0.0)):
        assert np.abs(D @ _vec(E) - mu * _vec(E)).max() < 1e-14
    ev = np.sort(np.linalg.eigvalsh(D))
    assert np.abs(ev - np.sort([0.0, mu1, mu2, 0.5 * (mu1 + mu2)])).max() < 1e-14
    assert np.linalg.norm(D, 2) <= 1.0 + 1e-14


def test_D_matches_eigenframe_rotation(oracle):
    rng = np.random.default_rng(11)
    for _ in range(20):
        th = rng.uniform(-math.pi, math.pi)
        mu1, mu2 = rng.uniform(0.0, 1.0, size=2)
        hxx, hxy, hyy = rng.normal(size=3)
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        Hm = np.array([[hxx, hxy], [hxy, hyy]])
        Ht = R.T @ Hm @ R
        Tt = np.array([[mu1 * Ht[0, 0], 0.5 * (mu1 + mu2) * Ht[0, 1]],
                       [0.5 * (mu1 + mu2) * Ht[1, 0], mu2 * Ht[1, 1]]])
        T = R @ Tt @ R.T
        D = oracle.tensor_matrix(math.cos(2 * th), math.sin(2 * th), mu1, mu2)
        assert np.abs(D @ _vec(Hm) - _vec(T)).max() < 1e-14


def test_isotropic_D_is_scaled_identity_on_symmetric(oracle):
    D = oracle.tensor_matrix(0.3, math.sqrt(1 - 0.09), 0.4, 0.4)
    H = np.array([[0.7, -0.2], [-0.2, 0.1]])
    assert np.abs(D @ _vec(H) - 0.4 * _vec(H)).max() < 1e-15


@pytest.mark.parametrize("grad_sq", [False, True])
def test_normalised_hessian_closed_form(oracle, grad_sq):
    h, w, y0 = 61, 71, 30
    g, q, lam = 0.5, 0.02, 0.005
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    u = g * x + 0.5 * q * (y - y0) ** 2
    idx = np.zeros((h, w), dtype=np.uint8)
    f = 1.0 / math.sqrt(1.0 + (g * g if grad_sq else g))
    nu = q * f
    pm = 1.0 / (1.0 + nu * nu / (lam * lam))
    expect = {oracle.BOTH: (pm, 1.0), oracle.RIDGE: (1.0, 1.0), oracle.VALLEY: (pm, 1.0)}
    for mode, (m1, m2) in expect.items():
        t, nr = oracle.build_tensor(u, idx, [1.5], lam=lam, rho=0.5, mode=mode, grad_sq=grad_sq)
        px = (y0, 35)
        # G_rho adds about rho^2/2 N'' along y, a 3e-5 relative change here
        assert abs(nr[2][px] - nu) < 1e-4 * nu
        assert abs(nr[0][px]) < 1e-14 and abs(nr[1][px]) < 1e-14
        # e1 (larger eigenvalue nu > 0) is the y axis: 2 theta = pi
        assert abs(t[0][px] + 1.0) < 1e-12 and abs(t[1][px]) < 1e-12
        assert abs(t[2][px] - m1) < 2e-4 * m1 and abs(t[3][px] - m2) < 1e-14


def test_transpose_equivariance(oracle):
    img, _ = synth.ridges_128(1000)
    sig = [1.0, 2.0, 3.0]
    idx, _, _, _ = oracle.select_scales(img, sig, oracle.RIDGE)
    t, _ = oracle.build_tensor(img, idx, sig, mode=oracle.BOTH)
    tt, _ = oracle.build_tensor(img.T.copy(), idx.T.copy(), sig, mode=oracle.BOTH)
    assert np.abs(tt[0] + t[0].T).max() < 1e-9
    assert np.abs(tt[1] - t[1].T).max() < 1e-9
    assert np.abs(tt[2] - t[2].T).max() < 1e-12
    assert np.abs(tt[3] - t[3].T).max() < 1e-12
    assert t[2].min() > 0 and t[2].max() <= 1 and t[3].min() > 0 and t[3].max() <= 1


def test_per_pixel_scale_is_respected(oracle):
    img, _ = synth.ridges_128(1003)
    sig = [1.0, 2.0, 4.0]
    one = np.ones((128, 128), dtype=np.uint8)
    t_all, _ = oracle.build_tensor(img, one, sig, mode=oracle.VALLEY)
    t_single, _ = oracle.build_tensor(img, np.zeros_like(one), [2.0], mode=oracle.VALLEY)
    assert np.array_equal(t_all, t_single)


@pytest.mark.parametrize("seed", range(4))
def test_D_action_closed_form_of_the_fed_step(oracle, seed):
    """The FED kernel applies D_i to the Hessian without rotating into the
    eigenframe: with mu3 = (mu1 + mu2) / 2, q = (mu1 - mu2) / 4, R = [[c, s], [s, -c]]
    and z = R:H, D_i H = mu3 H + q (z I + tr H R), i.e. on the coefficients
    (mu3, q c, q s) that its tensor build leaves:
    Txx = mu3 hxx + Z + qc tr H, Tyy = mu3 hyy + Z - qc tr H, Txy = mu3 hxy + qs tr H,
    Z = qc (hxx - hyy) + 2 qs hxy.  Checked against the oracle's 4 x 4 D_i on
    random symmetric H, orientations and diffusivities (Sec. 3.4)."""
    rng = np.random.default_rng(100 + seed)
    for _ in range(50):
        th = rng.uniform(-math.pi, math.pi)
        mu1, mu2 = rng.uniform(0.0, 1.0, size=2)
        hxx, hxy, hyy = rng.normal(size=3)
        c, s = math.cos(2 * th), math.sin(2 * th)
        D = oracle.tensor_matrix(c, s, mu1, mu2)
        T = (D @ np.array([hxx, hxy, hxy, hyy])).reshape(2, 2)
        mu3, q = 0.5 * (mu1 + mu2), 0.25 * (mu1 - mu2)
        qc, qs = q * c, q * s
        tr, Z = hxx + hyy, qc * (hxx - hyy) + 2.0 * qs * hxy
        assert abs(T[0, 0] - (mu3 * hxx + Z + qc * tr)) < 1e-14
        assert abs(T[1, 1] - (mu3 * hyy + Z - qc * tr)) < 1e-14
        assert abs(T[0, 1] - (mu3 * hxy + qs * tr)) < 1e-14
        assert abs(T[1, 0] - T[0, 1]) < 1e-14
