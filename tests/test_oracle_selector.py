"""Pins of the FP64 oracle of the learned scale selector: the forward
convolution against scipy's correlation (a library routine used independently
of the oracle's tap loop), and every gradient against central finite
differences of the oracle's own loss."""
import numpy as np
import pytest

from oracle import selector_oracle as S


def test_conv_forward_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(13, 17, 3))
    for d in (1, 2, 4):
        W = rng.normal(size=(3, 3, 2, 3))
        b = rng.normal(size=2)
        out = S.conv_forward(x, W, b, d)
        for co in range(2):
            ref = np.full(x.shape[:2], b[co])
            for ci in range(3):
                k = np.zeros((2 * d + 1, 2 * d + 1))
                k[::d, ::d] = W[:, :, co, ci]
                ref += ndimage.correlate(x[:, :, ci], k, mode="constant", cval=0.0)
            assert np.abs(out[:, :, co] - ref).max() < 1e-12


def _tiny(rng):
    return S.init_params(rng, channels=(1, 3, 3, 3, 4))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = _tiny(rng)
    params = [(W, rng.normal(0, 0.1, size=b.shape)) for W, b in params]
    img = rng.normal(size=(9, 11))
    labels = rng.integers(0, 4, size=(9, 11))
    loss, grads = S.loss_and_grads(img, labels, params)
    eps = 1e-6
    for l in range(4):
        W, b = params[l]
        for idx in [(0, 0, 0, 0), (1, 2, 1, 0), (2, 1, W.shape[2] - 1, W.shape[3] - 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += eps
            Wm[idx] -= eps
            pp = list(params)
            pp[l] = (Wp, b)
            lp, _ = S.loss_and_grads(img, labels, pp)
            pp[l] = (Wm, b)
            lm, _ = S.loss_and_grads(img, labels, pp)
            num = (lp - lm) / (2 * eps)
            assert abs(num - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(num))
        for c in range(b.size):
            bp, bm = b.copy(), b.copy()
            bp[c] += eps
            bm[c] -= eps
            pp = list(params)
            pp[l] = (W, bp)
            lp, _ = S.loss_and_grads(img, labels, pp)
            pp[l] = (W, bm)
            lm, _ = S.loss_and_grads(img, labels, pp)
            assert abs((lp - lm) / (2 * eps) - grads[l][1][c]) <= 1e-6


def test_input_gradient_of_one_layer():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(7, 8, 2))
    W = rng.normal(size=(3, 3, 3, 2))
    g = rng.normal(size=(7, 8, 3))
    gx, _, _ = S.conv_backward(x, W, 2, g)
    eps = 1e-6
    for idx in [(0, 0, 0), (3, 4, 1), (6, 7, 0), (2, 5, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        num = ((S.conv_forward(xp, W, np.zeros(3), 2) - S.conv_forward(xm, W, np.zeros(3), 2)) * g).sum() / (2 * eps)
        assert abs(num - gx[idx]) < 1e-7


def test_loss_of_uniform_logits():
    """Zero weights give uniform probabilities: loss = log(n_bins)."""
    params = [(np.zeros((3, 3, co, ci)), np.zeros(co)) for ci, co in ((1, 4), (4, 4), (4, 4), (4, 8))]
    loss, _ = S.loss_and_grads(np.ones((5, 6)), np.zeros((5, 6), dtype=int), params)
    assert abs(loss - np.log(8)) < 1e-14
