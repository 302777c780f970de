"""FP64 CPU oracle of the learned scale selector.

TEST INFRASTRUCTURE ONLY (imported by tests/ and never by the library).

The paper selects the scale per pixel with the vesselness argmax (Sec. 3.3);
the learned selector is an addition of this project that predicts that
argmax with a small convolutional network, checked against the plain sweep.
Network (all 3 x 3 correlations, zero padding, "same" output size):

    layer l: out[y, x, co] = b[co] + sum_{ky, kx, ci} W[ky, kx, co, ci] in[y + d (ky - 1), x + d (kx - 1), ci]
    dilations d = 1, 2, 4, 8; channels 1 -> 32 -> 32 -> 32 -> n_bins;
    ReLU after layers 1-3; softmax over the n_bins outputs;
    loss = mean over pixels of -log p[label].

Everything is plain numpy loops over taps in float64; the gradients are the
chain rule written out layer by layer.  Activations are (H, W, C) arrays.
"""
from __future__ import annotations

import numpy as np

DILATIONS = (1, 2, 4, 8)


def conv_forward(x, W, b, d):
    """x: (H, W, Ci); W: (3, 3, Co, Ci); b: (Co,) -> (H, W, Co)."""
    H, Wd, Ci = x.shape
    Co = W.shape[2]
    xp = np.zeros((H + 2 * d, Wd + 2 * d, Ci))
    xp[d:d + H, d:d + Wd] = x
    out = np.broadcast_to(b, (H, Wd, Co)).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            patch = xp[ky * d:ky * d + H, kx * d:kx * d + Wd, :]  # in[y + d(ky-1), x + d(kx-1)]
            out += patch @ W[ky, kx].T
    return out


def conv_backward(x, W, d, g):
    """Gradients of sum(g * conv_forward(x, W, b, d)) w.r.t. x, W and b."""
    H, Wd, Ci = x.shape
    xp = np.zeros((H + 2 * d, Wd + 2 * d, Ci))
    xp[d:d + H, d:d + Wd] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            patch = xp[ky * d:ky * d + H, kx * d:kx * d + Wd, :]
            gW[ky, kx] = g.reshape(-1, g.shape[2]).T @ patch.reshape(-1, Ci)
            gxp[ky * d:ky * d + H, kx * d:kx * d + Wd, :] += g @ W[ky, kx]
    gx = gxp[d:d + H, d:d + Wd]
    gb = g.sum(axis=(0, 1))
    return gx, gW, gb


def forward(img, params):
    """img: (H, W) -> (list of layer inputs, pre-activations, logits)."""
    a = img[:, :, None].astype(np.float64)
    inputs, pre = [], []
    for l, (W, b) in enumerate(params):
        inputs.append(a)
        z = conv_forward(a, W, b, DILATIONS[l])
        pre.append(z)
        a = np.maximum(z, 0.0) if l < len(params) - 1 else z
    return inputs, pre, a


def softmax(z):
    m = z.max(axis=-1, keepdims=True)
    e = np.exp(z - m)
    return e / e.sum(axis=-1, keepdims=True)


def loss_and_grads(img, labels, params):
    """Mean cross-entropy over pixels and its gradients (list of (gW, gb))."""
    inputs, pre, logits = forward(img, params)
    p = softmax(logits)
    H, Wd, C = logits.shape
    npx = H * Wd
    lab = labels.astype(np.int64)
    loss = -np.log(np.take_along_axis(p, lab[:, :, None], axis=-1)).sum() / npx
    g = p.copy()
    np.put_along_axis(g, lab[:, :, None], np.take_along_axis(g, lab[:, :, None], axis=-1) - 1.0, axis=-1)
    g /= npx
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        if l < len(params) - 1:
            g = g * (pre[l] > 0)
        gx, gW, gb = conv_backward(inputs[l], params[l][0], DILATIONS[l], g)
        grads[l] = (gW, gb)
        g = gx
    return loss, grads


def init_params(rng, channels=(1, 32, 32, 32, 8)):
    params = []
    for ci, co in zip(channels[:-1], channels[1:]):
        std = np.sqrt(2.0 / (9 * ci))
        params.append((rng.normal(0.0, std, size=(3, 3, co, ci)), np.zeros(co)))
    return params
