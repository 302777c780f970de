"""GPU parity: every stage of the CUDA path against the FP64 oracle, element by
element, on the same seeded inputs (float32 values; the oracle reads them
upcast).  Tolerances, and where they come from:

  * FED cycle / whole filter: max-abs <= 1e-4 on [0, 1]-scale images.  FP32
    rounding of one step is ~1e-7 relative; the kappa ordering bounds its growth
    over a cycle by A(kappa) ~ 10 (the FP32 experiment gave ~3e-7).
  * V map: max-abs <= 1e-4; sigma* agreement >= 99 %, and every disagreement
    must be a near-tie of the oracle's own V values.
  * tensor field: mu and the action of D on symmetric matrices to 1e-4.
"""
import math

import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4, synth

pytestmark = pytest.mark.gpu

TOL_U = 1e-4


def _np(t, w):
    return t[..., :w].cpu().numpy() if t.dim() == 2 else t[:, :w].cpu().numpy()


def _ridges():
    img, _ = synth.ridges_128(1000)
    wl = synth.WORKLOADS["ridges_128"]
    return img, wl


def _D_action(t):
    """3x3 matrix of T = D : h on (hxx, hxy, hyy), per pixel, from (cos2t, sin2t, mu1, mu2)."""
    C, S, m1, m2 = t
    m3 = 0.5 * (m1 + m2)
    out = []
    for h in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)):
        hxx, hxy, hyy = h
        sh, dh = 0.5 * (hxx + hyy), 0.5 * (hxx - hyy)
        h11 = sh + C * dh + S * hxy
        h22 = sh - C * dh - S * hxy
        h12 = C * hxy - S * dh
        t11, t22, t12 = m1 * h11, m2 * h22, m3 * h12
        st, dt = 0.5 * (t11 + t22), 0.5 * (t11 - t22)
        out += [st + C * dt - S * t12, S * dt + C * t12, st - C * dt + S * t12]
    return np.stack(out)


def _random_tensor(rng, h, w):
    th = rng.uniform(-math.pi, math.pi, size=(h, w))
    mu = rng.uniform(0.0, 1.0, size=(2, h, w))
    return np.stack([np.cos(2 * th), np.sin(2 * th), mu[0], mu[1]]).astype(np.float32)


def _tensor_to_device(t, w):
    import torch
    _, h, _ = t.shape
    buf = fd4.empty_image(h, w, channels=4)
    buf[:, :w, :] = torch.from_numpy(np.ascontiguousarray(np.moveaxis(t, 0, -1))).cuda()
    return buf


@pytest.fixture(params=[(1, 0, 0), (2, 64, 2), (2, 64, 1), (2, 32, 2), (2, 32, 1), (3, 0, 0), (4, 64, 2),
                        (4, 64, 1), (4, 32, 2), (4, 32, 1)],
                ids=["step", "fuse2-r64-q2", "fuse2-r64-q1", "fuse2-r32-q2", "fuse2-r32-q1", "fuse3",
                     "fuse4-r64-q2", "fuse4-r64-q1", "fuse4-r32-q2", "fuse4-r32-q1"])
def fed_variant(request):
    """FED kernel schedule (fd4_fed_cycle_sched): one launch per step, 3 steps
    per launch on the scalar kernel, or 2 / 4 steps per launch on the TMA
    quad kernel with 64- or 32-row regions and 1 or 2 quads per thread (the
    periodic boundary runs the scalar kernel for 2 and 4 steps)."""
    return request.param


@pytest.mark.parametrize("shape,boundary,n", [((128, 128), 0, 20), ((53, 37), 0, 20), ((61, 130), 0, 19),
                                              ((32, 40), 1, 20), ((3, 3), 0, 5), ((5, 7), 1, 7),
                                              ((260, 97), 0, 25)])
def test_fed_cycle_random_tensor(oracle, fed_variant, shape, boundary, n):
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    h, w = shape
    u0 = rng.random((h, w)).astype(np.float32)
    t = _random_tensor(rng, h, w)
    tau, _, _ = oracle.fed_taus(n * (n + 1) * 0.05 / 3, 1, 0.05, n=n)
    ref = oracle.fed_cycle(u0, t, tau, boundary)
    u = fd4.to_device(u0)
    fd4.fed_cycle(u, w, _tensor_to_device(t, w), tau, boundary, sched=fed_variant)
    got = _np(u, w)
    assert np.abs(got - ref).max() <= TOL_U
    # the padding columns are never written
    assert float(u[:, w:].abs().max()) == 0.0 if u.shape[1] > w else True


def test_fed_single_step_equals_oracle_operator(oracle, fed_variant):
    rng = np.random.default_rng(1)
    h, w = 70, 90
    u0 = rng.random((h, w)).astype(np.float32)
    t = _random_tensor(rng, h, w)
    ref = u0 - oracle.apply_P(u0, t) / 17.0
    u = fd4.to_device(u0)
    fd4.fed_cycle(u, w, _tensor_to_device(t, w), [1.0 / 17.0], sched=fed_variant)
    assert np.abs(_np(u, w) - ref).max() <= 2e-6


def test_biharmonic_mode_periodic(oracle, fed_variant):
    h, w = 32, 40
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    kx, ky = 2 * math.pi * 3 / w, 2 * math.pi * 2 / h
    mode = (0.5 + 0.25 * np.cos(kx * x + ky * y)).astype(np.float32)
    ident = np.stack([np.ones((h, w)), np.zeros((h, w)), np.ones((h, w)), np.ones((h, w))]).astype(np.float32)
    tau, _, _ = oracle.fed_taus(10 * 11 * 0.05 / 3, 1, 0.05, n=10)
    p = 16 * math.sin(kx / 2) ** 4 + 2 * math.sin(kx) ** 2 * math.sin(ky) ** 2 + 16 * math.sin(ky / 2) ** 4
    expect = 0.5 + 0.25 * float(np.prod(1 - tau * p)) * np.cos(kx * x + ky * y)
    u = fd4.to_device(mode)
    fd4.fed_cycle(u, w, _tensor_to_device(ident, w), tau, fd4.PERIODIC, sched=fed_variant)
    assert np.abs(_np(u, w) - expect).max() <= 1e-5


def test_mean_is_conserved_natural_boundary(fed_variant):
    import torch
    rng = np.random.default_rng(2)
    h, w = 300, 257
    u0 = rng.random((h, w)).astype(np.float32)
    t = _random_tensor(rng, h, w)
    u = fd4.to_device(u0)
    tau, _ = fd4.fed_taus(35.0, 5, 0.05, n=20)
    fd4.fed_cycle(u, w, _tensor_to_device(t, w), tau, sched=fed_variant)
    got = u[:, :w].double()
    assert abs(float(got.mean()) - float(u0.astype(np.float64).mean())) < 2e-6
    assert bool(torch.isfinite(got).all())


def _check_selection(oracle, img, sig, mode, min_agree=0.99, tie_rel=1e-3):
    h, w = img.shape
    idx_o, vmax_o, vall_o, c_o = oracle.select_scales(img, sig, mode)
    u = fd4.to_device(img)
    idx_g, vmax_g = fd4.select_scales(u, w, sig, fd4.params(mode=mode), want_vmax=True)
    idx_g = _np(idx_g, w)
    vmax_g = _np(vmax_g, w)
    assert np.abs(vmax_g - vmax_o).max() <= 1e-4
    mism = idx_g != idx_o
    agree = 1.0 - mism.mean()
    assert agree >= min_agree, agree
    if mism.any():
        yy, xx = np.nonzero(mism)
        v_at_gpu = vall_o[idx_g[yy, xx], yy, xx]
        v_best = vall_o[idx_o[yy, xx], yy, xx]
        assert np.all(v_at_gpu >= v_best * (1 - tie_rel) - 1e-7), "non-tie scale disagreement"
    return idx_o, agree


def test_select_scales_ridges_128(oracle):
    img, wl = _ridges()
    _check_selection(oracle, img, wl["sigmas"], oracle.RIDGE)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_select_scales_tree_ragged(oracle, mode):
    img = synth.vessel_tree(2001, 203, 157, depth=4, r0=4.0)
    _check_selection(oracle, img, [1.0, 1.5, 2.2, 3.3, 5.0], mode)


def _check_tensor(oracle, img, idx, sig, mode, grad_sq=False):
    h, w = img.shape
    t_o, n_o = oracle.build_tensor(img, idx, sig, mode=mode, grad_sq=grad_sq)
    u = fd4.to_device(img)
    import torch
    idx_d = torch.zeros((h, fd4.pitch_for(w)), dtype=torch.uint8, device="cuda")
    idx_d[:, :w] = torch.from_numpy(idx).cuda()
    t_g = fd4.build_tensor(u, w, idx_d, sig, fd4.params(mode=mode, grad_norm_squared=int(grad_sq)))
    t_g = np.moveaxis(t_g[:, :w, :].cpu().numpy(), -1, 0).astype(np.float64)
    assert np.abs(t_g[2] - t_o[2]).max() <= 1e-4
    assert np.abs(t_g[3] - t_o[3]).max() <= 1e-4
    assert np.abs(_D_action(t_g) - _D_action(t_o)).max() <= 1e-4
    return t_o


def test_build_tensor_ridges_128(oracle):
    img, wl = _ridges()
    idx, _, _, _ = oracle.select_scales(img, wl["sigmas"], oracle.RIDGE)
    _check_tensor(oracle, img, idx, wl["sigmas"], oracle.RIDGE)


@pytest.mark.parametrize("mode,grad_sq", [(1, False), (2, False), (2, True)])
def test_build_tensor_tree_ragged(oracle, mode, grad_sq):
    img = synth.vessel_tree(2002, 221, 149, depth=4, r0=5.0)
    sig = list(synth.log_sigmas(1.0, 8.0, 8))
    idx, _, _, _ = oracle.select_scales(img, sig, mode)
    _check_tensor(oracle, img, idx, sig, mode, grad_sq)


@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("shape", [(600, 97), (53, 37), (300, 1000), (257, 64), (1100, 70)])
def test_tensor_strips_edges_match_oracle(oracle, shape, dense):
    """The per-scale strip kernels at their edges, against the oracle: the
    largest radius (sigma 12, R 48, whose rolling buffer is shifted in two
    pieces), strip and segment ends on ragged sizes, every scale of the set
    present in one chunk, and chunks where one scale holds most pixels."""
    h, w = shape
    rng = np.random.default_rng(h * 31 + w)
    img = synth.vessel_tree(2100 + h, w, h, depth=4, r0=4.0)
    sig = [0.75, 1.0, 1.6, 2.5, 4.0, 6.0, 9.0, 12.0]
    idx = rng.integers(0, len(sig), size=(h, w)).astype(np.uint8)
    if dense:
        idx[rng.random((h, w)) < 0.6] = 0
    _check_tensor(oracle, img, idx, sig, fd4.BOTH)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("shape", [(600, 97), (53, 37), (300, 1000)])
def test_select_strips_edges_match_oracle(oracle, shape, mode):
    """Selection by the per-scale strip kernels on ragged sizes with radii up to
    48, against the oracle (V to 1e-4, sigma* on >= 99 % with near-ties only)."""
    h, w = shape
    img = synth.vessel_tree(2200 + h, w, h, depth=4, r0=4.0)
    _check_selection(oracle, img, [0.75, 1.0, 1.6, 2.5, 4.0, 6.0, 9.0, 12.0], mode)


@pytest.mark.parametrize("shape", [(2560, 2560), (700, 97)])
def test_tensor_sparse_scales_match_oracle(oracle, shape):
    """The tensor build's strips walk only the 32 x 32 chunks that hold a
    pixel of their scale (and the rows those chunks read): scale images where
    most chunks hold scale 0 only and each other scale sits in a few scattered
    chunks -- gaps of every length between them (rolled through or refilled),
    segments without any, indices outside the set -- give the oracle's tensor.
    The 2560^2 image takes both segment lengths (512 rows for the largest
    radii, 128 for the smallest)."""
    h, w = shape
    rng = np.random.default_rng(h + w)
    img = synth.vessel_tree(2400 + h, w, h, depth=5, r0=6.0)
    sig = [0.75, 1.0, 1.6, 2.5, 4.0, 6.0, 9.0, 12.0]
    idx = np.zeros((h, w), dtype=np.uint8)
    ch, cw = (h + 31) // 32, (w + 31) // 32
    for s in range(1, len(sig) + 1):  # len(sig): an index outside the set
        for cy, cx in zip(*np.nonzero(rng.random((ch, cw)) < 0.08)):
            y = min(32 * cy + int(rng.integers(0, 30)), h - 3)
            x = min(32 * cx + int(rng.integers(0, 30)), w - 3)
            idx[y:y + 3, x:x + 3] = s
    _check_tensor(oracle, img, idx, sig, fd4.BOTH)


def test_index_outside_the_set_gives_zero_tensor_input():
    """A selected index outside the scale set (caller-given scale images only)
    zeroes N there: mu = 1 and the orientation (1, 0)."""
    import torch
    h, w = 70, 90
    img = synth.vessel_tree(2300, w, h, depth=4, r0=4.0)
    sig = [1.0, 2.0, 4.0]
    u = fd4.to_device(img)
    idx_d = torch.full((h, fd4.pitch_for(w)), len(sig), dtype=torch.uint8, device="cuda")
    t_g = fd4.build_tensor(u, w, idx_d, sig, fd4.params(mode=fd4.BOTH))
    t_g = t_g[:, :w, :].cpu().numpy()
    assert np.all(t_g[..., 2] == 1.0) and np.all(t_g[..., 3] == 1.0)
    assert np.all(t_g[..., 0] == 1.0) and np.all(t_g[..., 1] == 0.0)


def test_build_tensor_large_scales(oracle):
    img = synth.vessel_tree(2003, 131, 290, depth=4, r0=6.0)
    sig = [3.0, 6.0, 9.0, 12.0]
    idx, _, _, _ = oracle.select_scales(img, sig, oracle.BOTH)
    _check_tensor(oracle, img, idx, sig, oracle.BOTH)


def test_filter_ridges_128_end_to_end(oracle):
    """Configuration 'ridges_128': 2 cycles of 10 steps, ridge mode."""
    img, wl = _ridges()
    sig, M, n, T = wl["sigmas"], wl["M"], wl["n"], wl["T"]
    tau, _, _ = oracle.fed_taus(T, M, 0.05, n=n)
    ref, idx_o = oracle.filter_image(img, sig, tau, M, mode=oracle.RIDGE)
    u = fd4.to_device(img)
    prm = fd4.params(mode=fd4.RIDGE)
    out, idx_g = fd4.filter_image(u, 128, sig, T, M, n, prm)
    agree = float((_np(idx_g, 128) == idx_o).mean())
    import torch
    idx_in = torch.zeros_like(idx_g)
    idx_in[:, :128] = torch.from_numpy(idx_o).cuda()
    out2, _ = fd4.filter_image(u, 128, sig, T, M, n, prm, sigma_idx=idx_in)
    assert np.abs(_np(out2, 128) - ref).max() <= TOL_U
    if agree == 1.0:
        assert np.abs(_np(out, 128) - ref).max() <= TOL_U
    assert agree >= 0.99
