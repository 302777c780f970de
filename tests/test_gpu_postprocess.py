"""Scale-image post-processing (Sec. 3.3, after Eq. 9) on the GPU: the entry
point against the FP64 oracle on the same inputs, the filters with
postprocess_scales against the oracle's filter, and the batched, graph and
two-stream paths against the per-image entry point."""
import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4, synth

pytestmark = pytest.mark.gpu

SIGMAS = [1.0, 1.6, 2.5, 4.0]
M, N = 2, 10
T = M * N * (N + 1) * 0.05 / 3
THETA = float(np.float32(0.2))  # the library compares in float32: the oracle gets the same threshold


def _gpu_post(img, idx, vmax, sig, theta=THETA):
    import torch
    h, w = img.shape
    u = fd4.to_device(img)
    pitch = u.shape[1]
    idx_d = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
    idx_d[:, :w] = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.uint8)).cuda()
    vm = torch.zeros((h, pitch), dtype=torch.float32, device="cuda")
    vm[:, :w] = torch.from_numpy(np.ascontiguousarray(vmax, dtype=np.float32)).cuda()
    fd4.postprocess_scales(u, w, idx_d, vm, sig, fd4.params(theta=theta))
    torch.cuda.synchronize()
    return idx_d[:, :w].cpu().numpy()


def test_straight_ridge_equals_oracle(oracle):
    sig = [1.0, 1.5, 2.0, 3.0, 4.0, 6.0]
    img = (0.2 + synth.ridge_profile(96, 64, 3.0)).astype(np.float32)
    idx, vmax, _, _ = oracle.select_scales(img, sig, oracle.RIDGE)
    vmax = vmax.astype(np.float32)
    want = oracle.postprocess_scales(img, idx, vmax, sig, THETA)
    assert np.array_equal(_gpu_post(img, idx, vmax, sig), want)


@pytest.mark.parametrize("shape", [(160, 200), (67, 45), (300, 97)])
@pytest.mark.parametrize("mode", [0, 1])
def test_entry_point_matches_oracle(oracle, shape, mode):
    h, w = shape
    img = synth.vessel_tree(4500 + h, w, h, depth=5, r0=5.0)
    idx, vmax, _, _ = oracle.select_scales(img, SIGMAS, mode)
    vmax = vmax.astype(np.float32)
    want = oracle.postprocess_scales(img, idx, vmax, SIGMAS, THETA)
    got = _gpu_post(img, idx, vmax, SIGMAS)
    # the walks follow eigenvector directions from FP32 (GPU) and FP64 (oracle)
    # Hessians: a rounded line position may differ where it falls on .5
    assert float((got == want).mean()) >= 0.999
    assert (want != idx).any()  # the post-processing did change scales here


def test_empty_mask_changes_nothing(oracle):
    img = synth.vessel_tree(4600, 64, 48, depth=4, r0=4.0)
    idx, vmax, _, _ = oracle.select_scales(img, SIGMAS, 1)
    assert np.array_equal(_gpu_post(img, idx, vmax.astype(np.float32), SIGMAS, theta=1.0), idx)


def _images():
    shapes = [(128, 128), (53, 37), (150, 211), (97, 64)]
    return [synth.vessel_tree(4700 + i, w, h, depth=4, r0=4.0) for i, (h, w) in enumerate(shapes)]


def _batch(imgs):
    import torch
    ins = [fd4.to_device(im) for im in imgs]
    outs = [torch.zeros_like(u) for u in ins]
    idx = [torch.zeros(u.shape, dtype=torch.uint8, device="cuda") for u in ins]
    return ins, outs, idx, fd4.image_list(ins, [im.shape[1] for im in imgs], outs, idx)


def test_filter_matches_oracle(oracle):
    import torch
    imgs = _images()
    ins, outs, idx, lst = _batch(imgs)
    prm = fd4.params(mode=fd4.VALLEY, postprocess_scales=1, theta=THETA)
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm)
    tau, _, _ = oracle.fed_taus(T, M, 0.05, n=N)
    refs = {}
    for k in (0, 2, 3):
        im = imgs[k]
        w = im.shape[1]
        ref, ridx = oracle.filter_image(im, SIGMAS, tau, M, mode=oracle.VALLEY, postprocess=True, theta=THETA)
        agree = float((idx[k][:, :w].cpu().numpy() == ridx).mean())
        assert agree >= 0.99
        refs[k] = ref
        idx[k][:, :w] = torch.from_numpy(ridx).cuda()
    # the cycles again from the oracle's post-processed scale images: every
    # output pixel is compared, also where a near-tie moved a scale
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm, sigma_given=True)
    for k, ref in refs.items():
        w = imgs[k].shape[1]
        assert np.abs(outs[k][:, :w].cpu().numpy() - ref).max() <= 1e-4


# Re-selection with post-processing cannot be given the oracle's scale images;
# these inputs (chosen with the oracle alone) have every selected scale ahead
# of its runner-up by at least 3e-4 relative at every re-selection, so the
# scale images must agree exactly and u within the tolerance.
RESEL_CASES = [(4204, 53, 37), (4218, 53, 37), (4236, 53, 37), (4248, 64, 80)]


def test_filter_reselect_matches_oracle(oracle, selection_margin):
    imgs = [synth.vessel_tree(s, w, h, depth=4, r0=4.0) for s, h, w in RESEL_CASES]
    ins, outs, idx, lst = _batch(imgs)
    prm = fd4.params(mode=fd4.VALLEY, postprocess_scales=1, theta=THETA, reselect_each_cycle=1)
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm)
    tau, _, _ = oracle.fed_taus(T, M, 0.05, n=N)
    for k, im in enumerate(imgs):
        w = im.shape[1]
        assert selection_margin(im, SIGMAS, tau, M, oracle.VALLEY) >= 3e-4
        ref, ridx = oracle.filter_image(im, SIGMAS, tau, M, mode=oracle.VALLEY, reselect=True,
                                        postprocess=True, theta=THETA)
        assert np.array_equal(idx[k][:, :w].cpu().numpy(), ridx)
        assert np.abs(outs[k][:, :w].cpu().numpy() - ref).max() <= 1e-4


@pytest.mark.parametrize("reselect", [0, 1])
def test_batched_graph_and_two_streams_equal_per_image(reselect):
    import torch
    imgs = _images()
    prm = fd4.params(mode=fd4.VALLEY, postprocess_scales=1, reselect_each_cycle=reselect)
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    ref_idx = [i.clone() for i in idx]
    for im, u_in, o, ix in zip(imgs, ins, outs, idx):
        w = im.shape[1]
        single, single_idx = fd4.filter_image(u_in, w, SIGMAS, T, M, N, prm)
        assert torch.equal(ix[:, :w], single_idx[:, :w])
        assert float((o[:, :w] - single[:, :w]).abs().max()) == 0.0
    for stages in (15, 15 | fd4.GRAPH_TWO_STREAMS):
        for o in outs:
            o.zero_()
        for i in idx:
            i.zero_()
        g = fd4.Graph(lst, SIGMAS, T, M, N, prm, stages=stages)
        g.launch()
        torch.cuda.synchronize()
        for o, r, ix, ri, im in zip(outs, ref, idx, ref_idx, imgs):
            w = im.shape[1]
            assert torch.equal(ix[:, :w], ri[:, :w])
            assert float((o[:, :w] - r[:, :w]).abs().max()) == 0.0
        g.close()


def test_launch_count_and_threshold_validation():
    import torch
    imgs = _images()
    _, _, _, lst = _batch(imgs)
    plain = fd4.Graph(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY))
    post = fd4.Graph(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY, postprocess_scales=1))
    # one post-processing: the chunk masks and K strip launches (N at the selected
    # scales), the walk, the copy
    assert post.kernel_count() == plain.kernel_count() + 1 + len(SIGMAS) + 2
    plain.close()
    post.close()
    u = fd4.to_device(synth.vessel_tree(4800, 32, 32, depth=3, r0=3.0))
    for bad in (dict(theta=1.5), dict(theta=-0.1), dict(postprocess_scales=2)):
        with pytest.raises(fd4.Fd4Error):
            fd4.filter_image(u, 32, SIGMAS, T, M, N, fd4.params(**bad))
    torch.cuda.synchronize()
