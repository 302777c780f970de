"""Batched path (one launch per stage across images of uneven sizes), its CUDA
graph, the FED schedule autotuner, and the kernel-schedule variants, against
the per-image entry point and the FP64 oracle."""
import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4, synth

pytestmark = pytest.mark.gpu

SIGMAS = [1.0, 1.6, 2.5, 4.0]
M, N = 2, 10
T = M * N * (N + 1) * 0.05 / 3


def _images():
    shapes = [(128, 128), (53, 37), (150, 211), (3, 5), (97, 64), (61, 300)]
    return [synth.vessel_tree(4000 + i, w, h, depth=4, r0=4.0) for i, (h, w) in enumerate(shapes)]


def _batch(imgs, same_out=False):
    import torch
    ins = [fd4.to_device(im) for im in imgs]
    outs = ins if same_out else [torch.zeros_like(u) for u in ins]
    idx = [torch.zeros(u.shape, dtype=torch.uint8, device="cuda") for u in ins]
    widths = [im.shape[1] for im in imgs]
    return ins, outs, idx, fd4.image_list(ins, widths, outs, idx)


@pytest.mark.parametrize("mode", [fd4.VALLEY, fd4.BOTH])
def test_batched_equals_per_image(mode):
    import torch
    imgs = _images()
    prm = fd4.params(mode=mode)
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm)
    torch.cuda.synchronize()
    for im, u_in, o, ix in zip(imgs, ins, outs, idx):
        w = im.shape[1]
        ref, ref_idx = fd4.filter_image(u_in, w, SIGMAS, T, M, N, prm)
        assert torch.equal(ix[:, :w], ref_idx[:, :w])
        assert float((o[:, :w] - ref[:, :w]).abs().max()) == 0.0
        # inputs are left untouched
        assert np.array_equal(u_in[:, :w].cpu().numpy(), im)


def test_batched_matches_oracle(oracle):
    imgs = _images()
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY))
    import torch
    tau, _, _ = oracle.fed_taus(T, M, 0.05, n=N)
    refs = {}
    for k in (0, 2, 3):
        im = imgs[k]
        w = im.shape[1]
        ref, ridx = oracle.filter_image(im, SIGMAS, tau, M, mode=oracle.VALLEY)
        agree = float((idx[k][:, :w].cpu().numpy() == ridx).mean())
        assert agree >= 0.99
        refs[k] = ref
        # where FP32 and FP64 pick different scales at near-ties the outputs
        # legitimately differ there: the batch is filtered again with the
        # oracle's scale image given, and every output pixel is compared
        idx[k][:, :w] = torch.from_numpy(ridx).cuda()
    fd4.filter_batched(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY), sigma_given=True)
    for k, ref in refs.items():
        w = imgs[k].shape[1]
        assert np.abs(outs[k][:, :w].cpu().numpy() - ref).max() <= 1e-4


def test_graph_replays_the_batched_filter():
    import torch
    imgs = _images()
    prm = fd4.params(mode=fd4.VALLEY)
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm)
    ref = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    g = fd4.Graph(lst, SIGMAS, T, M, N, prm)
    for _ in range(2):
        g.launch()
        torch.cuda.synchronize()
        for o, r, im in zip(outs, ref, imgs):
            w = im.shape[1]
            assert float((o[:, :w] - r[:, :w]).abs().max()) == 0.0
    # launch accounting: per FED cycle ceil(N / 2) fused launches (+ one copy-back
    # when that count is odd); the whole filter adds selection and tensor builds
    g_fed = fd4.Graph(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY, fed_steps_per_launch=2),
                      stages=fd4.STAGE_FED)
    per_cycle = -(-N // 2)
    assert g_fed.kernel_count() >= M * (per_cycle + per_cycle % 2)
    assert g.kernel_count() > g_fed.kernel_count() + M * len(SIGMAS)
    g_fed.close()
    g.close()


def test_in_place_batch_and_given_scales():
    import torch
    imgs = _images()[:3]
    prm = fd4.params(mode=fd4.VALLEY)
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm)
    # same scales supplied, filtered in place
    ins2, _, _, _ = _batch(imgs, same_out=True)
    lst2 = fd4.image_list(ins2, [im.shape[1] for im in imgs], ins2, idx)
    fd4.filter_batched(lst2, SIGMAS, T, M, N, prm, sigma_given=True)
    torch.cuda.synchronize()
    for a, b, im in zip(ins2, outs, imgs):
        w = im.shape[1]
        assert float((a[:, :w] - b[:, :w]).abs().max()) == 0.0


def test_fed_schedules_agree_and_autotune():
    import torch
    imgs = _images()
    res = []
    for steps in (1, 2, 3, 4):
        ins, outs, idx, lst = _batch(imgs)
        fd4.filter_batched(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY, fed_steps_per_launch=steps))
        torch.cuda.synchronize()
        res.append([o[:, :im.shape[1]].clone() for o, im in zip(outs, imgs)])
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert float((a - b).abs().max()) <= 1e-5
    ins, outs, idx, lst = _batch(imgs)
    best, times = fd4.autotune_batched(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY))
    assert best in (1, 2, 3, 4)
    assert all(t > 0 for t in times)


def test_bad_batch_is_rejected_before_launch():
    imgs = _images()[:2]
    ins, outs, idx, lst = _batch(imgs)
    lst[1].pitch = lst[1].w + 1  # not a multiple of 4
    with pytest.raises(fd4.Fd4Error) as e:
        fd4.filter_batched(lst, SIGMAS, T, M, N, ws=fd4.batch_workspace(fd4.image_list(ins, [128, 37]), 4))
    assert e.value.status == -4


def test_fed_kernels_report_no_timeout():
    """After the batched runs above, no bounded device wait of the FED kernels gave up."""
    imgs = _images()
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, fd4.params(mode=fd4.VALLEY))
    assert fd4.device_status(reset=True) == 0


def test_two_stream_graph_equals_one_stream_graph():
    import torch
    imgs = _images()
    prm = fd4.params(mode=fd4.VALLEY)
    ins, outs, idx, lst = _batch(imgs)
    g1 = fd4.Graph(lst, SIGMAS, T, M, N, prm)
    g1.launch()
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    ref_idx = [i.clone() for i in idx]
    for o in outs:
        o.zero_()
    for i in idx:
        i.zero_()
    g2 = fd4.Graph(lst, SIGMAS, T, M, N, prm, stages=fd4.STAGES_ALL | fd4.GRAPH_TWO_STREAMS)
    for _ in range(2):
        g2.launch()
        torch.cuda.synchronize()
        for o, r, i, ri, im in zip(outs, ref, idx, ref_idx, imgs):
            w = im.shape[1]
            assert torch.equal(i[:, :w], ri[:, :w])
            assert float((o[:, :w] - r[:, :w]).abs().max()) == 0.0
    g1.close()
    g2.close()
