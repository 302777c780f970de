"""The IFOD comparator (Eq. 2, model = FD4_MODEL_IFOD) on the GPU: its tensor
field and whole filter against the FP64 oracle, and the batched, graph and
two-stream paths against the per-image entry point."""
import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4, synth

pytestmark = pytest.mark.gpu

SIGMAS = [1.0, 1.6, 2.5, 4.0]  # validated by the entry points, unused by IFOD
M, N = 3, 10
T = M * N * (N + 1) * 0.05 / 3
TOL_U = 1e-4


@pytest.mark.parametrize("sigma", [1.0, 2.5])
@pytest.mark.parametrize("shape", [(150, 211), (67, 45)])
def test_tensor_matches_oracle(oracle, sigma, shape):
    h, w = shape
    img = synth.vessel_tree(5000 + h, w, h, depth=5, r0=4.0)
    want = oracle.build_tensor_ifod(img, sigma=sigma, lam=0.005)
    got = fd4.build_tensor_ifod(fd4.to_device(img), w, fd4.params(ifod_sigma=sigma))[:, :w].cpu().numpy()
    assert np.all(got[..., 0] == 1.0) and np.all(got[..., 1] == 0.0)
    assert np.array_equal(got[..., 2], got[..., 3])
    assert np.abs(got[..., 2] - want[2]).max() <= 1e-5


def _images():
    shapes = [(128, 128), (53, 37), (150, 211), (97, 64)]
    return [synth.vessel_tree(5100 + i, w, h, depth=4, r0=4.0) for i, (h, w) in enumerate(shapes)]


def _batch(imgs):
    import torch
    ins = [fd4.to_device(im) for im in imgs]
    outs = [torch.zeros_like(u) for u in ins]
    idx = [torch.zeros(u.shape, dtype=torch.uint8, device="cuda") for u in ins]
    return ins, outs, idx, fd4.image_list(ins, [im.shape[1] for im in imgs], outs, idx)


def test_filter_matches_oracle(oracle):
    imgs = _images()
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, fd4.params(model=fd4.MODEL_IFOD))
    tau, _, _ = oracle.fed_taus(T, M, 0.05, n=N)
    for k, im in enumerate(imgs):
        w = im.shape[1]
        ref = oracle.filter_ifod(im, tau, M, sigma=1.0, lam=0.005)
        assert np.abs(outs[k][:, :w].cpu().numpy() - ref).max() <= TOL_U


def test_batched_graph_and_two_streams_equal_per_image():
    import torch
    imgs = _images()
    prm = fd4.params(model=fd4.MODEL_IFOD)
    ins, outs, idx, lst = _batch(imgs)
    fd4.filter_batched(lst, SIGMAS, T, M, N, prm)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    for im, u_in, o in zip(imgs, ins, outs):
        w = im.shape[1]
        single, _ = fd4.filter_image(u_in, w, SIGMAS, T, M, N, prm)
        assert float((o[:, :w] - single[:, :w]).abs().max()) == 0.0
    for stages in (15, 15 | fd4.GRAPH_TWO_STREAMS):
        for o in outs:
            o.zero_()
        g = fd4.Graph(lst, SIGMAS, T, M, N, prm, stages=stages)
        g.launch()
        torch.cuda.synchronize()
        for o, r, im in zip(outs, ref, imgs):
            w = im.shape[1]
            assert float((o[:, :w] - r[:, :w]).abs().max()) == 0.0
        g.close()
    # one strip launch per cycle replaces the selection and the tensor build
    # (plus the two kernels that write the descriptor and tensor-map tables)
    g = fd4.Graph(lst, SIGMAS, T, M, N, prm, stages=fd4.STAGE_TENSOR)
    assert g.kernel_count() == M + 2
    g.close()


def test_model_arguments_are_validated():
    import torch
    u = fd4.to_device(synth.vessel_tree(5200, 32, 32, depth=3, r0=3.0))
    for bad in (dict(model=2), dict(model=fd4.MODEL_IFOD, ifod_sigma=0.0),
                dict(model=fd4.MODEL_IFOD, ifod_sigma=20.0)):
        with pytest.raises(fd4.Fd4Error):
            fd4.filter_image(u, 32, SIGMAS, T, M, N, fd4.params(**bad))
    torch.cuda.synchronize()
