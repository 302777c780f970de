"""Crease extraction on the GPU (fd4_extract_creases) against the FP64 oracle:
the same cells and segment end points on a noisy vessel tree (the decisions
d > 0 and the crease-type filter are taken from FP32 values here and FP64
values in the oracle, so a few cells whose corner values are within rounding
of zero may differ), the exact ridge line of an elongated blob, and argument
checks."""
import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("sigma", [1.0, 2.0])
def test_segments_match_oracle(oracle, mode, sigma):
    h, w = 160, 200
    img = synth.vessel_tree(5300, w, h, depth=5, r0=4.0)
    want, wkeys = oracle.extract_creases(img, sigma=sigma, mode=mode)
    got, gkeys = fd4.extract_creases(fd4.to_device(img), w, sigma=sigma, mode=mode)
    assert len(want) > 100
    common, wi, gi = np.intersect1d(wkeys, gkeys, return_indices=True)
    assert common.size >= 0.98 * max(wkeys.size, gkeys.size)
    err = np.abs(got[gi] - want[wi]).max(axis=1)
    assert np.quantile(err, 0.98) < 1e-3 and err.max() < 1.0


def test_elongated_blob_ridge_line():
    h, w = 40, 61
    Y, X = np.mgrid[0:h, 0:w].astype(np.float64)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    img = np.exp(-(X - cx) ** 2 / (2 * 12.0 ** 2) - (Y - cy) ** 2 / (2 * 3.0 ** 2)).astype(np.float32)
    segs, _ = fd4.extract_creases(fd4.to_device(img), w, sigma=1.0, mode=fd4.RIDGE)
    near = [s for s in segs if abs(s[1] - cy) < 0.5 and abs(s[3] - cy) < 0.5 and abs(0.5 * (s[0] + s[2]) - cx) < 15]
    assert len(near) >= 20
    assert max(max(abs(s[1] - cy), abs(s[3] - cy)) for s in near) < 1e-3


def test_arguments_are_checked():
    u = fd4.to_device(synth.vessel_tree(5301, 32, 32, depth=3, r0=3.0))
    for kw in (dict(sigma=5.0), dict(sigma=0.0), dict(mode=3)):
        with pytest.raises(fd4.Fd4Error):
            fd4.extract_creases(u, 32, **kw)
