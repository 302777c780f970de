"""The allocation-free FED cycle (fd4_fed_cycle_noalloc) against the regular
entry point (fd4_fed_cycle).

fd4_fed_cycle_noalloc is for callers that cannot allocate device memory (host
applications that own all device memory, programs that must not call
cudaMalloc once running); its scratch lives in a static array inside the
library.  This file is collected last, so a run that stops at the first
failure has run every other test before it; it passes both on its own in a
fresh process and after the rest of the suite.  Two calls in a row are checked,
because every call reuses the one built-in scratch array.
"""
import math

import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4

pytestmark = pytest.mark.gpu

def _case(seed, h, w):
    import torch
    rng = np.random.default_rng(seed)
    u0 = rng.random((h, w)).astype(np.float32)
    th = rng.uniform(-math.pi, math.pi, size=(h, w))
    mu = rng.uniform(0.0, 1.0, size=(2, h, w))
    t = np.stack([np.cos(2 * th), np.sin(2 * th), mu[0], mu[1]], axis=-1).astype(np.float32)
    ten = fd4.empty_image(h, w, channels=4)
    ten[:, :w, :] = torch.from_numpy(t).cuda()
    return u0, ten


def test_noalloc_matches_fed_cycle_twice_in_a_row():
    import torch
    n = 20
    tau, _ = fd4.fed_taus(n * (n + 1) * 0.05 / 3, 1, 0.05, n=n)
    for seed, (h, w) in ((11, (301, 257)), (12, (130, 97))):
        u0, ten = _case(seed, h, w)
        ref = fd4.to_device(u0)
        fd4.fed_cycle(ref, w, ten, tau)
        got = fd4.to_device(u0)
        fd4.fed_cycle_noalloc(got, w, ten, tau)
        torch.cuda.synchronize()
        # the same kernels on the same inputs: identical results
        assert torch.equal(got[:, :w], ref[:, :w]), seed


def test_noalloc_rejects_images_beyond_its_scratch():
    h, pitch = 2049, 2048  # one row more than the built-in 4 Mi-pixel plane
    assert h * pitch > fd4.NOALLOC_MAX_PIXELS
    u = fd4.empty_image(h, pitch)
    ten = fd4.empty_image(h, pitch, channels=4)
    with pytest.raises(fd4.Fd4Error) as e:
        fd4.fed_cycle_noalloc(u, pitch, ten, [0.01])
    assert e.value.status == -5
