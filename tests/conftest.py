import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def selection_margin(oracle):
    """min over the re-selections of a filter run (the oracle's schedule) and
    over the pixels with a positive vesselness of (V_best - V_second) / V_best:
    how far every selected scale leads its runner-up.  A lead far above FP32
    rounding (~1e-6 relative) means the FP32 selection must agree exactly."""
    import numpy as np

    def margin(img, sigmas, tau, M, mode, reselect=True):
        u = img.astype(np.float64)
        lead = np.inf
        idx = None
        for k in range(M):
            if k == 0 or reselect:
                idx, _, vall, _ = oracle.select_scales(u, sigmas, mode)
                s = np.sort(vall, axis=0)
                pos = s[-1] > 0
                if pos.any():
                    lead = min(lead, float(((s[-1] - s[-2])[pos] / s[-1][pos]).min()))
            tensor, _ = oracle.build_tensor(u, idx, sigmas, mode=mode)
            u = oracle.fed_cycle(u, tensor, tau)
        return lead
    return margin
