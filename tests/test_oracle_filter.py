"""Pins of the oracle's whole-filter schedule (Sec. 3, the cycle structure of
Eq. 21): M cycles of (tensor build at the selected scales, FED cycle).

  * the filter equals its composition from the separately pinned primitives
    (select_scales, build_tensor, fed_cycle), both for one selection on the
    input image and for a selection on the current image before every cycle;
  * with one cycle the two schedules coincide;
  * the re-selected scale image follows the filtered image: it differs from
    the first selection once the diffusion has changed the structures;
  * either schedule conserves the mean grey value (natural boundary).
"""
import numpy as np
import pytest

from paper_1611_06906_gb300 import synth

SIG = [1.0, 1.6, 2.5, 4.0]


def _T(M, n):  # n steps per cycle exactly at tau_max = 0.05
    return M * n * (n + 1) * 0.05 / 3


def _case(seed=4100, w=48, h=40):
    img = synth.vessel_tree(seed, w, h, depth=4, r0=3.0)
    return img.astype(np.float64)


def _compose(oracle, img, tau, M, reselect, mode):
    u = img.copy()
    idx = None
    for k in range(M):
        if k == 0 or reselect:
            idx = oracle.select_scales(u, SIG, mode)[0]
        tensor, _ = oracle.build_tensor(u, idx, SIG, mode=mode)
        u = oracle.fed_cycle(u, tensor, tau)
    return u, idx


@pytest.mark.parametrize("reselect", [False, True])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_filter_equals_composition(oracle, reselect, mode):
    img = _case()
    tau, _, _ = oracle.fed_taus(_T(3, 10), 3, 0.05, n=10)
    out, idx = oracle.filter_image(img, SIG, tau, 3, mode=mode, reselect=reselect)
    ref, ref_idx = _compose(oracle, img, tau, 3, reselect, mode)
    assert np.array_equal(out, ref)
    assert np.array_equal(idx, ref_idx)


def test_one_cycle_schedules_coincide(oracle):
    img = _case(4101)
    tau, _, _ = oracle.fed_taus(_T(1, 10), 1, 0.05, n=10)
    a, ia = oracle.filter_image(img, SIG, tau, 1, mode=oracle.BOTH)
    b, ib = oracle.filter_image(img, SIG, tau, 1, mode=oracle.BOTH, reselect=True)
    assert np.array_equal(a, b) and np.array_equal(ia, ib)


def test_reselection_follows_the_filtered_image(oracle):
    img = _case(4102)
    tau, _, _ = oracle.fed_taus(_T(5, 20), 5, 0.05, n=20)
    first = oracle.select_scales(img, SIG, oracle.VALLEY)[0]
    out, last = oracle.filter_image(img, SIG, tau, 5, mode=oracle.VALLEY, reselect=True)
    _, once = oracle.filter_image(img, SIG, tau, 5, mode=oracle.VALLEY)
    assert np.array_equal(once, first)
    assert np.array_equal(last, oracle.select_scales(_compose(oracle, img, tau, 4, True, oracle.VALLEY)[0],
                                                     SIG, oracle.VALLEY)[0])
    assert (last != first).any()


@pytest.mark.parametrize("reselect", [False, True])
def test_mean_is_conserved(oracle, reselect):
    img = _case(4103)
    tau, _, _ = oracle.fed_taus(_T(5, 20), 5, 0.05, n=20)
    out, _ = oracle.filter_image(img, SIG, tau, 5, mode=oracle.BOTH, reselect=reselect)
    assert abs(out.mean() - img.mean()) < 1e-12
