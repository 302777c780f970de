"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/fd4.h declares, computes the host-side FED table like the
oracle, and rejects bad arguments on the host before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1611_06906_gb300 import fd4

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fd4.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    names = re.findall(r"\b(fd4_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    L = fd4.lib()
    names = declared_functions()
    assert "fd4_filter" in names and "fd4_fed_cycle" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(fd4.SIGNATURES) | set(n for n in names if n not in fd4.SIGNATURES)


def test_defaults_and_strerror():
    p = fd4.params()
    assert abs(p.lambda_ - 0.005) < 1e-9 and p.rho == 0.5 and p.beta == 0.5 and p.tau_max == pytest.approx(0.05)
    assert p.mode == fd4.BOTH and p.boundary == fd4.NATURAL and p.c == 0.0 and p.gamma == 1.0
    assert p.reselect_each_cycle == 0 and p.grad_norm_squared == 0 and p.fed_steps_per_launch == 0
    assert fd4.strerror(0) == "ok"
    assert "workspace" in fd4.strerror(-5)
    assert fd4.lib().fd4_version() >= 100


@pytest.mark.parametrize("T,M,n", [(11 / 3, 2, 10), (35.0, 5, 20), (325 / 3, 10, 25), (12.0, 2, 0),
                                   (500.0, 10000, 0), (20.0, 1000, 0)])
def test_fed_taus_match_oracle(oracle, T, M, n):
    tau_o, kappa_o, _ = oracle.fed_taus(T, M, 0.05, n=n, kappa=0)
    tau_l, kappa_l = fd4.fed_taus(T, M, 0.05, n=n, kappa=0)
    assert kappa_l == kappa_o
    assert tau_l.size == tau_o.size
    assert np.abs(tau_l - tau_o).max() <= 1e-14 * tau_o.max()


def test_fed_taus_errors():
    with pytest.raises(fd4.Fd4Error) as e:
        fd4.fed_taus(35.0, 5, 0.05, n=10)
    assert e.value.status == -2
    with pytest.raises(fd4.Fd4Error) as e:
        fd4.fed_taus(1.0, 1, 0.07)  # above the 1/17 bound of Sec. 3.4
    assert e.value.status == -2
    with pytest.raises(fd4.Fd4Error) as e:
        fd4.fed_taus(35.0, 5, 0.05, n=20, kappa=4)  # not coprime with 20
    assert e.value.status == -1


def test_workspace_sizes_grow_with_the_problem():
    a = fd4.workspace_bytes(fd4.OP_SELECT_SCALES, 100, 100, 4)
    b = fd4.workspace_bytes(fd4.OP_SELECT_SCALES, 100, 100, 8)
    assert 0 < a < b
    f = fd4.workspace_bytes(fd4.OP_FILTER, 1024, 1024, 8)
    assert f >= b and f >= 1024 * 1024 * (1 + 16)
    assert fd4.workspace_bytes(99, 10, 10, 1) == 0


def test_host_side_argument_errors():
    """Every check below fails before any CUDA call is made."""
    L = fd4.lib()
    sig = (ctypes.c_float * 2)(1.0, 2.0)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: validation rejects first
    ws = ctypes.c_void_p(1 << 24)
    # null image
    assert L.fd4_select_scales(None, 8, 8, 8, sig, 2, None, fake, None, ws, 1 << 30, None) == -1
    # pitch not a multiple of 4
    assert L.fd4_select_scales(fake, 8, 8, 10, sig, 2, None, fake, None, ws, 1 << 30, None) == -4
    # pitch < w
    assert L.fd4_select_scales(fake, 8, 8, 4, sig, 2, None, fake, None, ws, 1 << 30, None) == -4
    # unaligned image pointer
    assert L.fd4_select_scales(ctypes.c_void_p((1 << 20) + 4), 8, 8, 8, sig, 2, None, fake, None, ws,
                               1 << 30, None) == -8
    # scales not increasing / out of range
    bad = (ctypes.c_float * 2)(2.0, 1.0)
    assert L.fd4_select_scales(fake, 8, 8, 8, bad, 2, None, fake, None, ws, 1 << 30, None) == -9
    big = (ctypes.c_float * 1)(17.0)
    assert L.fd4_select_scales(fake, 8, 8, 8, big, 1, None, fake, None, ws, 1 << 30, None) == -9
    many = (ctypes.c_float * 40)(*[1 + 0.1 * i for i in range(40)])
    assert L.fd4_select_scales(fake, 8, 8, 8, many, 40, None, fake, None, ws, 1 << 30, None) == -3
    # workspace too small
    assert L.fd4_select_scales(fake, 8, 8, 8, sig, 2, None, fake, None, ws, 16, None) == -5
    # image too small
    assert L.fd4_select_scales(fake, 2, 8, 4, sig, 2, None, fake, None, ws, 1 << 30, None) == -1
    # FED cycle: bad step sizes and boundary
    tau = (ctypes.c_double * 2)(0.1, -0.2)
    assert L.fd4_fed_cycle(fake, 8, 8, 8, fake, tau, 2, 0, ws, 1 << 30, None) == -1
    tau = (ctypes.c_double * 2)(0.1, 0.2)
    assert L.fd4_fed_cycle(fake, 8, 8, 8, fake, tau, 2, 7, ws, 1 << 30, None) == -1
    # filter: unstable schedule is reported before any launch
    p = fd4.params(tau_max=0.05)
    assert L.fd4_filter(fake, fake, 8, 8, 8, sig, 2, ctypes.byref(p), 35.0, 5, 10, None, 0, ws,
                        1 << 40, None) == -2


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of fd4_params and fd4_image have the header's size and
    field offsets (compiled with the host C compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"fd4_params": fd4.Params, "fd4_image": fd4.Image, "fd4_fed_schedule": fd4.FedSchedule}
    lines = ['#include <stdio.h>', '#include "fd4.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            c_field = "lambda" if fname == "lambda_" else fname
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, c_field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py)
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_host_side_argument_errors_of_the_added_entry_points():
    """Scale post-processing, IFOD tensor, crease extraction and the added
    filter parameters: every check below fails before any CUDA call."""
    L = fd4.lib()
    sig = (ctypes.c_float * 2)(1.0, 2.0)
    fake = ctypes.c_void_p(1 << 20)
    odd = ctypes.c_void_p((1 << 20) + 2)
    ws = ctypes.c_void_p(1 << 24)
    big = 1 << 40
    # post-processing: null index / V map, unaligned V map, small workspace, theta outside [0, 1]
    assert L.fd4_postprocess_scales(fake, 8, 8, 8, None, fake, sig, 2, None, ws, big, None) == -1
    assert L.fd4_postprocess_scales(fake, 8, 8, 8, fake, None, sig, 2, None, ws, big, None) == -1
    assert L.fd4_postprocess_scales(fake, 8, 8, 8, fake, odd, sig, 2, None, ws, big, None) == -8
    assert L.fd4_postprocess_scales(fake, 8, 8, 8, fake, fake, sig, 2, None, ws, 16, None) == -5
    p = fd4.params(theta=1.5)
    assert L.fd4_postprocess_scales(fake, 8, 8, 8, fake, fake, sig, 2, ctypes.byref(p), ws, big, None) == -1
    # IFOD tensor: null / unaligned output, bad scale, bad model
    assert L.fd4_build_tensor_ifod(fake, 8, 8, 8, None, None, None) == -1
    assert L.fd4_build_tensor_ifod(fake, 8, 8, 8, None, ctypes.c_void_p((1 << 20) + 4), None) == -8
    for kw in (dict(ifod_sigma=0.0), dict(ifod_sigma=13.0), dict(model=5)):
        p = fd4.params(**kw)
        assert L.fd4_build_tensor_ifod(fake, 8, 8, 8, ctypes.byref(p), fake, None) == -1
    # creases: scale, mode, outputs, capacity, alignment, workspace
    cnt = ctypes.c_void_p(1 << 22)
    assert L.fd4_extract_creases(fake, 8, 8, 8, 5.0, 0, fake, fake, 10, cnt, ws, big, None) == -1
    assert L.fd4_extract_creases(fake, 8, 8, 8, 1.0, 3, fake, fake, 10, cnt, ws, big, None) == -1
    assert L.fd4_extract_creases(fake, 8, 8, 8, 1.0, 0, None, fake, 10, cnt, ws, big, None) == -1
    assert L.fd4_extract_creases(fake, 8, 8, 8, 1.0, 0, fake, fake, -1, cnt, ws, big, None) == -1
    assert L.fd4_extract_creases(fake, 8, 8, 8, 1.0, 0, ctypes.c_void_p((1 << 20) + 4), fake, 10, cnt, ws, big,
                                 None) == -8
    assert L.fd4_extract_creases(fake, 8, 8, 8, 1.0, 0, fake, fake, 10, cnt, ws, 16, None) == -5
    # whole filter: the added switches take 0 or 1, theta lies in [0, 1]
    for kw in (dict(reselect_each_cycle=2), dict(postprocess_scales=-1), dict(theta=-0.5), dict(model=2)):
        p = fd4.params(**kw)
        assert L.fd4_filter(fake, fake, 8, 8, 8, sig, 2, ctypes.byref(p), 11 / 3, 2, 10, None, 0, ws, big,
                            None) == -1


def test_workspace_sizes_of_the_added_entry_points():
    a = fd4.workspace_bytes(fd4.OP_POSTPROCESS, 100, 100, 4)
    b = fd4.workspace_bytes(fd4.OP_POSTPROCESS, 200, 100, 4)
    assert 0 < a < b and a >= 100 * 100 * 17
    c = fd4.workspace_bytes(fd4.OP_CREASES, 100, 100, 0)
    assert c >= 100 * 100 * 8


def test_host_side_argument_errors_of_the_fed_schedule():
    """FED kernel schedules outside their ranges, on the explicit-schedule
    cycle, the filters and the wait self-test: rejected before any CUDA call."""
    L = fd4.lib()
    sig = (ctypes.c_float * 2)(1.0, 2.0)
    fake = ctypes.c_void_p(1 << 20)
    ws = ctypes.c_void_p(1 << 24)
    big = 1 << 40
    tau = (ctypes.c_double * 2)(0.1, 0.2)
    for steps, rows, quads in ((5, 0, 0), (-1, 0, 0), (2, 48, 2), (2, 16, 2), (2, 64, 3), (2, 64, -1)):
        assert L.fd4_fed_cycle_sched(fake, 8, 8, 8, fake, tau, 2, 0, steps, rows, quads, ws, big, None) == -1
    for kw in (dict(fed_steps_per_launch=5), dict(fed_tile_rows=100), dict(fed_quads_per_thread=4)):
        p = fd4.params(**kw)
        assert L.fd4_filter(fake, fake, 8, 8, 8, sig, 2, ctypes.byref(p), 11 / 3, 2, 10, None, 0, ws, big,
                            None) == -1
    st = ctypes.c_int(0)
    assert L.fd4_selftest_fed_wait_timeout(fake, 8, 8, 8, None, ws, big, ctypes.byref(st), None) == -1
    assert L.fd4_selftest_fed_wait_timeout(fake, 8, 8, 8, fake, ws, 16, ctypes.byref(st), None) == -5
    assert L.fd4_selftest_fed_wait_timeout(fake, 8, 8, 8, fake, ws, big, None, None) == -1


def test_schedule_defaults_and_struct_layout():
    p = fd4.params()
    assert p.fed_tile_rows == 0 and p.fed_quads_per_thread == 0
    assert ctypes.sizeof(fd4.FedSchedule) == 16
    s = fd4.FedSchedule(2, 64, 2, 1.5)
    assert s.as_params() == dict(fed_steps_per_launch=2, fed_tile_rows=64, fed_quads_per_thread=2)
