"""Thin Python binding of the fd4 C ABI (include/fd4.h).

Argument marshalling only: every step of the filter runs in the CUDA kernels
of libfd4.so.  PyTorch provides device memory and the current stream.  There
is no CPU fallback; if the library cannot be loaded every call raises.

Device images are float32 tensors of shape (h, pitch) with pitch a multiple
of 4 and the image in the first w columns (``to_device`` pads a numpy image).
The tensor field has shape (h, pitch, 4): (cos 2t, sin 2t, mu1, mu2).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

RIDGE, VALLEY, BOTH = 0, 1, 2
NATURAL, PERIODIC = 0, 1
OP_SELECT_SCALES, OP_BUILD_TENSOR, OP_FED_CYCLE, OP_FILTER, OP_POSTPROCESS, OP_CREASES = 0, 1, 2, 3, 4, 5
MODEL_MAFOD, MODEL_IFOD = 0, 1
STAGE_SELECT, STAGE_COPY, STAGE_TENSOR, STAGE_FED, STAGES_ALL = 1, 2, 4, 8, 15
GRAPH_TWO_STREAMS = 16
MAX_FED_STEPS = 4096

_lock = threading.Lock()
_lib = None


class Fd4Error(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, strerror(status), status))


class Params(ctypes.Structure):
    """fd4_params (include/fd4.h)."""
    _fields_ = [("lambda_", ctypes.c_float), ("rho", ctypes.c_float), ("beta", ctypes.c_float),
                ("c", ctypes.c_float), ("gamma", ctypes.c_float), ("tau_max", ctypes.c_float),
                ("mode", ctypes.c_int), ("boundary", ctypes.c_int), ("kappa", ctypes.c_int),
                ("grad_norm_squared", ctypes.c_int), ("fed_steps_per_launch", ctypes.c_int),
                ("reselect_each_cycle", ctypes.c_int), ("postprocess_scales", ctypes.c_int),
                ("theta", ctypes.c_float), ("model", ctypes.c_int), ("ifod_sigma", ctypes.c_float),
                ("fed_tile_rows", ctypes.c_int), ("fed_quads_per_thread", ctypes.c_int)]


class FedSchedule(ctypes.Structure):
    """fd4_fed_schedule (include/fd4.h)."""
    _fields_ = [("steps_per_launch", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("quads_per_thread", ctypes.c_int), ("ms", ctypes.c_float)]

    def as_params(self) -> dict:
        """The fd4_params fields of this schedule (zero: the library default)."""
        return dict(fed_steps_per_launch=self.steps_per_launch, fed_tile_rows=self.tile_rows,
                    fed_quads_per_thread=self.quads_per_thread)

    def as_dict(self) -> dict:
        return dict(steps_per_launch=self.steps_per_launch, tile_rows=self.tile_rows,
                    quads_per_thread=self.quads_per_thread, ms=self.ms)


AUTOTUNE_CANDIDATES = 10


class Image(ctypes.Structure):
    """fd4_image (include/fd4.h)."""
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("d_sigma_idx", ctypes.c_void_p),
                ("w", ctypes.c_int), ("h", ctypes.c_int), ("pitch", ctypes.c_int)]


_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i = ctypes.c_int
_fp = ctypes.POINTER(ctypes.c_float)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_pp = ctypes.POINTER(Params)

SIGNATURES = {
    "fd4_default_params": (None, [_pp]),
    "fd4_strerror": (ctypes.c_char_p, [_i]),
    "fd4_version": (_i, []),
    "fd4_fed_taus": (_i, [ctypes.c_double, _i, ctypes.c_double, _i, _i, _dp, _i, _ip, _ip]),
    "fd4_workspace_bytes": (_sz, [_i, _i, _i, _i]),
    "fd4_select_scales": (_i, [_vp, _i, _i, _i, _fp, _i, _pp, _vp, _vp, _vp, _sz, _vp]),
    "fd4_build_tensor": (_i, [_vp, _i, _i, _i, _vp, _fp, _i, _pp, _vp, _vp, _sz, _vp]),
    "fd4_postprocess_scales": (_i, [_vp, _i, _i, _i, _vp, _vp, _fp, _i, _pp, _vp, _sz, _vp]),
    "fd4_build_tensor_ifod": (_i, [_vp, _i, _i, _i, _pp, _vp, _vp]),
    "fd4_extract_creases": (_i, [_vp, _i, _i, _i, ctypes.c_float, _i, _vp, _vp, _i, _vp, _vp, _sz, _vp]),
    "fd4_fed_cycle": (_i, [_vp, _i, _i, _i, _vp, _dp, _i, _i, _vp, _sz, _vp]),
    "fd4_fed_cycle_sched": (_i, [_vp, _i, _i, _i, _vp, _dp, _i, _i, _i, _i, _i, _vp, _sz, _vp]),
    "fd4_selftest_fed_wait_timeout": (_i, [_vp, _i, _i, _i, _vp, _vp, _sz, _ip, _vp]),
    "fd4_measure_fma_rate": (_i, [_vp, _sz, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp]),
    "fd4_filter": (_i, [_vp, _vp, _i, _i, _i, _fp, _i, _pp, ctypes.c_double, _i, _i, _vp, _i, _vp,
                        _sz, _vp]),
    "fd4_fed_cycle_noalloc": (_i, [_vp, _i, _i, _i, _vp, _dp, _i, _i, _vp]),
    "fd4_batch_workspace_bytes": (_sz, [_vp, _i, _i]),
    "fd4_filter_batched": (_i, [_vp, _i, _fp, _i, _pp, ctypes.c_double, _i, _i, _i, _vp, _sz, _vp]),
    "fd4_graph_create": (_i, [_vp, _i, _fp, _i, _pp, ctypes.c_double, _i, _i, _i, _i, _vp, _sz,
                              ctypes.POINTER(ctypes.c_void_p)]),
    "fd4_graph_launch": (_i, [_vp, _vp]),
    "fd4_graph_destroy": (_i, [_vp]),
    "fd4_graph_kernel_count": (_i, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "fd4_device_status": (_i, [ctypes.POINTER(ctypes.c_int), _i]),
    "fd4_autotune_batched": (_i, [_vp, _i, _fp, _i, _pp, ctypes.c_double, _i, _i, _vp, _sz, _vp,
                                  ctypes.POINTER(FedSchedule), ctypes.POINTER(FedSchedule)]),
}
NOALLOC_MAX_PIXELS = 4 * 1024 * 1024
SELECTOR_SIGNATURES = {
    "fd4_selector_param_bytes": (_sz, []),
    "fd4_selector_workspace_bytes": (_sz, [_i, _i, _i, _i]),
    "fd4_selector_infer_workspace_bytes": (_sz, [_i, _i, _i, _i]),
    "fd4_selector_set_weights": (_i, [_vp, _fp, _vp]),
    "fd4_selector_get_weights": (_i, [_vp, _fp, _i, _vp]),
    "fd4_selector_init": (_i, [_vp, ctypes.c_ulonglong, _vp]),
    "fd4_selector_forward": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _sz, _vp]),
    "fd4_selector_grad": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _sz, _vp]),
    "fd4_selector_update": (_i, [_vp, ctypes.c_float, _i, _vp]),
    "fd4_selector_predict": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _sz, _vp]),
    "fd4_selector_status": (_i, [_vp, _ip, _vp]),
    "fd4_select_learned_workspace_bytes": (_sz, [_i, _i, _i, _i]),
    "fd4_selftest_wait_timeout": (_i, [_vp, _sz, _ip, _vp]),
    "fd4_select_scales_learned": (_i, [_vp, _vp, _i, _i, _i, _fp, _i, _pp, ctypes.c_float, _vp, _vp, _vp, _vp,
                                       _sz, _vp]),
}
SIGNATURES.update(SELECTOR_SIGNATURES)


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libfd4.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def strerror(status: int) -> str:
    return lib().fd4_strerror(int(status)).decode()


def _check(rc: int, what: str):
    if rc != 0:
        raise Fd4Error(rc, what)


def params(**kw) -> Params:
    """Defaults of fd4_default_params with keyword overrides (lambda_ for lambda)."""
    p = Params()
    lib().fd4_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def fed_taus(T: float, M: int, tau_max: float = 0.05, n: int = 0, kappa: int = 0):
    """FED step sizes in execution order (fd4_fed_taus).  Returns (tau, kappa)."""
    buf = (ctypes.c_double * MAX_FED_STEPS)()
    n_out, k_out = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().fd4_fed_taus(float(T), int(M), float(tau_max), int(n), int(kappa), buf, MAX_FED_STEPS,
                              ctypes.byref(n_out), ctypes.byref(k_out)), "fd4_fed_taus")
    return np.array(buf[: n_out.value]), k_out.value


def workspace_bytes(op: int, w: int, h: int, n_sigma: int = 0) -> int:
    return int(lib().fd4_workspace_bytes(int(op), int(w), int(h), int(n_sigma)))


# ---------------------------------------------------------------------------
# torch-side helpers (allocation and streams only)

def _torch():
    import torch
    return torch


def pitch_for(w: int) -> int:
    return (int(w) + 3) // 4 * 4


def empty_image(h: int, w: int, dtype=None, channels: int = 0, device="cuda"):
    torch = _torch()
    shape = (h, pitch_for(w)) + ((channels,) if channels else ())
    return torch.zeros(shape, dtype=dtype or torch.float32, device=device)


def to_device(img: np.ndarray, device="cuda"):
    """Copy a (h, w) float image into a zero-padded (h, pitch) float32 device tensor."""
    torch = _torch()
    h, w = img.shape
    buf = empty_image(h, w, device=device)
    buf[:, :w] = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).to(device)
    return buf


def workspace(op: int, w: int, h: int, n_sigma: int = 0, device="cuda"):
    torch = _torch()
    return torch.empty(max(workspace_bytes(op, w, h, n_sigma), 256), dtype=torch.uint8, device=device)


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _sigmas(sigmas):
    arr = (ctypes.c_float * len(sigmas))(*[float(s) for s in sigmas])
    return arr, len(sigmas)


def _pitch(buf):
    return int(buf.shape[1])


def select_scales(img, w: int, sigmas, prm: Params | None = None, want_vmax: bool = False,
                  ws=None, stream=None, idx=None):
    """fd4_select_scales.  Returns (sigma_idx uint8 (h, pitch), vmax or None)."""
    torch = _torch()
    h, pitch = img.shape
    if idx is None:
        idx = torch.zeros((h, pitch), dtype=torch.uint8, device=img.device)
    vmax = torch.zeros((h, pitch), dtype=torch.float32, device=img.device) if want_vmax else None
    sg, K = _sigmas(sigmas)
    if ws is None:
        ws = workspace(OP_SELECT_SCALES, pitch, h, K, img.device)
    _check(lib().fd4_select_scales(_ptr(img), int(w), h, pitch, sg, K,
                                   ctypes.byref(prm) if prm is not None else None, _ptr(idx), _ptr(vmax),
                                   _ptr(ws), ws.numel(), _stream(stream)), "fd4_select_scales")
    return idx, vmax


def postprocess_scales(u, w: int, sigma_idx, vmax, sigmas, prm: Params | None = None, ws=None, stream=None):
    """fd4_postprocess_scales, in place on sigma_idx (uint8 (h, pitch)); vmax is
    the selection's V_max (float32 (h, pitch)).  Returns sigma_idx."""
    h, pitch = u.shape
    sg, K = _sigmas(sigmas)
    if ws is None:
        ws = workspace(OP_POSTPROCESS, pitch, h, K, u.device)
    _check(lib().fd4_postprocess_scales(_ptr(u), int(w), h, pitch, _ptr(sigma_idx), _ptr(vmax), sg, K,
                                        ctypes.byref(prm) if prm is not None else None, _ptr(ws), ws.numel(),
                                        _stream(stream)), "fd4_postprocess_scales")
    return sigma_idx


def extract_creases(u, w: int, sigma: float = 1.0, mode: int = BOTH, max_segs: int = 0, ws=None, stream=None):
    """fd4_extract_creases.  Returns (segments (n, 4) float64 as x0, y0, x1, y1;
    keys (n,)), sorted by key (the cell walk's order)."""
    torch = _torch()
    h, pitch = u.shape
    if max_segs <= 0:
        max_segs = 2 * max(w - 1, 1) * max(h - 1, 1)
    segs = torch.empty((max_segs, 4), dtype=torch.float32, device=u.device)
    keys = torch.empty(max_segs, dtype=torch.int32, device=u.device)
    count = torch.zeros(1, dtype=torch.int32, device=u.device)
    if ws is None:
        ws = workspace(OP_CREASES, pitch, h, 0, u.device)
    _check(lib().fd4_extract_creases(_ptr(u), int(w), h, pitch, float(sigma), int(mode), _ptr(segs), _ptr(keys),
                                     int(max_segs), _ptr(count), _ptr(ws), ws.numel(), _stream(stream)),
           "fd4_extract_creases")
    n = min(int(count.item()), max_segs)
    k = keys[:n].cpu().numpy()
    order = np.argsort(k, kind="stable")
    return segs[:n].cpu().numpy().astype(np.float64)[order], k[order]


def build_tensor_ifod(u, w: int, prm: Params | None = None, out=None, stream=None):
    """fd4_build_tensor_ifod.  Returns the (h, pitch, 4) IFOD tensor field (1, 0, g, g)."""
    torch = _torch()
    h, pitch = u.shape
    if out is None:
        out = torch.zeros((h, pitch, 4), dtype=torch.float32, device=u.device)
    _check(lib().fd4_build_tensor_ifod(_ptr(u), int(w), h, pitch, ctypes.byref(prm) if prm is not None else None,
                                       _ptr(out), _stream(stream)), "fd4_build_tensor_ifod")
    return out


def build_tensor(u, w: int, sigma_idx, sigmas, prm: Params | None = None, out=None, ws=None, stream=None):
    """fd4_build_tensor.  Returns the (h, pitch, 4) tensor field."""
    torch = _torch()
    h, pitch = u.shape
    if out is None:
        out = torch.zeros((h, pitch, 4), dtype=torch.float32, device=u.device)
    sg, K = _sigmas(sigmas)
    if ws is None:
        ws = workspace(OP_BUILD_TENSOR, pitch, h, K, u.device)
    _check(lib().fd4_build_tensor(_ptr(u), int(w), h, pitch, _ptr(sigma_idx), sg, K,
                                  ctypes.byref(prm) if prm is not None else None, _ptr(out), _ptr(ws),
                                  ws.numel(), _stream(stream)), "fd4_build_tensor")
    return out


def fed_cycle(u, w: int, tensor, tau, boundary: int = NATURAL, ws=None, stream=None, sched=None):
    """fd4_fed_cycle, in place on u; sched = (steps per launch, tile rows, quads
    per thread) runs fd4_fed_cycle_sched with that kernel schedule instead."""
    h, pitch = u.shape
    t = np.ascontiguousarray(tau, dtype=np.float64)
    if ws is None:
        ws = workspace(OP_FED_CYCLE, pitch, h, 0, u.device)
    if sched is None:
        _check(lib().fd4_fed_cycle(_ptr(u), int(w), h, pitch, _ptr(tensor), t.ctypes.data_as(_dp), t.size,
                                   int(boundary), _ptr(ws), ws.numel(), _stream(stream)), "fd4_fed_cycle")
    else:
        steps, rows, quads = (int(x) for x in sched)
        _check(lib().fd4_fed_cycle_sched(_ptr(u), int(w), h, pitch, _ptr(tensor), t.ctypes.data_as(_dp), t.size,
                                         int(boundary), steps, rows, quads, _ptr(ws), ws.numel(), _stream(stream)),
               "fd4_fed_cycle_sched")
    return u


def measure_fma_rate(stream=None):
    """fd4_measure_fma_rate: (scalar, packed-pair) FP32 FMA rates in 1e12 FMA/s."""
    torch = _torch()
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().fd4_measure_fma_rate(_ptr(buf), buf.numel(), ctypes.byref(a), ctypes.byref(b), _stream(stream)),
           "fd4_measure_fma_rate")
    return a.value, b.value


def selftest_fed_wait_timeout(u, w: int, tensor, ws=None, stream=None) -> int:
    """Runs fd4_selftest_fed_wait_timeout on u (left unchanged); returns the
    device status word it read (FD4_ERR_TIMEOUT when detection works)."""
    h, pitch = u.shape
    if ws is None:
        ws = workspace(OP_FED_CYCLE, pitch, h, 0, u.device)
    st = ctypes.c_int(0)
    _check(lib().fd4_selftest_fed_wait_timeout(_ptr(u), int(w), h, pitch, _ptr(tensor), _ptr(ws), ws.numel(),
                                               ctypes.byref(st), _stream(stream)), "fd4_selftest_fed_wait_timeout")
    return st.value


def filter_image(u_in, w: int, sigmas, T: float, M: int, n: int = 0, prm: Params | None = None,
                 sigma_idx=None, out=None, ws=None, stream=None, keep_idx: bool = True):
    """fd4_filter.  Returns (out, sigma_idx); sigma_idx is None if not kept."""
    torch = _torch()
    h, pitch = u_in.shape
    if out is None:
        out = torch.zeros_like(u_in)
    given = sigma_idx is not None
    if sigma_idx is None and keep_idx:
        sigma_idx = torch.zeros((h, pitch), dtype=torch.uint8, device=u_in.device)
    sg, K = _sigmas(sigmas)
    if ws is None:
        ws = workspace(OP_FILTER, pitch, h, K, u_in.device)
    _check(lib().fd4_filter(_ptr(u_in), _ptr(out), int(w), h, pitch, sg, K,
                            ctypes.byref(prm) if prm is not None else None, float(T), int(M), int(n),
                            _ptr(sigma_idx), int(given), _ptr(ws), ws.numel(), _stream(stream)),
           "fd4_filter")
    return out, sigma_idx


def fed_cycle_noalloc(u, w: int, tensor, tau, boundary: int = NATURAL, stream=None):
    """fd4_fed_cycle_noalloc, in place on u: the FED cycle without a workspace,
    for callers that cannot allocate device memory (scratch is built into the
    library; see include/fd4.h)."""
    h, pitch = u.shape
    t = np.ascontiguousarray(tau, dtype=np.float64)
    _check(lib().fd4_fed_cycle_noalloc(_ptr(u), int(w), h, pitch, _ptr(tensor), t.ctypes.data_as(_dp),
                                       t.size, int(boundary), _stream(stream)), "fd4_fed_cycle_noalloc")
    return u


# ---------------------------------------------------------------------------
# Batches

def image_list(inputs, widths, outputs=None, sigma_idx=None):
    """ctypes array of fd4_image for device tensors (h, pitch) with widths w."""
    n = len(inputs)
    arr = (Image * n)()
    for i, (u, w) in enumerate(zip(inputs, widths)):
        arr[i].d_in = u.data_ptr()
        arr[i].d_out = (outputs[i] if outputs is not None else u).data_ptr()
        arr[i].d_sigma_idx = sigma_idx[i].data_ptr() if sigma_idx is not None else None
        arr[i].w, arr[i].h, arr[i].pitch = int(w), int(u.shape[0]), int(u.shape[1])
    return arr


def batch_workspace(imgs, n_sigma: int, device="cuda"):
    torch = _torch()
    nbytes = int(lib().fd4_batch_workspace_bytes(ctypes.cast(imgs, ctypes.c_void_p), len(imgs), n_sigma))
    if nbytes == 0:
        raise Fd4Error(-1, "fd4_batch_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def filter_batched(imgs, sigmas, T: float, M: int, n: int = 0, prm: Params | None = None,
                   sigma_given: bool = False, ws=None, stream=None):
    """fd4_filter_batched on an image_list()."""
    sg, K = _sigmas(sigmas)
    if ws is None:
        ws = batch_workspace(imgs, K)
    _check(lib().fd4_filter_batched(ctypes.cast(imgs, ctypes.c_void_p), len(imgs), sg, K,
                                    ctypes.byref(prm) if prm is not None else None, float(T), int(M), int(n),
                                    int(sigma_given), _ptr(ws), ws.numel(), _stream(stream)),
           "fd4_filter_batched")
    return ws


def device_status(reset: bool = False) -> int:
    """fd4_device_status: the FED kernels' device status word (0 or FD4_ERR_TIMEOUT)."""
    st = ctypes.c_int(0)
    _check(lib().fd4_device_status(ctypes.byref(st), int(reset)), "fd4_device_status")
    return st.value


class Graph:
    """fd4_graph: the batched schedule captured once, replayed by launch()."""

    def __init__(self, imgs, sigmas, T: float, M: int, n: int = 0, prm: Params | None = None,
                 sigma_given: bool = False, ws=None, stages: int = 15):
        sg, K = _sigmas(sigmas)
        self.ws = ws if ws is not None else batch_workspace(imgs, K)
        self.imgs = imgs
        h = ctypes.c_void_p(0)
        _check(lib().fd4_graph_create(ctypes.cast(imgs, ctypes.c_void_p), len(imgs), sg, K,
                                      ctypes.byref(prm) if prm is not None else None, float(T), int(M),
                                      int(n), int(sigma_given), int(stages), _ptr(self.ws), self.ws.numel(),
                                      ctypes.byref(h)), "fd4_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib().fd4_graph_launch(self.handle, _stream(stream)), "fd4_graph_launch")

    def kernel_count(self) -> int:
        """fd4_graph_kernel_count: kernel launches per launch()."""
        n = ctypes.c_int(0)
        _check(lib().fd4_graph_kernel_count(self.handle, ctypes.byref(n)), "fd4_graph_kernel_count")
        return n.value

    def close(self):
        if self.handle:
            lib().fd4_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_batched(imgs, sigmas, T: float, M: int, n: int = 0, prm: Params | None = None, ws=None,
                     stream=None):
    """fd4_autotune_batched.  Returns (the fastest FedSchedule, every candidate's
    FedSchedule with its time); best.as_params() gives its fd4_params fields."""
    sg, K = _sigmas(sigmas)
    if ws is None:
        ws = batch_workspace(imgs, K)
    best = FedSchedule()
    tried = (FedSchedule * AUTOTUNE_CANDIDATES)()
    _check(lib().fd4_autotune_batched(ctypes.cast(imgs, ctypes.c_void_p), len(imgs), sg, K,
                                      ctypes.byref(prm) if prm is not None else None, float(T), int(M), int(n),
                                      _ptr(ws), ws.numel(), _stream(stream), ctypes.byref(best), tried),
           "fd4_autotune_batched")
    return best, list(tried)


# ---------------------------------------------------------------------------
# Learned scale selector (network weights live in a caller-owned device buffer)

SEL_MAX_BINS = 16  # FD4_SELECTOR_MAX_BINS: outputs of the last layer, the first n_bins used
SEL_LAYERS = [(1, 32), (32, 32), (32, 32), (32, SEL_MAX_BINS)]  # (in, out) channels


def selector_n_master() -> int:
    return sum(9 * co * ci + co for ci, co in SEL_LAYERS)


class Selector:
    """Parameters of the learned selector on the device and the calls on them."""

    def __init__(self, device="cuda"):
        torch = _torch()
        self.device = device
        self.params = torch.zeros(int(lib().fd4_selector_param_bytes()), dtype=torch.uint8, device=device)

    def init(self, seed: int, stream=None):
        _check(lib().fd4_selector_init(_ptr(self.params), int(seed), _stream(stream)), "fd4_selector_init")

    def set_weights(self, flat: np.ndarray, stream=None):
        f = np.ascontiguousarray(flat, dtype=np.float32)
        assert f.size == selector_n_master()
        _check(lib().fd4_selector_set_weights(_ptr(self.params), f.ctypes.data_as(_fp), _stream(stream)),
               "fd4_selector_set_weights")

    def get(self, which: int = 0, stream=None) -> np.ndarray:
        """which: 0 weights, 1 Adam m, 2 Adam v, 3 accumulated gradients."""
        f = np.zeros(selector_n_master(), dtype=np.float32)
        _check(lib().fd4_selector_get_weights(_ptr(self.params), f.ctypes.data_as(_fp), int(which),
                                              _stream(stream)), "fd4_selector_get_weights")
        return f

    @staticmethod
    def workspace(n_img: int, w: int, h: int, pitch: int, device="cuda", infer: bool = False):
        """Workspace of grad (training), or of forward / predict with infer=True."""
        torch = _torch()
        fn = lib().fd4_selector_infer_workspace_bytes if infer else lib().fd4_selector_workspace_bytes
        return torch.empty(int(fn(n_img, w, h, pitch)), dtype=torch.uint8, device=device)

    def forward(self, imgs, w: int, n_bins: int = 8, ws=None, stream=None):
        """imgs: (n, h, pitch) float32 -> logits (n, h, pitch, n_bins)."""
        torch = _torch()
        n, h, pitch = imgs.shape
        ws = ws if ws is not None else self.workspace(n, w, h, pitch, imgs.device, infer=True)
        out = torch.empty((n, h, pitch, n_bins), dtype=torch.float32, device=imgs.device)
        _check(lib().fd4_selector_forward(_ptr(self.params), _ptr(imgs), n, int(w), h, pitch, int(n_bins), _ptr(out),
                                          _ptr(ws), ws.numel(), _stream(stream)), "fd4_selector_forward")
        return out

    def grad(self, imgs, labels, w: int, loss, n_bins: int = 8, ws=None, stream=None):
        """Adds the loss gradient of the batch to the parameter buffer; loss += mean CE."""
        n, h, pitch = imgs.shape
        ws = ws if ws is not None else self.workspace(n, w, h, pitch, imgs.device)
        _check(lib().fd4_selector_grad(_ptr(self.params), _ptr(imgs), _ptr(labels), n, int(w), h, pitch,
                                       int(n_bins), _ptr(loss), _ptr(ws), ws.numel(), _stream(stream)),
               "fd4_selector_grad")

    def update(self, lr: float, step: int, stream=None):
        _check(lib().fd4_selector_update(_ptr(self.params), float(lr), int(step), _stream(stream)),
               "fd4_selector_update")

    def predict(self, img, w: int, n_bins: int = 8, idx=None, conf=None, ws=None, stream=None):
        """img: (h, pitch) or a stack (n, h, pitch) of float32 -> (scale index uint8,
        confidence float32), both of img's shape (one launch per layer for the stack)."""
        torch = _torch()
        n, h, pitch = (1,) + tuple(img.shape) if img.dim() == 2 else tuple(img.shape)
        ws = ws if ws is not None else self.workspace(n, w, h, pitch, img.device, infer=True)
        if idx is None:
            idx = torch.zeros(img.shape, dtype=torch.uint8, device=img.device)
        if conf is None:
            conf = torch.zeros(img.shape, dtype=torch.float32, device=img.device)
        _check(lib().fd4_selector_predict(_ptr(self.params), _ptr(img), n, int(w), h, pitch, int(n_bins), _ptr(idx),
                                          _ptr(conf), _ptr(ws), ws.numel(), _stream(stream)), "fd4_selector_predict")
        return idx, conf

    def select_learned(self, img, w: int, sigmas, prm: Params | None = None, conf_threshold: float = 0.5,
                       idx=None, ws=None, stream=None):
        """fd4_select_scales_learned: (scale index, confidence, device count of fallback tiles)."""
        torch = _torch()
        h, pitch = img.shape
        sg, K = _sigmas(sigmas)
        if ws is None:
            ws = torch.empty(int(lib().fd4_select_learned_workspace_bytes(int(w), h, pitch, K)), dtype=torch.uint8,
                             device=img.device)
        if idx is None:
            idx = torch.zeros((h, pitch), dtype=torch.uint8, device=img.device)
        conf = None
        nfb = torch.zeros(1, dtype=torch.int32, device=img.device)
        _check(lib().fd4_select_scales_learned(_ptr(self.params), _ptr(img), int(w), h, pitch, sg, K,
                                               ctypes.byref(prm) if prm is not None else None,
                                               float(conf_threshold), _ptr(idx), _ptr(conf), _ptr(nfb), _ptr(ws),
                                               ws.numel(), _stream(stream)), "fd4_select_scales_learned")
        return idx, conf, nfb

    @staticmethod
    def status(ws, stream=None) -> int:
        st = ctypes.c_int(0)
        _check(lib().fd4_selector_status(_ptr(ws), ctypes.byref(st), _stream(stream)), "fd4_selector_status")
        return st.value


def selftest_wait_timeout(stream=None) -> int:
    """Runs fd4_selftest_wait_timeout; returns the device status word it read."""
    torch = _torch()
    ws = torch.empty(int(lib().fd4_selector_workspace_bytes(1, 128, 4, 128)), dtype=torch.uint8, device="cuda")
    st = ctypes.c_int(0)
    _check(lib().fd4_selftest_wait_timeout(_ptr(ws), ws.numel(), ctypes.byref(st), _stream(stream)),
           "fd4_selftest_wait_timeout")
    return st.value
