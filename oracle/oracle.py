"""FP64 CPU oracle for the MAFOD hot path -- ctypes wrapper around fd4_oracle.c.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA library and never calls it.  All arrays are float64 numpy
arrays in row-major (y, x) layout; the tensor field is four planes
(cos 2theta, sin 2theta, mu1, mu2) stacked along axis 0.

Section and equation numbers refer to arXiv:1611.06906 (Sec. 3, "Method").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd4_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfd4_oracle.so")
_lock = threading.Lock()
_lib = None

RIDGE, VALLEY, BOTH = 0, 1, 2
NATURAL, PERIODIC = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile fd4_oracle.c into oracle/_build (OpenMP if the compiler has it)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.or_gauss_radius.restype = ctypes.c_int
        lib.or_gauss_radius.argtypes = [ctypes.c_double]
        lib.or_gauss_kernels.argtypes = [ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
        lib.or_derivatives.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       _dp, _dp, _dp, _dp, _dp]
        lib.or_derivative_direct.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, _dp]
        lib.or_select_scales.restype = ctypes.c_double
        lib.or_select_scales.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _u8p, _dp, _dp]
        lib.or_build_tensor.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _u8p, _dp, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, _dp, _dp]
        lib.or_tensor_matrix.argtypes = [ctypes.c_double] * 4 + [_dp]
        lib.or_apply_P.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]
        lib.or_fed_taus.restype = ctypes.c_int
        lib.or_fed_taus.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), _dp]
        lib.or_fed_cycle.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                     ctypes.c_int]
        lib.or_filter.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _u8p,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.or_build_tensor_ifod.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, _dp]
        lib.or_filter_ifod.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int]
        lib.or_crease_field.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]
        lib.or_marching_squares.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                            ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        lib.or_marching_squares.restype = ctypes.c_int
        lib.or_strong_direction.argtypes = [ctypes.c_double] * 3 + [_dp, _dp]
        lib.or_strong_direction.restype = ctypes.c_int
        lib.or_postprocess_core.argtypes = [_u8p, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int]
        lib.or_postprocess_scales.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _u8p, _dp, _dp,
                                              ctypes.c_int, ctypes.c_double]
        lib.or_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's pixel-row loops from now on (results do not depend on it)."""
    lib = _load()
    lib.or_set_num_threads.argtypes = [ctypes.c_int]
    lib.or_set_num_threads(int(n))


def gauss_radius(sigma: float) -> int:
    return int(_load().or_gauss_radius(float(sigma)))


def gauss_kernels(sigma: float):
    """Sampled correlation weights (w0, w1, w2) on offsets -r..r (Sec. 3.1, Eq. 6)."""
    r = gauss_radius(sigma)
    w0, w1, w2 = (np.zeros(2 * r + 1) for _ in range(3))
    _load().or_gauss_kernels(float(sigma), r, _d(w0), _d(w1), _d(w2))
    return w0, w1, w2


def derivatives(u, sigma: float):
    """(ux, uy, uxx, uxy, uyy) of u_sigma = u * G_sigma (Sec. 3.1, Eq. 6)."""
    u = _f64(u)
    h, w = u.shape
    outs = [np.zeros((h, w)) for _ in range(5)]
    _load().or_derivatives(_d(u), w, h, float(sigma), *[_d(o) for o in outs])
    return tuple(outs)


def derivative_direct(u, sigma: float, order_x: int, order_y: int):
    u = _f64(u)
    h, w = u.shape
    out = np.zeros((h, w))
    _load().or_derivative_direct(_d(u), w, h, float(sigma), order_x, order_y, _d(out))
    return out


def select_scales(u, sigmas, mode=RIDGE, beta=0.5, c=0.0, gamma=1.0):
    """Vesselness scale selection (Sec. 3.3, Eq. 9).

    Returns (sigma_idx uint8 (h, w), v_max (h, w), v_all (K, h, w), c_used)."""
    u = _f64(u)
    h, w = u.shape
    sig = _f64(sigmas)
    K = sig.size
    idx = np.zeros((h, w), dtype=np.uint8)
    vmax = np.zeros((h, w))
    vall = np.zeros((K, h, w))
    c_used = _load().or_select_scales(_d(u), w, h, _d(sig), K, int(mode), float(beta), float(c),
                                      float(gamma), idx.ctypes.data_as(_u8p), _d(vmax), _d(vall))
    return idx, vmax, vall, float(c_used)


def build_tensor(u, sigma_idx, sigmas, lam=0.005, rho=0.5, mode=RIDGE, grad_sq=False):
    """Tensor field (cos2th, sin2th, mu1, mu2) as (4, h, w) plus N_rho (3, h, w).

    Sec. 3.1 Eq. 6 (normalised Hessian), Sec. 3.2 Eq. 7-8 (diffusivities)."""
    u = _f64(u)
    h, w = u.shape
    idx = np.ascontiguousarray(sigma_idx, dtype=np.uint8)
    assert idx.shape == (h, w)
    sig = _f64(sigmas)
    tensor = np.zeros((4, h, w))
    nrho = np.zeros((3, h, w))
    _load().or_build_tensor(_d(u), w, h, idx.ctypes.data_as(_u8p), _d(sig), sig.size, float(lam),
                            float(rho), int(mode), int(bool(grad_sq)), _d(tensor), _d(nrho))
    return tensor, nrho


def tensor_matrix(c2, s2, mu1, mu2):
    """4x4 D_i = E diag(mu1, mu2, (mu1+mu2)/2, 0) E^T on (xx, xy, yx, yy) (Sec. 3.4)."""
    D = np.zeros(16)
    _load().or_tensor_matrix(float(c2), float(s2), float(mu1), float(mu2), _d(D))
    return D.reshape(4, 4)


def apply_P(u, tensor, boundary=NATURAL):
    """P u = L^T D L u (Sec. 3.4, Eq. 17)."""
    u = _f64(u)
    h, w = u.shape
    t = _f64(tensor)
    assert t.shape == (4, h, w)
    out = np.zeros((h, w))
    _load().or_apply_P(_d(u), w, h, _d(t), int(boundary), _d(out))
    return out


class UnstableTau(ValueError):
    pass


def fed_taus(T: float, M: int, tau_max: float = 0.05, n: int = 0, kappa: int = 0):
    """FED step sizes (Sec. 3.5, Eq. 22-23), ordered.  Returns (tau, kappa, amplification)."""
    nmax = max(int(n), 1)
    if n == 0:
        nmax = int(np.ceil(-0.5 + 0.5 * np.sqrt(1.0 + 12.0 * T / (M * tau_max)))) + 2
    tau = np.zeros(nmax)
    n_out = ctypes.c_int(0)
    k_out = ctypes.c_int(0)
    amp = np.zeros(1)
    rc = _load().or_fed_taus(float(T), int(M), float(tau_max), int(n), int(kappa), _d(tau),
                             ctypes.byref(n_out), ctypes.byref(k_out), _d(amp))
    if rc == -1:
        raise UnstableTau("3T/(M(n^2+n)) exceeds tau_max")
    if rc != 0:
        raise ValueError("bad FED arguments")
    return tau[: n_out.value].copy(), int(k_out.value), float(amp[0])


def fed_cycle(u, tensor, tau, boundary=NATURAL):
    """One FED cycle u <- prod_i (I - tau_i P) u (Sec. 3.5, Eq. 21).  Returns a new array."""
    u = _f64(u).copy()
    h, w = u.shape
    t = _f64(tensor)
    tau = _f64(tau)
    _load().or_fed_cycle(_d(u), w, h, _d(t), _d(tau), tau.size, int(boundary))
    return u


def build_tensor_ifod(u, sigma=1.0, lam=0.005):
    """IFOD tensor field (1, 0, g, g) as (4, h, w), g = 1 / (1 + ||H(u_sigma)||_F^2 / lambda^2) (Eq. 2)."""
    u = _f64(u)
    h, w = u.shape
    t = np.zeros((4, h, w))
    _load().or_build_tensor_ifod(_d(u), w, h, float(sigma), float(lam), _d(t))
    return t


def filter_ifod(u, tau, M, sigma=1.0, lam=0.005, boundary=NATURAL):
    """The IFOD filter: M cycles of (IFOD tensor from u^k, FED cycle).  Returns a new array."""
    u = _f64(u).copy()
    h, w = u.shape
    tau = _f64(tau)
    _load().or_filter_ifod(_d(u), w, h, float(sigma), float(lam), int(boundary), _d(tau), tau.size, int(M))
    return u


def crease_field(u, sigma=1.0):
    """d = det(g | Hg) and the strongest Hessian eigenvalue of u_sigma, each (h, w) (Sec. 4)."""
    u = _f64(u)
    h, w = u.shape
    d, nu = np.zeros((h, w)), np.zeros((h, w))
    _load().or_crease_field(_d(u), w, h, float(sigma), _d(d), _d(nu))
    return d, nu


def marching_squares(d, nu, mode=BOTH):
    """Zero-contour segments of d kept by the crease-type filter on nu.
    Returns (segments (n, 4) as x0, y0, x1, y1; keys (n,) = 2 * cell + k)."""
    d, nu = _f64(d), _f64(nu)
    h, w = d.shape
    cap = 2 * max(w - 1, 1) * max(h - 1, 1)
    segs = np.zeros((cap, 4))
    keys = np.zeros(cap, dtype=np.int32)
    n = _load().or_marching_squares(_d(d), _d(nu), w, h, int(mode), _d(segs),
                                    keys.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap)
    return segs[:n].copy(), keys[:n].copy()


def extract_creases(u, sigma=1.0, mode=BOTH):
    """Crease extraction of Sec. 4 on u: marching squares on det(g | Hg) of u_sigma."""
    d, nu = crease_field(u, sigma)
    return marching_squares(d, nu, mode)


def strong_direction(a, b, d):
    """Unit eigenvector of [a b; b d] for its eigenvalue of largest magnitude
    (the negative one on a tie), or None for equal eigenvalues."""
    ex, ey = np.zeros(1), np.zeros(1)
    if not _load().or_strong_direction(float(a), float(b), float(d), _d(ex), _d(ey)):
        return None
    return float(ex[0]), float(ey[0])


def postprocess_core(sigma_idx, vmax, hxx, hxy, hyy, sigmas, theta, cap):
    """Scale-image post-processing (Sec. 3.3, after Eq. 9) from given Hessian
    fields; returns the new scale index image."""
    idx = np.ascontiguousarray(sigma_idx, dtype=np.uint8).copy()
    h, w = idx.shape
    f = [_f64(a) for a in (vmax, hxx, hxy, hyy)]
    assert all(a.shape == (h, w) for a in f)
    sig = _f64(sigmas)
    _load().or_postprocess_core(idx.ctypes.data_as(_u8p), _d(f[0]), _d(f[1]), _d(f[2]), _d(f[3]), w, h,
                                _d(sig), sig.size, float(theta), int(cap))
    return idx


def postprocess_scales(u, sigma_idx, vmax, sigmas, theta):
    """Scale-image post-processing of the scale image selected on u (Hessian at
    each pixel's selected scale, walk capped at ceil(4 sigma_max))."""
    u = _f64(u)
    h, w = u.shape
    idx = np.ascontiguousarray(sigma_idx, dtype=np.uint8).copy()
    vm = _f64(vmax)
    sig = _f64(sigmas)
    _load().or_postprocess_scales(_d(u), w, h, idx.ctypes.data_as(_u8p), _d(vm), _d(sig), sig.size,
                                  float(theta))
    return idx


def filter_image(u, sigmas, tau, M, lam=0.005, rho=0.5, beta=0.5, c=0.0, gamma=1.0,
                 mode=RIDGE, grad_sq=False, boundary=NATURAL, sigma_idx=None, reselect=False,
                 postprocess=False, theta=0.2):
    """Whole MAFOD filter (Sec. 3).  Returns (filtered u, sigma_idx).

    reselect: the scale image is selected again on the current image before
    every cycle (otherwise once, on the input); postprocess: every selection is
    followed by the scale-image post-processing at threshold theta; sigma_idx
    returned is the last (post-processed) selection."""
    u = _f64(u).copy()
    h, w = u.shape
    sig = _f64(sigmas)
    tau = _f64(tau)
    if sigma_idx is None:
        idx = np.zeros((h, w), dtype=np.uint8)
        given = 0
    else:
        idx = np.ascontiguousarray(sigma_idx, dtype=np.uint8).copy()
        given = 1
    _load().or_filter(_d(u), w, h, _d(sig), sig.size, float(lam), float(rho), float(beta),
                      float(c), float(gamma), int(mode), int(bool(grad_sq)), int(boundary),
                      _d(tau), tau.size, int(M), idx.ctypes.data_as(_u8p), given,
                      int(bool(reselect)), int(bool(postprocess)), float(theta))
    return u, idx
