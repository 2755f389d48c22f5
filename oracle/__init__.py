"""FP64 CPU oracle for DISK (arXiv 2512.04556) -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it, and the two share no code: this module
wraps ``disk_oracle.c`` (plain C, FP64, OpenMP over rows) through ctypes and
adds thin numpy conveniences.  Each wrapper names the paper passage that the C
routine implements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "disk_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile disk_oracle.c into oracle/_lib/liboracle.so with gcc."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            l.orc_num_threads.restype = ctypes.c_int
            l.orc_splitmix64.restype = ctypes.c_uint64
            l.orc_splitmix64.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
            l.orc_locate.argtypes = [ctypes.c_double, _dp, ctypes.c_int, _ip, _dp]
            l.orc_alpha.argtypes = [_dp, ctypes.c_int, _ip, _dp, _dp]
            l.orc_blend.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
            l.orc_layer.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, _dp, ctypes.c_long, ctypes.c_int]
            sv_args = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                       _ip, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
            l.orc_sv_filter.argtypes = sv_args
            l.orc_sv_filter_adjoint.argtypes = sv_args
            l.orc_sv_filter_rot.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                            ctypes.c_int, _ip, _dp, ctypes.c_int, ctypes.c_int,
                                            _dp, _dp]
            l.orc_sv_filter_grad_theta.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, _dp, ctypes.c_int, _ip, _dp,
                                                   ctypes.c_int, ctypes.c_int, _dp, _dp]
            l.orc_support_radius.argtypes = [_dp, ctypes.c_int, ctypes.c_int]
            l.orc_synth_canvas.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
            l.orc_synth.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
            l.orc_fit_loss.restype = ctypes.c_double
            l.orc_fit_loss.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, _dp]
            l.orc_init_ir.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
            l.orc_init_ss.restype = ctypes.c_long
            l.orc_init_ss.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_uint64, _dp]
            l.orc_init_rand.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_uint64, _dp]
            l.orc_fit.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_uint64, _dp, _dp]
            l.orc_dense_sv.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                       ctypes.c_int, _ip, _dp, _dp, ctypes.c_int, _dp]
            _lib = l
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def num_threads() -> int:
    return lib().orc_num_threads()


def splitmix64(seed: int, n: int) -> list[int]:
    """n successive SplitMix64 outputs from state ``seed``."""
    st = ctypes.c_uint64(seed)
    return [lib().orc_splitmix64(ctypes.byref(st)) for _ in range(n)]


def locate(p: float, nodes) -> tuple[int, float]:
    """Eq. 9, one axis: lower node index and blend t."""
    nd, ndp = _d(nodes)
    k = ctypes.c_int()
    t = ctypes.c_double()
    lib().orc_locate(float(p), ndp, len(nd), ctypes.byref(k), ctypes.byref(t))
    return k.value, t.value


def alpha(pv, n_nodes, node_vals) -> np.ndarray:
    """Eq. 9 weight vector over all basis nodes."""
    n_nodes = list(n_nodes)
    B = int(np.prod(n_nodes))
    pv, pvp = _d(pv)
    nn, nnp = _i(n_nodes)
    nv, nvp = _d(node_vals)
    out = np.zeros(B)
    lib().orc_alpha(pvp, len(n_nodes), nnp, nvp, out.ctypes.data_as(_dp))
    return out


def layer(img, taps, boundary: str = "clamp") -> np.ndarray:
    """Eq. 3, one layer.  img [H][W][C]; taps [T][3] (shift invariant) or
    [H][W][T][3] (per pixel)."""
    img, ip = _d(img)
    H, W, C = img.shape
    taps, tp = _d(taps)
    T = taps.shape[-2]
    stride = 0 if taps.ndim == 2 else T * 3
    out = np.zeros_like(img)
    lib().orc_layer(ip, out.ctypes.data_as(_dp), H, W, C, T, tp, stride,
                    0 if boundary == "clamp" else 1)
    return out


def _basis_args(n_nodes, node_vals, theta):
    nn, nnp = _i(list(n_nodes))
    nv, nvp = _d(node_vals)
    th, thp = _d(theta)
    return nn, nnp, nv, nvp, th, thp


def sv_filter(img, maps, n_nodes, node_vals, theta) -> np.ndarray:
    """Spatially varying filter: Eq. 3 with the per-pixel complex of Eq. 9.
    img [H][W][C]; maps [dims][H][W]; theta [B][L][T][3] (pixel offsets)."""
    img, ip = _d(img)
    H, W, C = img.shape
    maps, mp = _d(np.reshape(maps, (-1, H, W)))
    nn, nnp, nv, nvp, th, thp = _basis_args(n_nodes, node_vals, theta)
    B, L, T, _ = th.shape
    out = np.zeros_like(img)
    rc = lib().orc_sv_filter(ip, H, W, C, mp, len(nn), nnp, nvp, L, T, thp,
                             out.ctypes.data_as(_dp))
    if rc:
        raise ValueError(f"orc_sv_filter failed ({rc})")
    return out


def sv_filter_rotated(img, maps, angle, n_nodes, node_vals, theta) -> np.ndarray:
    """sv_filter with every pixel's blended tap offsets rotated by angle[H][W]
    (radians, x right, y down): (dx, dy) -> (dx cos a - dy sin a, dx sin a + dy cos a)."""
    img, ip = _d(img)
    H, W, C = img.shape
    maps, mp = _d(np.reshape(maps, (-1, H, W)))
    ang, ap = _d(np.reshape(angle, (H, W)))
    nn, nnp, nv, nvp, th, thp = _basis_args(n_nodes, node_vals, theta)
    B, L, T, _ = th.shape
    out = np.zeros_like(img)
    rc = lib().orc_sv_filter_rot(ip, H, W, C, mp, ap, len(nn), nnp, nvp, L, T, thp,
                                 out.ctypes.data_as(_dp))
    if rc:
        raise ValueError(f"orc_sv_filter_rot failed ({rc})")
    return out


def sv_filter_adjoint(g_out, maps, n_nodes, node_vals, theta) -> np.ndarray:
    """Transpose of sv_filter with respect to the image."""
    g, gp = _d(g_out)
    H, W, C = g.shape
    maps, mp = _d(np.reshape(maps, (-1, H, W)))
    nn, nnp, nv, nvp, th, thp = _basis_args(n_nodes, node_vals, theta)
    B, L, T, _ = th.shape
    out = np.zeros_like(g)
    rc = lib().orc_sv_filter_adjoint(gp, H, W, C, mp, len(nn), nnp, nvp, L, T, thp,
                                     out.ctypes.data_as(_dp))
    if rc:
        raise ValueError(f"orc_sv_filter_adjoint failed ({rc})")
    return out


def sv_filter_grad_theta(img, g_out, maps, n_nodes, node_vals, theta) -> np.ndarray:
    """d<g_out, sv_filter(img)>/d theta [B][L][T][3] (Eq. 9 blend is linear in theta)."""
    img, ip = _d(img)
    H, W, C = img.shape
    g, gp = _d(g_out)
    maps, mp = _d(np.reshape(maps, (-1, H, W)))
    nn, nnp, nv, nvp, th, thp = _basis_args(n_nodes, node_vals, theta)
    B, L, T, _ = th.shape
    out = np.zeros_like(th)
    rc = lib().orc_sv_filter_grad_theta(ip, gp, H, W, C, mp, len(nn), nnp, nvp, L, T, thp,
                                        out.ctypes.data_as(_dp))
    if rc:
        raise ValueError(f"orc_sv_filter_grad_theta failed ({rc})")
    return out


def support_radius(theta) -> int:
    th, tp = _d(theta)
    L, T, _ = th.shape
    return lib().orc_support_radius(tp, L, T)


def synth_canvas(theta, R: int, with_acts: bool = False):
    """Eq. 10 on a zero-padded canvas of half-width R."""
    th, tp = _d(theta)
    L, T, _ = th.shape
    N = 2 * R + 1
    out = np.zeros((N, N))
    acts = np.zeros((L + 1, N, N)) if with_acts else None
    rc = lib().orc_synth_canvas(tp, L, T, R, out.ctypes.data_as(_dp),
                                acts.ctypes.data_as(_dp) if with_acts else None)
    if rc:
        raise ValueError(f"orc_synth_canvas failed ({rc})")
    return (out, acts) if with_acts else out


def synth(theta, K: int) -> np.ndarray:
    """Eq. 10: impulse response of complex theta [L][T][3], cropped K x K."""
    th, tp = _d(theta)
    L, T, _ = th.shape
    out = np.zeros((K, K))
    rc = lib().orc_synth(tp, L, T, K, out.ctypes.data_as(_dp))
    if rc:
        raise ValueError(f"orc_synth failed ({rc})")
    return out


LOSS_MSE, LOSS_CHARB = 0, 1


def fit_loss(theta, target, loss: int = LOSS_MSE, eps: float = 0.0, grad: bool = False):
    """Eq. 4 objective with impulse supervision (Eq. 10-11) and its gradient."""
    th, tp = _d(theta)
    L, T, _ = th.shape
    tg, tgp = _d(target)
    K = tg.shape[0]
    g = np.zeros_like(th) if grad else None
    v = lib().orc_fit_loss(tp, L, T, tgp, K, loss, eps,
                           g.ctypes.data_as(_dp) if grad else None)
    return (v, g) if grad else v


def init_ir(target, L: int, T: int) -> np.ndarray:
    """Eq. 6 radial initialisation."""
    tg, tgp = _d(target)
    th = np.zeros((L, T, 3))
    lib().orc_init_ir(tgp, tg.shape[0], L, T, th.ctypes.data_as(_dp))
    return th


def init_ss(target, L: int, T: int, seed: int):
    """Sec. 4.2 sparse-sampling initialisation (Eq. 7).  Returns (theta, draws)."""
    tg, tgp = _d(target)
    th = np.zeros((L, T, 3))
    n = lib().orc_init_ss(tgp, tg.shape[0], L, T, ctypes.c_uint64(seed), th.ctypes.data_as(_dp))
    return th, n


def init_rand(K: int, L: int, T: int, seed: int) -> np.ndarray:
    th = np.zeros((L, T, 3))
    lib().orc_init_rand(K, L, T, ctypes.c_uint64(seed), th.ctypes.data_as(_dp))
    return th


INIT_GIVEN, INIT_IR, INIT_SS, INIT_RAND = 0, 1, 2, 3


def fit(target, L: int, T: int, steps: int, lr0: float = 1e-3, lr1: float = 1e-4,
        init: int = INIT_IR, loss: int = LOSS_MSE, eps: float = 0.0, seed: int = 0,
        theta0=None):
    """Eq. 4 fit with Adam and linear lr decay (Sec. 5.1).
    Returns (theta [L][T][3] in pixels, loss history [steps+1])."""
    tg, tgp = _d(target)
    th = np.zeros((L, T, 3)) if theta0 is None else np.array(theta0, dtype=np.float64)
    th = np.ascontiguousarray(th)
    hist = np.zeros(steps + 1)
    rc = lib().orc_fit(tgp, tg.shape[0], L, T, steps, lr0, lr1, init, loss, eps,
                       ctypes.c_uint64(seed), th.ctypes.data_as(_dp), hist.ctypes.data_as(_dp))
    if rc:
        raise ValueError(f"orc_fit failed ({rc})")
    return th, hist


def dense_sv(img, maps, n_nodes, node_vals, lut) -> np.ndarray:
    """Eq. 1 per pixel with the node kernels blended by Eq. 9 weights."""
    img, ip = _d(img)
    H, W, C = img.shape
    maps, mp = _d(np.reshape(maps, (-1, H, W)))
    nn, nnp = _i(list(n_nodes))
    nv, nvp = _d(node_vals)
    lt, ltp = _d(lut)
    Kd = lt.shape[-1]
    out = np.zeros_like(img)
    rc = lib().orc_dense_sv(ip, H, W, C, mp, len(nn), nnp, nvp, ltp, Kd,
                            out.ctypes.data_as(_dp))
    if rc:
        raise ValueError(f"orc_dense_sv failed ({rc})")
    return out
