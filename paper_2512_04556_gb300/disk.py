"""Thin Python binding of libdisk.so (the C ABI in include/disk.h).

Argument marshalling only: torch tensors are checked (device, dtype, layout)
and their device pointers, pitches and the current stream are handed to the
C entry points of the same names.  Every step of the computation runs in the
library's CUDA kernels.  There is no fallback: if libdisk.so is missing or
fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdisk.so")

DISK_OK = 0
F32, F16 = 0, 1
LOSS_MSE, LOSS_CHARB = 0, 1
INIT_GIVEN, INIT_IR, INIT_SS, INIT_RAND = 0, 1, 2, 3

_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)
_sz = ctypes.c_size_t
_i = ctypes.c_int

_lock = threading.Lock()
_lib = None


class DiskError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed: {code} ({msg})")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded libdisk.so.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libdisk.so not found at {LIB_PATH}: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        l = ctypes.CDLL(LIB_PATH)
        sig = {
            "disk_version": (_i, []),
            "disk_error_string": (ctypes.c_char_p, [_i]),
            "disk_last_error_message": (ctypes.c_char_p, []),
            "disk_basis_from_arrays": (_i, [_i, _ip, _fp, _i, _i, _fp, ctypes.POINTER(_vp)]),
            "disk_basis_load": (_i, [ctypes.c_char_p, ctypes.POINTER(_vp)]),
            "disk_basis_save": (_i, [_vp, ctypes.c_char_p]),
            "disk_basis_info": (_i, [_vp, _ip, _ip, _ip, _ip]),
            "disk_basis_free": (None, [_vp]),
            "disk_sv_filter": (_i, [_vp, _vp, _sz, _vp, _sz, _i, _i, _i, _i, _vp, _vp]),
            "disk_sv_filter_backward_image": (_i, [_vp, _vp, _sz, _vp, _sz, _i, _i, _i, _i, _vp,
                                                   _vp]),
            "disk_sv_filter_backward": (_i, [_vp, _vp, _sz, _vp, _sz, _vp, _sz, _vp, _i, _i, _i, _i,
                                             _vp, _vp]),
            "disk_sv_filter_autotune": (_i, [_vp, _vp, _sz, _vp, _sz, _i, _i, _i, _i, _vp, _ip, _vp]),
            "disk_sv_filter_set_tile": (_i, [_vp, _i, _i, _i, _i, _i]),
            "disk_device_status": (_i, [_vp]),
            "disk_selftest_bounded_wait": (_i, [ctypes.c_longlong, _vp]),
            "disk_sv_filter_frames": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                           ctypes.POINTER(_vp), _i, _i, _i, _i, _i, _vp]),
            "disk_sv_filter_rotated": (_i, [_vp, _vp, _sz, _vp, _sz, _i, _i, _i, _i, _vp, _vp, _vp]),
            "disk_sv_filter_rotated_autotune": (_i, [_vp, _vp, _sz, _vp, _sz, _i, _i, _i, _i, _vp,
                                                     _vp, _ip, _vp]),
            "disk_sv_filter_noalloc": (_i, [_vp, _vp, _sz, _vp, _sz, _i, _i, _i, _i, _vp, _vp]),
            "disk_dense_sv": (_i, [_i, _ip, _fp, _vp, _i, _vp, _sz, _vp, _sz, _i, _i, _i, _i,
                                   _vp, _vp]),
            "disk_synth_kernel": (_i, [_vp, _i, _i, _i, _i, ctypes.c_float, _vp, _vp]),
            "disk_fit": (_i, [_vp, _ip, _i, _i, _i, _i, ctypes.c_float, ctypes.c_float, _i, _i,
                              ctypes.c_float, ctypes.c_uint64, _vp, _vp, _vp, _vp]),
            "disk_fit_resume": (_i, [_vp, _ip, _i, _i, _i, _i, _i, _i, ctypes.c_float,
                                     ctypes.c_float, _i, _i, ctypes.c_float, ctypes.c_uint64,
                                     _vp, _vp, _vp, _vp, _vp]),
            "disk_fit_autotune": (_i, [_vp, _ip, _i, _i, _i, _i, ctypes.c_float, _ip, _vp]),
            "disk_sv_filter_set_layers": (_i, [_vp, _i, _i, _i, _i, _ip]),
            "disk_fit_set_config": (_i, [_i, _i, _i, _i]),
            "disk_mlp_param_count": (ctypes.c_longlong, [_i, _i, _i, _i]),
            "disk_mlp_init": (_i, [_vp, _i, _i, _i, _i, ctypes.c_uint64, _vp]),
            "disk_mlp_forward": (_i, [_vp, _i, _i, _i, _i, _vp, _i, _vp, _vp]),
            "disk_mlp_train_step": (_i, [_vp, _vp, _vp, _i, ctypes.c_float, _i, _i, _i, _i, _vp, _vp,
                                         _i, _vp, _vp]),
            "disk_downsample_targets": (_i, [_vp, _ip, _i, _i, _vp, _vp]),
            "disk_mlp_grad": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _i, _vp, _vp, _vp]),
            "disk_mlp_adam": (_i, [_vp, _vp, _vp, _vp, _i, ctypes.c_float, _i, _i, _i, _i, _vp]),
            "disk_fit_loss_grad": (_i, [_vp, _ip, _i, _i, _i, _i, ctypes.c_float, _vp, _vp, _vp,
                                        _vp]),
            "disk_learned_init": (_i, [_vp, _ip, _i, _i, _i, _vp, _i, _i, _i, _i,
                                       ctypes.c_float, _vp, _vp, _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
        return l


def exported_symbols() -> list[str]:
    return [n for n in dir(lib()) if n.startswith("disk_")]


def _check(fn: str, rc: int):
    if rc != DISK_OK:
        msg = lib().disk_last_error_message().decode(errors="replace")
        raise DiskError(fn, rc, f"{lib().disk_error_string(rc).decode()}: {msg}")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float16:
        return F16
    raise TypeError(f"image dtype must be float32 or float16, got {t.dtype}")


def _image_args(t):
    """(pointer, pitch in bytes, H, W, C) of an H x W x C image whose pixels
    are contiguous within a row."""
    if t.dim() != 3 or not t.is_cuda:
        raise ValueError("image must be a CUDA tensor of shape [H, W, C]")
    H, W, C = t.shape
    if t.stride(2) != 1 or t.stride(1) != C:
        raise ValueError("image rows must be contiguous [W][C]")
    return t.data_ptr(), t.stride(0) * t.element_size(), H, W, C


def _int_arr(v):
    a = (ctypes.c_int * len(v))(*[int(x) for x in v])
    return a


def _float_arr(v):
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float32).ravel())
    return (ctypes.c_float * len(v))(*v.tolist()), v


class Basis:
    """A disk_basis handle (Sec. 4.3 Eq. 8): node values per kernel-space axis
    and theta [B][L][T][3] (dx, dy, w in pixels)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        dims, nn, L, T = _i(), (ctypes.c_int * 2)(), _i(), _i()
        _check("disk_basis_info", lib().disk_basis_info(self._h, ctypes.byref(dims), nn,
                                                        ctypes.byref(L), ctypes.byref(T)))
        self.dims, self.n_nodes, self.L, self.T = dims.value, [nn[0], nn[1]][:dims.value], L.value, T.value

    @classmethod
    def from_arrays(cls, node_vals, theta) -> "Basis":
        """node_vals: one increasing sequence per axis (1 or 2 axes)."""
        if np.ndim(node_vals[0]) == 0:
            node_vals = [node_vals]
        n_nodes = [len(v) for v in node_vals]
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        B = int(np.prod(n_nodes))
        if th.ndim != 4 or th.shape[0] != B or th.shape[3] != 3:
            raise ValueError(f"theta must be [B={B}][L][T][3], got {th.shape}")
        nv, _ = _float_arr(np.concatenate([np.asarray(v, np.float32) for v in node_vals]))
        h = _vp()
        _check("disk_basis_from_arrays", lib().disk_basis_from_arrays(
            len(n_nodes), _int_arr(n_nodes), nv, th.shape[1], th.shape[2],
            th.ctypes.data_as(_fp), ctypes.byref(h)))
        return cls(h)

    @classmethod
    def load(cls, path: str) -> "Basis":
        h = _vp()
        _check("disk_basis_load", lib().disk_basis_load(os.fsencode(path), ctypes.byref(h)))
        return cls(h)

    def save(self, path: str):
        _check("disk_basis_save", lib().disk_basis_save(self._h, os.fsencode(path)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().disk_basis_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sv_filter(basis: Basis, img, maps, out=None, stream=None):
    """Spatially varying DISK filter (Eq. 9 + Eq. 3) of an [H, W, C] CUDA
    image (float32 or float16) with [dims, H, W] float32 maps."""
    import torch
    ip, ipitch, H, W, C = _image_args(img)
    if out is None:
        out = torch.empty_like(img, memory_format=torch.contiguous_format)
    op, opitch, *_ = _image_args(out)
    if out.dtype != img.dtype or tuple(out.shape) != tuple(img.shape):
        raise ValueError("out must match img in shape and dtype")
    if maps.dtype != torch.float32 or not maps.is_cuda or not maps.is_contiguous():
        raise ValueError("maps must be a contiguous float32 CUDA tensor [dims, H, W]")
    if maps.numel() != basis.dims * H * W:
        raise ValueError("maps must hold dims * H * W values")
    _check("disk_sv_filter", lib().disk_sv_filter(
        basis.handle, _vp(ip), ipitch, _vp(op), opitch, H, W, C, _dtype_code(img),
        _vp(maps.data_ptr()), _stream(stream)))
    return out


def sv_filter_set_layers(basis: Basis, img, choice):
    """Record every layer's launch choice for this image shape and dtype: 2 or
    4 pixels per thread, or 8 followed by 0 for a pair of layers fused into
    one launch."""
    _, _, H, W, C = _image_args(img)
    if len(choice) != basis.L:
        raise ValueError(f"choice needs {basis.L} codes")
    _check("disk_sv_filter_set_layers", lib().disk_sv_filter_set_layers(
        basis.handle, H, W, C, _dtype_code(img), _int_arr(list(choice))))


def sv_filter_autotune(basis: Basis, img, maps, out=None, stream=None) -> list:
    """Time the built tile configurations on this frame shape, record the
    fastest of every layer in the basis; returns pixels per thread per layer."""
    import torch
    ip, ipitch, H, W, C = _image_args(img)
    if out is None:
        out = torch.empty_like(img, memory_format=torch.contiguous_format)
    op, opitch, *_ = _image_args(out)
    chosen = (ctypes.c_int * basis.L)()
    _check("disk_sv_filter_autotune", lib().disk_sv_filter_autotune(
        basis.handle, _vp(ip), ipitch, _vp(op), opitch, H, W, C, _dtype_code(img),
        _vp(maps.data_ptr()), chosen, _stream(stream)))
    return list(chosen)


def _angle_arg(angle, H: int, W: int):
    import torch
    if (angle.dtype != torch.float32 or not angle.is_cuda or not angle.is_contiguous()
            or angle.numel() != H * W):
        raise ValueError("angle must be a contiguous float32 CUDA tensor of H x W values")
    return _vp(angle.data_ptr())


def sv_filter_rotated(basis: Basis, img, maps, angle, out=None, stream=None):
    """sv_filter with every pixel's blended tap offsets turned by angle [H, W]
    (float32 radians, x right, y down)."""
    import torch
    ip, ipitch, H, W, C = _image_args(img)
    if out is None:
        out = torch.empty_like(img, memory_format=torch.contiguous_format)
    op, opitch, *_ = _image_args(out)
    _check("disk_sv_filter_rotated", lib().disk_sv_filter_rotated(
        basis.handle, _vp(ip), ipitch, _vp(op), opitch, H, W, C, _dtype_code(img),
        _vp(maps.data_ptr()), _angle_arg(angle, H, W), _stream(stream)))
    return out


def sv_filter_rotated_autotune(basis: Basis, img, maps, angle, out=None, stream=None) -> list:
    """Tile autotuner of sv_filter_rotated; returns pixels per thread per layer."""
    import torch
    ip, ipitch, H, W, C = _image_args(img)
    if out is None:
        out = torch.empty_like(img, memory_format=torch.contiguous_format)
    op, opitch, *_ = _image_args(out)
    chosen = (ctypes.c_int * basis.L)()
    _check("disk_sv_filter_rotated_autotune", lib().disk_sv_filter_rotated_autotune(
        basis.handle, _vp(ip), ipitch, _vp(op), opitch, H, W, C, _dtype_code(img),
        _vp(maps.data_ptr()), _angle_arg(angle, H, W), chosen, _stream(stream)))
    return list(chosen)


def sv_filter_frames(basis: Basis, h_imgs, h_maps, h_outs, stream=None):
    """Filters frames held in host memory (CPU tensors [H, W, C], pinned for
    the copies to overlap the filtering), maps h_maps[i] ([dims, H, W] float32
    CPU), writing h_outs[i].  Asynchronous: synchronise the stream before
    reading h_outs."""
    import torch
    n = len(h_imgs)
    if len(h_maps) != n or len(h_outs) != n:
        raise ValueError("h_imgs, h_maps and h_outs must have the same length")
    if n == 0:
        return h_outs
    H, W, C = h_imgs[0].shape
    dt = h_imgs[0].dtype
    for a, m, o in zip(h_imgs, h_maps, h_outs):
        if (a.device.type != "cpu" or o.device.type != "cpu" or m.device.type != "cpu"
                or not a.is_contiguous() or not o.is_contiguous() or not m.is_contiguous()):
            raise ValueError("frames, maps and outputs must be contiguous CPU tensors")
        if tuple(a.shape) != (H, W, C) or tuple(o.shape) != (H, W, C) or a.dtype != dt or o.dtype != dt:
            raise ValueError("all frames and outputs must share one shape and dtype")
        if m.dtype != torch.float32 or m.numel() != basis.dims * H * W:
            raise ValueError("maps must be float32 [dims, H, W]")
    arr = lambda ts: (_vp * n)(*[t.data_ptr() for t in ts])
    _check("disk_sv_filter_frames", lib().disk_sv_filter_frames(
        basis.handle, arr(h_imgs), arr(h_outs), arr(h_maps), n, H, W, C, _dtype_code(h_imgs[0]),
        _stream(stream)))
    return h_outs


def device_status(stream=None):
    """Raises DiskError (DISK_ERR_TIMEOUT) if a kernel gave up a bounded wait
    since the last call; synchronises the stream."""
    _check("disk_device_status", lib().disk_device_status(_stream(stream)))


def selftest_bounded_wait(iterations: int = 1000, stream=None):
    """Queue a block whose bounded wait runs out (see device_status)."""
    _check("disk_selftest_bounded_wait", lib().disk_selftest_bounded_wait(iterations, _stream(stream)))


def sv_filter_set_tile(basis: Basis, H: int, W: int, C: int, dtype: int, pix: int):
    """Record the tile configuration (2 or 4 pixels per thread) for a frame shape."""
    _check("disk_sv_filter_set_tile", lib().disk_sv_filter_set_tile(basis.handle, H, W, C, dtype, pix))


def sv_filter_backward_image(basis: Basis, grad_out, maps, grad_in=None, stream=None):
    """Gradient of sv_filter with respect to its input image: the transpose of
    the cascade applied to grad_out [H, W, C] (float32 or float16); returns a
    float32 [H, W, C] tensor."""
    import torch
    gp, gpitch, H, W, C = _image_args(grad_out)
    if grad_in is None:
        grad_in = torch.empty((H, W, C), device=grad_out.device, dtype=torch.float32)
    ip, ipitch, *_ = _image_args(grad_in)
    if grad_in.dtype != torch.float32 or tuple(grad_in.shape) != (H, W, C):
        raise ValueError("grad_in must be float32 [H, W, C]")
    if maps.dtype != torch.float32 or not maps.is_cuda or not maps.is_contiguous():
        raise ValueError("maps must be a contiguous float32 CUDA tensor [dims, H, W]")
    _check("disk_sv_filter_backward_image", lib().disk_sv_filter_backward_image(
        basis.handle, _vp(gp), gpitch, _vp(ip), ipitch, H, W, C, _dtype_code(grad_out),
        _vp(maps.data_ptr()), _stream(stream)))
    return grad_in


def sv_filter_backward(basis: Basis, img, grad_out, maps, grad_img: bool = True,
                       grad_theta: bool = True, stream=None):
    """Gradients of <grad_out, sv_filter(img)> with respect to the image
    (float32 [H, W, C]) and the basis theta (float32 [B, L, T, 3]); either may
    be skipped (returned as None).  Activations are recomputed from img."""
    import torch
    ip, ipitch, H, W, C = _image_args(img)
    gp, gpitch, *_ = _image_args(grad_out)
    if grad_out.dtype != img.dtype or tuple(grad_out.shape) != tuple(img.shape):
        raise ValueError("grad_out must match img in shape and dtype")
    if maps.dtype != torch.float32 or not maps.is_cuda or not maps.is_contiguous():
        raise ValueError("maps must be a contiguous float32 CUDA tensor [dims, H, W]")
    gi = torch.empty((H, W, C), device=img.device, dtype=torch.float32) if grad_img else None
    B = int(np.prod(basis.n_nodes))
    gt = torch.empty((B, basis.L, basis.T, 3), device=img.device, dtype=torch.float32) if grad_theta else None
    _check("disk_sv_filter_backward", lib().disk_sv_filter_backward(
        basis.handle, _vp(ip), ipitch, _vp(gp), gpitch,
        _vp(gi.data_ptr()) if gi is not None else None, W * C * 4,
        _vp(gt.data_ptr()) if gt is not None else None, H, W, C, _dtype_code(img),
        _vp(maps.data_ptr()), _stream(stream)))
    return gi, gt


def sv_filter_noalloc(basis: Basis, img, maps, out, stream=None):
    """disk_sv_filter_noalloc: the same filter for callers that cannot
    allocate device memory.  ``out`` must be given (nothing is allocated)."""
    import torch
    ip, ipitch, H, W, C = _image_args(img)
    op, opitch, *_ = _image_args(out)
    if out.dtype != img.dtype or tuple(out.shape) != tuple(img.shape):
        raise ValueError("out must match img in shape and dtype")
    if maps.dtype != torch.float32 or not maps.is_cuda or not maps.is_contiguous():
        raise ValueError("maps must be a contiguous float32 CUDA tensor [dims, H, W]")
    if maps.numel() != basis.dims * H * W:
        raise ValueError("maps must hold dims * H * W values")
    _check("disk_sv_filter_noalloc", lib().disk_sv_filter_noalloc(
        basis.handle, _vp(ip), ipitch, _vp(op), opitch, H, W, C, _dtype_code(img),
        _vp(maps.data_ptr()), _stream(stream)))
    return out


def dense_sv(node_vals, lut, img, maps, out=None, stream=None):
    """Dense spatially varying convolution (Eq. 1 per pixel) with node kernels
    lut [B, Kd, Kd] (float32, CUDA) blended by the Eq. 9 weights."""
    import torch
    if np.ndim(node_vals[0]) == 0:
        node_vals = [node_vals]
    n_nodes = [len(v) for v in node_vals]
    nv, _ = _float_arr(np.concatenate([np.asarray(v, np.float32) for v in node_vals]))
    ip, ipitch, H, W, C = _image_args(img)
    if out is None:
        out = torch.empty_like(img, memory_format=torch.contiguous_format)
    op, opitch, *_ = _image_args(out)
    if lut.dtype != torch.float32 or not lut.is_cuda or not lut.is_contiguous() or lut.dim() != 3:
        raise ValueError("lut must be a contiguous float32 CUDA tensor [B, Kd, Kd]")
    _check("disk_dense_sv", lib().disk_dense_sv(
        len(n_nodes), _int_arr(n_nodes), nv, _vp(lut.data_ptr()), lut.shape[-1],
        _vp(ip), ipitch, _vp(op), opitch, H, W, C, _dtype_code(img),
        _vp(maps.data_ptr()), _stream(stream)))
    return out


def synth_kernel(theta, K: int, max_reach: float | None = None, out=None, stream=None):
    """Impulse responses (Eq. 10) of complexes theta [batch, L, T, 3] (float32
    CUDA, pixels), cropped to K x K."""
    import torch
    if theta.dim() == 3:
        theta = theta[None]
    if theta.dtype != torch.float32 or not theta.is_cuda or not theta.is_contiguous():
        raise ValueError("theta must be a contiguous float32 CUDA tensor [batch, L, T, 3]")
    batch, L, T, _ = theta.shape
    if max_reach is None:
        max_reach = float(theta[..., :2].abs().max().item()) if theta.numel() else 0.0
    if out is None:
        out = torch.empty((batch, K, K), device=theta.device, dtype=torch.float32)
    _check("disk_synth_kernel", lib().disk_synth_kernel(
        _vp(theta.data_ptr()), batch, L, T, K, float(max_reach), _vp(out.data_ptr()),
        _stream(stream)))
    return out


def pack_targets(targets, device="cuda"):
    """Packs square odd-sized targets back to back: (device tensor, sizes)."""
    import torch
    sizes = [int(t.shape[0]) for t in targets]
    flat = np.concatenate([np.asarray(t, np.float32).ravel() for t in targets])
    return torch.from_numpy(flat).to(device), sizes


def fit(packed, sizes, L: int, T: int, steps: int, lr0: float = 1e-3, lr1: float = 1e-4,
        init: int = INIT_IR, loss: int = LOSS_MSE, eps: float = 0.0, seed: int = 0,
        theta=None, loss_hist: bool = False, stream=None):
    """Batched fit (Eq. 4) of complexes [batch, L, T, 3] (pixels) to packed
    targets.  Returns (theta, final loss [batch], history [batch, steps+1] or
    None)."""
    import torch
    batch = len(sizes)
    dev = packed.device
    if theta is None:
        theta = torch.zeros((batch, L, T, 3), device=dev, dtype=torch.float32)
    final = torch.empty(batch, device=dev, dtype=torch.float32)
    hist = torch.empty((batch, steps + 1), device=dev, dtype=torch.float32) if loss_hist else None
    _check("disk_fit", lib().disk_fit(
        _vp(packed.data_ptr()), _int_arr(sizes), batch, L, T, steps, lr0, lr1, init, loss,
        eps, seed, _vp(theta.data_ptr()), _vp(final.data_ptr()),
        _vp(hist.data_ptr()) if hist is not None else None, _stream(stream)))
    return theta, final, hist


def fit_resume(packed, sizes, state, theta, step0: int, steps: int, total_steps: int,
               lr0: float = 1e-3, lr1: float = 1e-4, init: int = INIT_GIVEN,
               loss: int = LOSS_MSE, eps: float = 0.0, seed: int = 0, loss_hist: bool = False,
               stream=None):
    """Steps step0 .. step0+steps-1 of a total_steps-step fit (Eq. 4), the
    optimiser's state carried in `state` [batch, 3, L*T*3] (updated in place;
    built from `init`/`seed`/`theta` when step0 == 0) and the complex in
    `theta` [batch, L, T, 3] (pixels, updated in place).  Returns (final loss
    [batch], history [batch, steps+1] or None)."""
    import torch
    batch, L, T, _ = theta.shape
    if tuple(state.shape) != (batch, 3, L * T * 3) or state.dtype != torch.float32 \
            or not state.is_contiguous():
        raise ValueError(f"state must be contiguous float32 [{batch}, 3, {L * T * 3}]")
    if theta.dtype != torch.float32 or not theta.is_contiguous():
        raise ValueError("theta must be a contiguous float32 tensor [batch, L, T, 3]")
    dev = packed.device
    final = torch.empty(batch, device=dev, dtype=torch.float32)
    hist = torch.empty((batch, steps + 1), device=dev, dtype=torch.float32) if loss_hist else None
    _check("disk_fit_resume", lib().disk_fit_resume(
        _vp(packed.data_ptr()), _int_arr(sizes), batch, L, T, step0, steps, total_steps, lr0, lr1,
        init, loss, eps, seed, _vp(state.data_ptr()), _vp(theta.data_ptr()), _vp(final.data_ptr()),
        _vp(hist.data_ptr()) if hist is not None else None, _stream(stream)))
    return final, hist


def fit_autotune(packed, sizes, L: int, T: int, loss: int = LOSS_MSE, eps: float = 0.0,
                 stream=None) -> tuple:
    """Pick the fit kernel's launch configuration for this batch shape;
    returns (threads per CTA, CTAs per target)."""
    out = ctypes.c_int()
    _check("disk_fit_autotune", lib().disk_fit_autotune(
        _vp(packed.data_ptr()), _int_arr(sizes), len(sizes), L, T, loss, eps,
        ctypes.byref(out), _stream(stream)))
    return out.value // 16, out.value % 16


def fit_set_config(L: int, T: int, kmax: int, threads: int, ctas: int):
    """Record the fit launch configuration (threads per CTA, CTAs per target)
    for batches with this L, T and largest target size."""
    _check("disk_fit_set_config", lib().disk_fit_set_config(L, T, kmax, threads * 16 + ctas))


def fit_loss_grad(packed, sizes, theta, loss: int = LOSS_MSE, eps: float = 0.0, stream=None):
    """Fit objective and its gradient at theta [batch, L, T, 3]."""
    import torch
    batch, L, T, _ = theta.shape
    l = torch.empty(batch, device=theta.device, dtype=torch.float32)
    g = torch.empty_like(theta)
    _check("disk_fit_loss_grad", lib().disk_fit_loss_grad(
        _vp(packed.data_ptr()), _int_arr(sizes), batch, L, T, loss, eps,
        _vp(theta.data_ptr()), _vp(l.data_ptr()), _vp(g.data_ptr()), _stream(stream)))
    return l, g


class MLP:
    """The learned initializer's network: parameters and Adam moments on the
    device; shape (n_in, hidden, depth, n_out)."""

    def __init__(self, n_in: int, hidden: int, depth: int, n_out: int, seed: int = 0,
                 device="cuda"):
        import torch
        self.shape = (n_in, hidden, depth, n_out)
        n = lib().disk_mlp_param_count(*self.shape)
        if n < 0:
            raise ValueError(f"bad MLP shape {self.shape}")
        self.params = torch.empty(n, device=device, dtype=torch.float32)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._loss = torch.zeros(1, device=device, dtype=torch.float32)
        _check("disk_mlp_init", lib().disk_mlp_init(_vp(self.params.data_ptr()), *self.shape,
                                                    seed, _stream(None)))

    def forward(self, x, stream=None):
        import torch
        y = torch.empty((x.shape[0], self.shape[3]), device=x.device, dtype=torch.float32)
        _check("disk_mlp_forward", lib().disk_mlp_forward(
            _vp(self.params.data_ptr()), *self.shape, _vp(x.data_ptr()), x.shape[0],
            _vp(y.data_ptr()), _stream(stream)))
        return y

    def grad(self, x, target, stream=None):
        """(loss, gradient) of the batch without updating; both device tensors."""
        import torch
        g = torch.empty_like(self.params)
        loss = torch.zeros(1, device=self.params.device, dtype=torch.float32)
        _check("disk_mlp_grad", lib().disk_mlp_grad(
            _vp(self.params.data_ptr()), *self.shape, _vp(x.data_ptr()), _vp(target.data_ptr()),
            x.shape[0], _vp(g.data_ptr()), _vp(loss.data_ptr()), _stream(stream)))
        return loss, g

    def apply(self, grad, lr: float, stream=None):
        """One Adam step with a given gradient (e.g. averaged over ranks)."""
        self.step += 1
        _check("disk_mlp_adam", lib().disk_mlp_adam(
            _vp(self.params.data_ptr()), _vp(self.m.data_ptr()), _vp(self.v.data_ptr()),
            _vp(grad.data_ptr()), self.step, lr, *self.shape, _stream(stream)))

    def save(self, path: str):
        """Writes the parameters, both Adam moments and the step count to a
        checkpoint file; `MLP.load` continues training from it exactly."""
        from . import checkpoint
        checkpoint.save_mlp(path, shape=self.shape, step=self.step, params=self.params,
                            m=self.m, v=self.v)

    @classmethod
    def load(cls, path: str, device="cuda") -> "MLP":
        """The network (and optimiser state) of a checkpoint file."""
        import torch

        from . import checkpoint
        shape, step, p, m, v = checkpoint.load_mlp(path)
        net = cls(*shape, device=device)
        if p.size != net.params.numel():
            raise checkpoint.CheckpointError(
                f"{path}: {p.size} parameters, shape {shape} has {net.params.numel()}")
        for name, a in (("params", p), ("m", m), ("v", v)):
            getattr(net, name).copy_(torch.from_numpy(a))
        net.step = step
        return net

    def train_step(self, x, target, lr: float, stream=None):
        """One Adam step on the batch; returns the loss as a device tensor."""
        self.step += 1
        _check("disk_mlp_train_step", lib().disk_mlp_train_step(
            _vp(self.params.data_ptr()), _vp(self.m.data_ptr()), _vp(self.v.data_ptr()),
            self.step, lr, *self.shape, _vp(x.data_ptr()), _vp(target.data_ptr()), x.shape[0],
            _vp(self._loss.data_ptr()), _stream(stream)))
        return self._loss


def downsample_targets(packed, sizes, side: int = 64, stream=None):
    """Area-resampled targets [batch, side, side], each scaled to max 1."""
    import torch
    out = torch.empty((len(sizes), side, side), device=packed.device, dtype=torch.float32)
    _check("disk_downsample_targets", lib().disk_downsample_targets(
        _vp(packed.data_ptr()), _int_arr(sizes), len(sizes), side, _vp(out.data_ptr()),
        _stream(stream)))
    return out


def learned_init(net: "MLP", packed, sizes, L: int, T: int, side: int = 64,
                 loss: int = LOSS_MSE, eps: float = 0.0, stream=None):
    """disk_learned_init: the network's start for each target (pixels), or the
    Eq. 6 start where that has the lower fitted loss.  Returns
    (theta [batch, L, T, 3], used_network [batch] bool), both on the device."""
    import torch
    n_in, hidden, depth, n_out = net.shape
    if n_in != side * side or n_out != L * T * 3:
        raise ValueError(f"network shape {net.shape} does not fit side={side}, L={L}, T={T}")
    theta = torch.empty((len(sizes), L, T, 3), device=packed.device, dtype=torch.float32)
    used = torch.empty(len(sizes), device=packed.device, dtype=torch.int32)
    _check("disk_learned_init", lib().disk_learned_init(
        _vp(packed.data_ptr()), _int_arr(sizes), len(sizes), L, T, _vp(net.params.data_ptr()),
        side, hidden, depth, loss, eps, _vp(theta.data_ptr()), _vp(used.data_ptr()),
        _stream(stream)))
    return theta, used.bool()
