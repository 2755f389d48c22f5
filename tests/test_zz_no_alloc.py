"""disk_sv_filter_noalloc against disk_sv_filter and the oracle, through the C ABI.

The allocation-free entry point serves callers that may not allocate device
memory: a plug-in whose host application owns the device-memory budget, or a
real-time loop that allocates nothing after start-up.  Its intermediate
layers live in a fixed array inside the library, and it runs the allocating
entry point's own code path on that array, so the two must agree bit for bit
(FP32 and FP16 storage, three and four channels, a four-layer basis), and
both must match the FP64 oracle within the parity tolerance.  Two calls in a
row with different inputs must not see each other's leftovers, an image
that fills the array to its last byte must still be exact, and images larger
than the array are refused before any work is queued.  This file sorts last
so that a run that stops at the first failure has already run every other
test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32, TOL16 = 1e-5, 2e-3
NODES = [1.0, 2.0, 4.0, 8.0]


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def _case(H, W, C, dtype, seed, L=4, T=8, scale=1.0):
    img = wl.image_uniform(H, W, C, seed=seed) * scale
    img = wl.to_fp16(img) if dtype == np.float16 else img.astype(np.float32)
    maps = wl.param_map(H, W, 1.0, 8.0, sigma=16.0, seed=seed + 1)[None]
    theta = wl.basis_random(NODES, L, T, 1.5, seed=seed + 2)
    return img, maps, theta


def _both(img, maps, theta):
    """(disk_sv_filter, disk_sv_filter_noalloc) outputs on the same inputs."""
    import torch
    from paper_2512_04556_gb300 import disk
    basis = disk.Basis.from_arrays(NODES, theta)
    d_img = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    d_maps = torch.from_numpy(np.ascontiguousarray(maps, np.float32)).cuda()
    ref = disk.sv_filter(basis, d_img, d_maps)
    out = torch.full_like(d_img, float("nan"))
    disk.sv_filter_noalloc(basis, d_img, d_maps, out)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


def _oracle(img, maps, theta):
    want = oracle.sv_filter(img.astype(np.float64), np.asarray(maps, np.float64), [len(NODES)],
                            np.asarray(NODES, np.float64), np.asarray(theta, np.float64))
    if img.dtype == np.float16:
        return want.astype(np.float16).astype(np.float64), TOL16
    return want, TOL32


@pytest.mark.parametrize("C", [3, 4])
@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_noalloc_equals_allocating_entry_point_and_oracle(dtype, C):
    import torch
    assert torch.cuda.is_available()
    img, maps, theta = _case(200, 176, C, dtype, seed=40 + C)
    ref, out = _both(img, maps, theta)
    np.testing.assert_array_equal(out, ref)
    want, tol = _oracle(img, maps, theta)
    assert _rel(out, want) <= tol


def test_noalloc_two_calls_in_a_row_do_not_share_leftovers():
    """The first call fills the array with large values; the second, on a
    different image of the same shape and type, must still be exact."""
    loud, maps, theta = _case(240, 200, 3, np.float32, seed=50, scale=1e4)
    quiet, _, _ = _case(240, 200, 3, np.float32, seed=51)
    ref0, out0 = _both(loud, maps, theta)
    np.testing.assert_array_equal(out0, ref0)
    ref1, out1 = _both(quiet, maps, theta)
    np.testing.assert_array_equal(out1, ref1)
    want, tol = _oracle(quiet, maps, theta)
    assert _rel(out1, want) <= tol


def test_noalloc_at_the_size_limit():
    """1024 x 1024 x 4 FP32 with three intermediate-producing layers: each
    plane is exactly half the array, so the second ends on its last byte.
    Compared with disk_sv_filter everywhere and with the oracle on sampled
    rows (the top, the bottom and one through the middle)."""
    img, maps, theta = _case(1024, 1024, 4, np.float32, seed=60, L=4, T=6)
    ref, out = _both(img, maps, theta)
    np.testing.assert_array_equal(out, ref)
    full = oracle.sv_filter(img[:64].astype(np.float64), np.asarray(maps[:, :64], np.float64),
                            [len(NODES)], np.asarray(NODES, np.float64),
                            np.asarray(theta, np.float64))
    # rows far enough from a crop's cut edge are exact on the crop: the
    # cascade reads at most sum_l (ceil(reach_l) + 1) rows away
    reach = int(sum(np.ceil(np.abs(theta[..., l, :, :2]).max()) + 1 for l in range(4)))
    assert reach < 64
    assert _rel(out[:2], full[:2]) <= TOL32
    lo = 511 - reach - 2
    mid = oracle.sv_filter(img[lo:lo + 2 * reach + 5].astype(np.float64),
                           np.asarray(maps[:, lo:lo + 2 * reach + 5], np.float64),
                           [len(NODES)], np.asarray(NODES, np.float64),
                           np.asarray(theta, np.float64))
    assert _rel(out[511], mid[511 - lo]) <= TOL32
    bot = oracle.sv_filter(img[-64:].astype(np.float64), np.asarray(maps[:, -64:], np.float64),
                           [len(NODES)], np.asarray(NODES, np.float64),
                           np.asarray(theta, np.float64))
    assert _rel(out[-2:], bot[-2:]) <= TOL32


def test_noalloc_rejects_images_beyond_its_array():
    import torch
    from paper_2512_04556_gb300 import disk
    img, maps, n_nodes, nodes, theta = wl.c1_inputs(16, 16)
    basis = disk.Basis.from_arrays(nodes, theta)
    d_img = torch.zeros((1025, 1024, 3), device="cuda")
    d_out = torch.zeros_like(d_img)
    d_maps = torch.zeros((1, 1025, 1024), device="cuda")
    rc = disk.lib().disk_sv_filter_noalloc(
        basis.handle, ctypes.c_void_p(d_img.data_ptr()), 1024 * 12,
        ctypes.c_void_p(d_out.data_ptr()), 1024 * 12, 1025, 1024, 3, 0,
        ctypes.c_void_p(d_maps.data_ptr()), None)
    assert rc == -3
    assert b"1048576" in disk.lib().disk_last_error_message()
