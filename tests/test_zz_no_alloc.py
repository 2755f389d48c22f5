"""disk_sv_filter_noalloc against disk_sv_filter, through the C ABI.

The allocation-free entry point serves callers that may not allocate device
memory (its intermediate layers live in a fixed array inside the library).
It must give the allocating entry point's results within the parity
tolerance, on two calls in a row with different inputs (the second call
must not see the first call's leftovers), and must refuse images larger than
its array before queueing any work.  This file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32, TOL16 = 1e-5, 2e-3


def _rel(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def test_noalloc_matches_allocating_entry_point_two_calls():
    import torch
    from paper_2512_04556_gb300 import disk
    assert torch.cuda.is_available()
    img, maps, n_nodes, nodes, theta = wl.c1_inputs(200, 176)
    basis = disk.Basis.from_arrays(nodes, theta)
    d_maps = torch.from_numpy(maps).cuda()
    cases = [img, wl.to_fp16(wl.image_rects(200, 176, seed=5))]
    for a in cases:
        d_img = torch.from_numpy(a).cuda()
        ref = disk.sv_filter(basis, d_img, d_maps)
        out = torch.full_like(d_img, float("nan"))
        disk.sv_filter_noalloc(basis, d_img, d_maps, out)
        torch.cuda.synchronize()
        tol = TOL32 if a.dtype == np.float32 else TOL16
        assert np.isfinite(out.cpu().numpy().astype(np.float64)).all()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= tol


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
