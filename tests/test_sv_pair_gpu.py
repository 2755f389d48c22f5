"""GPU parity of the fused layer pair (two adjacent layers of the cascade in
one launch, the intermediate kept in shared memory) through the C ABI.

Every pixel of a fused pair runs the same FP32 arithmetic as the
single-layer launches, so the output must equal the unfused filter bit for
bit, and match the FP64 oracle within the parity gates (1e-5 FP32, 2e-3 FP16
storage).  Cases: pairs starting at the first layer (the caller's image
staged through registers) and later (an FP32 intermediate copied by the
tensor-memory accelerator), 1-D and 2-D bases, three and four channels,
images smaller than a tile, ragged edges, and the 4K workload.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32, TOL16 = 1e-5, 2e-3
BASES = os.path.join(os.path.dirname(__file__), "golden", "bases")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2512_04556_gb300 import disk
    disk.lib()
    return torch


def _case(H, W, C, dims, L, T, seed, spread=1.2):
    g = np.random.default_rng(seed)
    if dims == 1:
        axes = [[1.0, 2.0, 4.0, 8.0]]
        th = wl.basis_random(axes[0], L, T, spread, seed)
        maps = wl.param_map(H, W, 0.5, 9.0, 6.0, seed)[None]
    else:
        axes = [list(np.linspace(1.0, 3.0, 3)), list(np.linspace(0.0, 1.0, 4))]
        th = wl.basis_random(np.repeat(np.linspace(1, 3, 3), 4), L, T, spread, seed)
        maps = np.stack([wl.param_map(H, W, 0.8, 3.2, 6.0, seed),
                         g.uniform(-0.1, 1.1, (H, W)).astype(np.float32)])
    img = wl.image_uniform(H, W, C, seed=seed + 1)
    return axes, th.astype(np.float32), maps.astype(np.float32), img


def _filter(torch, axes, th, maps, img, choice):
    from paper_2512_04556_gb300 import disk
    b = disk.Basis.from_arrays(axes, th)
    d_img = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    d_maps = torch.from_numpy(maps).cuda()
    disk.sv_filter_set_layers(b, d_img, choice)
    out = disk.sv_filter(b, d_img, d_maps)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle(axes, th, maps, img):
    want = oracle.sv_filter(img.astype(np.float64), maps.astype(np.float64), [len(a) for a in axes],
                            np.concatenate(axes).astype(np.float64), th.astype(np.float64))
    if img.dtype == np.float16:
        return want.astype(np.float16).astype(np.float64), TOL16
    return want, TOL32


def _rel(a, b):
    return float(np.abs(a.astype(np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("H,W,C,dims,dtype,L,choice", [
    (200, 176, 3, 1, "f32", 4, (8, 0, 8, 0)),
    (67, 53, 4, 2, "f16", 3, (2, 8, 0)),
    (67, 53, 3, 2, "f32", 3, (8, 0, 4)),
    (5, 7, 3, 1, "f32", 3, (8, 0, 2)),
    (1, 40, 3, 2, "f16", 2, (8, 0)),
    (45, 1, 4, 1, "f32", 3, (2, 8, 0)),
    (33, 97, 3, 1, "f16", 5, (4, 8, 0, 8, 0)),
])
def test_fused_pair_equals_single_layers_and_oracle(torch_cuda, H, W, C, dims, dtype, L, choice):
    axes, th, maps, img = _case(H, W, C, dims, L, 7 if dims == 2 else 5, H * 100 + W + L)
    if dtype == "f16":
        img = wl.to_fp16(img)
    fused = _filter(torch_cuda, axes, th, maps, img, choice)
    single = _filter(torch_cuda, axes, th, maps, img, [2] * L)
    np.testing.assert_array_equal(fused, single)
    want, tol = _oracle(axes, th, maps, img)
    assert _rel(fused, want) <= tol


def test_fused_pair_rejects_malformed_choices(torch_cuda):
    from paper_2512_04556_gb300 import disk
    axes, th, maps, img = _case(16, 16, 3, 1, 3, 4, 1)
    b = disk.Basis.from_arrays(axes, th)
    d_img = torch_cuda.from_numpy(img).cuda()
    for bad in ([8, 2, 2], [2, 2, 8], [3, 2, 2], [0, 2, 2]):
        with pytest.raises(disk.DiskError):
            disk.sv_filter_set_layers(b, d_img, bad)


def test_fused_pairs_on_the_4k_workload(torch_cuda):
    """The 3840 x 2160 FP16 frame with the 8 x 8 ellipse basis: every cover by
    fused pairs equals the single-layer filter bit for bit, and the autotuner
    returns a valid cover."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    H, W = wl.C4["H"], wl.C4["W"]
    img = wl.to_fp16(wl.image_rects(H, W, 3))
    m0 = wl.param_map(H, W, *wl.C4["map_range0"], sigma=wl.C4["map_sigma"], stream=0)
    m1 = wl.param_map(H, W, *wl.C4["map_range1"], sigma=wl.C4["map_sigma"], stream=1)
    b = disk.Basis.load(os.path.join(BASES, "ellipse8x8_L4T24.dkb"))
    d_img = torch.from_numpy(img).cuda()
    d_maps = torch.from_numpy(np.stack([m0, m1])).cuda()
    disk.sv_filter_set_layers(b, d_img, [2, 2, 2, 2])
    ref = disk.sv_filter(b, d_img, d_maps)
    for choice in ([8, 0, 2, 2], [2, 8, 0, 2], [8, 0, 8, 0]):
        try:
            disk.sv_filter_set_layers(b, d_img, choice)
        except disk.DiskError:
            continue  # a pair whose halos do not fit shared memory
        out = disk.sv_filter(b, d_img, d_maps)
        assert torch.equal(out, ref), choice
    chosen = disk.sv_filter_autotune(b, d_img, d_maps)
    l = 0
    while l < b.L:
        assert chosen[l] in (2, 4, 8)
        if chosen[l] == 8:
            assert chosen[l + 1] == 0
            l += 1
        l += 1
    torch.cuda.synchronize()
