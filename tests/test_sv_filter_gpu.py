"""GPU parity of the spatially varying filter, the dense baseline and impulse
synthesis against the FP64 oracle, through the C ABI.

Gates (normwise: max |gpu - oracle| / max |oracle| over the compared
outputs): 1e-5 for FP32 storage; 2e-3 for FP16 storage, where the oracle runs
on the FP16 input widened exactly and its output is rounded to FP16.
"""
import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL32, TOL16 = 1e-5, 2e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2512_04556_gb300 import disk
    disk.lib()
    return torch


def rel_err(got, want):
    return float(np.abs(got.astype(np.float64) - want).max() / max(np.abs(want).max(), 1e-30))


def gpu_filter(torch, img, maps, axes, theta, out_dtype=None):
    from paper_2512_04556_gb300 import disk
    b = disk.Basis.from_arrays(axes, theta)
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    m = torch.from_numpy(np.ascontiguousarray(maps, dtype=np.float32)).cuda()
    out = disk.sv_filter(b, t, m)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_filter(img, maps, axes, theta):
    n_nodes = [len(a) for a in axes]
    nv = np.concatenate([np.asarray(a, np.float64) for a in axes])
    return oracle.sv_filter(img.astype(np.float64), np.asarray(maps, np.float64), n_nodes, nv,
                            np.asarray(theta, np.float64))


def check(torch, img, maps, axes, theta, tol=None):
    got = gpu_filter(torch, img, maps, axes, theta)
    want = oracle_filter(img, maps, axes, theta)
    if img.dtype == np.float16:
        want = want.astype(np.float16).astype(np.float64)
        tol = tol or TOL16
    err = rel_err(got, want)
    assert err <= (tol or TOL32), f"max rel err {err:.3e}"
    return got


def _basis_1d(L, T, spread, seed, nodes=(1.0, 2.0, 4.0, 8.0)):
    return [list(nodes)], wl.basis_random(list(nodes), L, T, spread, seed)


def _maps(H, W, lo, hi, seed, dims=1):
    g = np.random.default_rng(seed)
    if dims == 1:
        return wl.param_map(H, W, lo, hi, 8.0, seed)[None]
    return np.stack([wl.param_map(H, W, lo, hi, 8.0, seed), g.uniform(0, 1, (H, W)).astype(np.float32)])


def test_c1_full_size_fp32(torch_cuda):
    """The 256 x 256 workload: random 4-node basis, L=3, T=8, offsets up to 3s."""
    img, maps, n_nodes, nodes, theta = wl.c1_inputs()
    check(torch_cuda, img, maps, [list(nodes)], theta)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (33, 1), (31, 33), (67, 53), (100, 129)])
def test_ragged_sizes(torch_cuda, H, W):
    axes, th = _basis_1d(3, 5, 1.5, H * 1000 + W)
    img = wl.image_uniform(H, W, 3, seed=H + W)
    check(torch_cuda, img, _maps(H, W, 0.5, 9.0, W), axes, th)


@pytest.mark.parametrize("H,W,dtype", [(1, 32768, "f32"), (32768, 1, "f32"), (3, 32768, "f16"),
                                        (32768, 2, "f16")])
def test_maximum_image_sides(torch_cuda, H, W, dtype):
    """Images at the 32768-pixel limit on either side (grid limits, index
    arithmetic, the tile copy's tensor map) against the oracle."""
    axes, th = _basis_1d(2, 5, 1.5, 91)
    img = wl.image_uniform(H, W, 3, seed=92)
    if dtype == "f16":
        img = wl.to_fp16(img)
    check(torch_cuda, img, _maps(H, W, 1.0, 8.0, 93), axes, th)


def test_rejects_sides_beyond_limit(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    axes, th = _basis_1d(2, 3, 1.0, 94)
    b = disk.Basis.from_arrays(axes, th)
    t = torch.zeros((1, 32769, 3), device="cuda")
    m = torch.zeros((1, 1, 32769), device="cuda")
    with pytest.raises(disk.DiskError) as e:
        disk.sv_filter(b, t, m)
    assert e.value.code == -1


def test_fp16_storage(torch_cuda):
    axes, th = _basis_1d(4, 8, 1.2, 3)
    img = wl.to_fp16(wl.image_rects(70, 91, seed=4))
    check(torch_cuda, img, _maps(70, 91, 1.0, 8.0, 5), axes, th)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_2d_basis(torch_cuda, dtype):
    n0, n1 = 4, 3
    axes = [list(np.linspace(2.0, 8.0, n0)), list(np.linspace(0.0, 1.0, n1))]
    th = wl.basis_random(np.repeat(np.linspace(0.5, 1.5, n0), n1), 3, 6, 2.0, seed=6)
    img = wl.image_uniform(45, 77, 3, seed=7)
    if dtype == "f16":
        img = wl.to_fp16(img)
    check(torch_cuda, img, _maps(45, 77, 1.0, 9.0, 8, dims=2), axes, th)


@pytest.mark.parametrize("C", [3, 4])
@pytest.mark.parametrize("smooth", [True, False])
def test_2d_large_table_odd_taps(torch_cuda, C, smooth):
    """A 10 x 10 basis with T = 7 (the node-tap table exceeds 8 KB, so blocks
    copy only their node range, or read the table from global memory when the
    range is too wide): taps taken in pairs plus the odd last tap for three
    channels, one at a time for four; smooth maps (one cell per thread) and
    per-pixel noise on the second axis (cells differ within threads)."""
    n0 = n1 = 10
    axes = [list(np.linspace(2.0, 8.0, n0)), list(np.linspace(0.0, 1.0, n1))]
    th = wl.basis_random(np.repeat(np.linspace(0.5, 1.5, n0), n1), 2, 7, 2.0, seed=81)
    H, W = 70, 90
    img = wl.image_uniform(H, W, C, seed=82)
    m0 = wl.param_map(H, W, 1.0, 9.0, 8.0, 83)
    m1 = (wl.param_map(H, W, 0.0, 1.0, 8.0, 84) if smooth
          else np.random.default_rng(85).uniform(0, 1, (H, W)).astype(np.float32))
    check(torch_cuda, img, np.stack([m0, m1]), axes, th)


def test_edge_offsets_integer_and_half(torch_cuda):
    """Exact integer and +-1/2 offsets (the floor/fraction split's edge cases)."""
    th = np.zeros((2, 2, 4, 3), np.float32)
    th[0, 0] = [[1, 0, 0.25], [-2, 3, 0.25], [0.5, -0.5, 0.25], [-0.5, 0.5, 0.25]]
    th[0, 1] = [[0, 0, 1.0], [4, -4, 0.0], [0.5, 0.5, 0.0], [-1, -1, 0.0]]
    th[1] = th[0]
    th[1, 1, 0] = [-3.0, 2.0, 1.0]
    img = wl.image_uniform(40, 41, 3, seed=9)
    maps = np.zeros((1, 40, 41), np.float32)
    maps[0, :, 20:] = 1.0
    maps[0, 10:20, :] = 0.5
    check(torch_cuda, img, maps, [[0.0, 1.0]], th)


def test_single_layer_single_tap(torch_cuda):
    th = np.array([[[[0.25, -0.75, 1.0]]]], np.float32)
    img = wl.image_uniform(19, 23, 3, seed=10)
    check(torch_cuda, img, np.zeros((1, 19, 23), np.float32), [[0.0]], th)


def test_four_channels_and_pitch(torch_cuda):
    """C = 4 (alpha filtered like colour) on a row-pitched view."""
    import torch
    from paper_2512_04556_gb300 import disk
    axes, th = _basis_1d(3, 4, 1.0, 11)
    full = wl.image_uniform(37, 60, 4, seed=12)
    img = full[:, :45]                                   # pitch 60 px, width 45
    maps = _maps(37, 45, 1.0, 8.0, 13)
    b = disk.Basis.from_arrays(axes, th)
    t = torch.from_numpy(full).cuda()[:, :45]
    out = disk.sv_filter(b, t, torch.from_numpy(maps).cuda())
    torch.cuda.synchronize()
    want = oracle_filter(np.ascontiguousarray(img), maps, axes, th)
    assert rel_err(out.cpu().numpy(), want) <= TOL32


def test_maps_out_of_range_and_nonfinite(torch_cuda):
    """Values beyond the node range clamp to the end nodes; NaN acts as the
    first node, +inf as the last."""
    axes, th = _basis_1d(3, 5, 1.0, 14)
    img = wl.image_uniform(24, 30, 3, seed=15)
    maps = _maps(24, 30, -5.0, 20.0, 16)
    maps[0, 3, 4] = np.nan
    maps[0, 5, 6] = np.inf
    maps[0, 7, 8] = -np.inf
    got = gpu_filter(torch_cuda, img, maps, axes, th)
    ref_maps = maps.copy()
    ref_maps[0, 3, 4] = axes[0][0]
    ref_maps[0, 5, 6] = axes[0][-1]
    ref_maps[0, 7, 8] = axes[0][0]
    assert rel_err(got, oracle_filter(img, ref_maps, axes, th)) <= TOL32
    assert np.isfinite(got).all()


def test_maximum_reach(torch_cuda):
    """Taps at the largest supported reach (40 px) on an image smaller than the halo."""
    th = wl.basis_random([1.0, 2.0], 2, 6, 20.0, seed=17)
    th[..., :2] = np.clip(th[..., :2], -40, 40)
    th[0, 0, 0, :2] = [40.0, -40.0]
    img = wl.image_uniform(50, 70, 3, seed=18)
    check(torch_cuda, img, _maps(50, 70, 1.0, 2.0, 19), [[1.0, 2.0]], th)


def test_deterministic(torch_cuda):
    img, maps, n_nodes, nodes, theta = wl.c1_inputs(96, 80)
    a = gpu_filter(torch_cuda, img, maps, [list(nodes)], theta)
    b = gpu_filter(torch_cuda, img, maps, [list(nodes)], theta)
    assert np.array_equal(a, b)


def test_rejects_reach_beyond_limit(torch_cuda):
    from paper_2512_04556_gb300 import disk
    th = np.zeros((1, 1, 1, 3), np.float32)
    th[0, 0, 0] = [41.0, 0.0, 1.0]
    with pytest.raises(disk.DiskError) as e:
        disk.Basis.from_arrays([[0.0]], th)
    assert e.value.code == -3


# --------------------------------------------------------------- dense baseline

@pytest.mark.parametrize("dims,dtype", [(1, "f32"), (1, "f16"), (2, "f32")])
def test_dense_sv_parity(torch_cuda, dims, dtype):
    import torch
    from paper_2512_04556_gb300 import disk
    H, W, Kd = 41, 67, 13
    if dims == 1:
        axes = [[1.0, 2.5, 4.0, 6.0]]
        lut = wl.disk_lut(axes[0], Kd)
    else:
        axes = [[2.0, 4.0, 6.0], [0.0, 0.5, 1.0]]
        lut = wl.ellipse_lut(axes[0], axes[1], Kd)
    img = wl.image_rects(H, W, seed=20)
    if dtype == "f16":
        img = wl.to_fp16(img)
    maps = _maps(H, W, 0.5, 7.0, 21, dims)
    out = disk.dense_sv(axes, torch.from_numpy(lut).cuda(), torch.from_numpy(img).cuda(),
                        torch.from_numpy(maps).cuda())
    torch.cuda.synchronize()
    n_nodes = [len(a) for a in axes]
    want = oracle.dense_sv(img.astype(np.float64), maps.astype(np.float64), n_nodes,
                           np.concatenate(axes), lut.astype(np.float64))
    tol = TOL32
    if dtype == "f16":
        want = want.astype(np.float16).astype(np.float64)
        tol = TOL16
    assert rel_err(out.cpu().numpy(), want) <= tol


# --------------------------------------------------------------- synthesis

@pytest.mark.parametrize("K", [1, 7, 21, 45])
def test_synth_parity(torch_cuda, K):
    import torch
    from paper_2512_04556_gb300 import disk
    ths = np.stack([wl.complex_random(3, 5, 4.0, s) for s in range(6)]).astype(np.float32)
    out = disk.synth_kernel(torch.from_numpy(ths).cuda(), K, max_reach=4.0)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for b in range(len(ths)):
        want = oracle.synth(ths[b].astype(np.float64), K)
        assert np.abs(got[b] - want).max() <= TOL32 * max(np.abs(want).max(), 1e-3)


def test_synth_flags_taps_beyond_declared_reach(torch_cuda):
    import torch
    from paper_2512_04556_gb300 import disk
    th = wl.complex_random(2, 3, 2.0, 3).astype(np.float32)[None].repeat(2, 0)
    th[1, 0, 0, 0] = 5.0
    out = disk.synth_kernel(torch.from_numpy(th).cuda(), 9, max_reach=2.0).cpu().numpy()
    assert np.isfinite(out[0]).all() and np.isnan(out[1]).all()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_tile_configurations_and_autotune(torch_cuda, dtype):
    """Both tile configurations match the oracle and each other bit for bit;
    the autotuner picks a tile per layer or a fused layer pair (code 8 then
    0), with the same output."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    n0, n1 = 3, 3
    axes = [list(np.linspace(2.0, 8.0, n0)), list(np.linspace(0.0, 1.0, n1))]
    th = wl.basis_random(np.repeat(np.linspace(0.5, 1.5, n0), n1), 3, 6, 3.0, seed=70)
    H, W = 83, 97
    img = wl.image_uniform(H, W, 3, seed=71)
    if dtype == "f16":
        img = wl.to_fp16(img)
    maps = _maps(H, W, 1.0, 9.0, 72, dims=2)
    b = disk.Basis.from_arrays(axes, th)
    t = torch.from_numpy(img).cuda()
    m = torch.from_numpy(maps).cuda()
    outs = {}
    for pix in (2, 4):
        disk.sv_filter_set_tile(b, H, W, 3, 0 if dtype == "f32" else 1, pix)
        outs[pix] = disk.sv_filter(b, t, m).cpu().numpy()
    assert np.array_equal(outs[2], outs[4])
    want = oracle_filter(img, maps, axes, th)
    if dtype == "f16":
        want = want.astype(np.float16).astype(np.float64)
    assert rel_err(outs[2], want) <= (TOL32 if dtype == "f32" else TOL16)
    chosen = disk.sv_filter_autotune(b, t, m)
    assert len(chosen) == 3 and set(chosen) <= {2, 4, 8, 0}
    for l, c in enumerate(chosen):
        if c == 8:
            assert chosen[l + 1] == 0
        if c == 0:
            assert l > 0 and chosen[l - 1] == 8
    assert np.array_equal(disk.sv_filter(b, t, m).cpu().numpy(), outs[2])
