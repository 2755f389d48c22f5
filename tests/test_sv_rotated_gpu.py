"""GPU parity of the rotated spatially varying filter (every pixel's blended
tap offsets turned by a per-pixel angle) against the FP64 oracle, through the
C ABI.  Gates as the plain filter: 1e-5 normwise for FP32 storage, 2e-3 for
FP16 storage (oracle on the FP16 input, its output rounded to FP16)."""
import math

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


def _case(H, W, dims, L, T, spread, seed, C=3, fp16=False):
    g = np.random.default_rng(seed)
    img = wl.image_uniform(H, W, C, seed=seed)
    if fp16:
        img = wl.to_fp16(img)
    if dims == 1:
        axes = [[1.0, 2.0, 4.0, 8.0]]
        maps = wl.param_map(H, W, 0.5, 9.0, 8.0, seed)[None]
    else:
        axes = [[1.0, 3.0, 6.0], [0.0, 0.5, 1.0]]
        maps = np.stack([wl.param_map(H, W, 0.5, 7.0, 8.0, seed),
                         g.uniform(0, 1, (H, W)).astype(np.float32)])
    B = int(np.prod([len(a) for a in axes]))
    th = wl.basis_random([1.0] * B, L, T, spread, seed + 1)
    angle = g.uniform(-math.pi, math.pi, (H, W)).astype(np.float32)
    return img, maps, axes, th, angle


def _gpu(torch, img, maps, axes, th, angle, tune=False):
    from paper_2512_04556_gb300 import disk
    b = disk.Basis.from_arrays(axes, th)
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    m = torch.from_numpy(np.ascontiguousarray(maps, dtype=np.float32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(angle, dtype=np.float32)).cuda()
    if tune:
        disk.sv_filter_rotated_autotune(b, t, m, a)
    out = disk.sv_filter_rotated(b, t, m, a)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle(img, maps, axes, th, angle):
    nn = [len(a) for a in axes]
    nv = np.concatenate([np.asarray(a, np.float64) for a in axes])
    return oracle.sv_filter_rotated(img.astype(np.float64), np.asarray(maps, np.float64),
                                    angle.astype(np.float64), nn, nv, th.astype(np.float64))


@pytest.mark.parametrize("dims", [1, 2])
@pytest.mark.parametrize("C", [3, 4])
@pytest.mark.parametrize("H,W", [(1, 1), (37, 29), (70, 133)])
def test_rotated_fp32(torch_cuda, dims, C, H, W):
    img, maps, axes, th, angle = _case(H, W, dims, 3, 6, 2.0, H * 7 + W + C, C=C)
    got = _gpu(torch_cuda, img, maps, axes, th, angle)
    assert rel_err(got, _oracle(img, maps, axes, th, angle)) <= TOL32


@pytest.mark.parametrize("dims", [1, 2])
def test_rotated_fp16(torch_cuda, dims):
    img, maps, axes, th, angle = _case(90, 101, dims, 4, 8, 2.5, 5, fp16=True)
    got = _gpu(torch_cuda, img, maps, axes, th, angle)
    want = _oracle(img, maps, axes, th, angle).astype(np.float16).astype(np.float64)
    assert rel_err(got, want) <= TOL16


def test_rotated_tuned_tiles_and_large_reach(torch_cuda):
    """Both tile configurations (autotuned) with taps up to 12 px on both
    axes (Euclidean length up to 17 px: the rotated halo is the larger one)."""
    img, maps, axes, th, angle = _case(150, 170, 2, 3, 8, 1.0, 9)
    th[..., :2] = np.random.default_rng(3).uniform(-12, 12, th[..., :2].shape)
    got = _gpu(torch_cuda, img, maps, axes, th, angle, tune=True)
    assert rel_err(got, _oracle(img, maps, axes, th, angle)) <= TOL32


def test_zero_angle_matches_plain_filter(torch_cuda):
    from paper_2512_04556_gb300 import disk
    torch = torch_cuda
    img, maps, axes, th, _ = _case(64, 80, 1, 3, 6, 2.0, 11)
    b = disk.Basis.from_arrays(axes, th)
    t, m = torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()
    a = torch.zeros((64, 80), device="cuda", dtype=torch.float32)
    r = disk.sv_filter_rotated(b, t, m, a).cpu().numpy()
    p = disk.sv_filter(b, t, m).cpu().numpy()
    assert np.abs(r - p).max() <= 1e-6 * np.abs(p).max()


def test_non_finite_angle_acts_as_zero(torch_cuda):
    img, maps, axes, th, angle = _case(40, 50, 1, 2, 5, 2.0, 13)
    bad = angle.copy()
    bad[5, 7], bad[20, 30], bad[39, 49] = np.nan, np.inf, -np.inf
    fixed = bad.copy()
    fixed[~np.isfinite(fixed)] = 0.0
    np.testing.assert_array_equal(_gpu(torch_cuda, img, maps, axes, th, bad),
                                  _gpu(torch_cuda, img, maps, axes, th, fixed))


def test_rotated_halo_limit(torch_cuda):
    """Taps of 40 px on both axes (the per-axis limit) are 56.6 px long: the
    plain filter runs, the rotated one reports that the halo does not fit."""
    from paper_2512_04556_gb300 import disk
    torch = torch_cuda
    th = np.zeros((1, 1, 2, 3), np.float32)
    th[0, 0, 0] = (40.0, 40.0, 0.5)
    th[0, 0, 1] = (-40.0, -40.0, 0.5)
    b = disk.Basis.from_arrays([[0.0]], th)
    t = torch.rand((64, 64, 3), device="cuda")
    m = torch.zeros((1, 64, 64), device="cuda")
    disk.sv_filter(b, t, m)
    with pytest.raises(disk.DiskError) as e:
        disk.sv_filter_rotated(b, t, m, torch.zeros((64, 64), device="cuda"))
    assert e.value.code == -3 or "halo" in str(e.value)


@pytest.mark.parametrize("h0", [52, 56])
def test_rotated_long_taps(torch_cuda, h0):
    """Taps up to 36 px on both axes (51 px long) give a rotated halo of 52 px,
    staged rows of 32 + 2 x 64 pixels (the tile copy's box: 240 eight-byte
    elements of the 256 allowed) and a first-layer region at the edge of
    shared memory; a diagonal tap of 38.2 px per axis (halo 56) leaves the
    regions rounded to 16 pixels too large, so the first layer keeps its
    exact halo and the others round it to 4 pixels only."""
    img, maps, axes, th, angle = _case(120, 140, 1, 3, 4, 1.0, 17)
    g = np.random.default_rng(5)
    th[..., :2] = g.uniform(-36.0, 36.0, th[..., :2].shape)
    d = 36.0 if h0 == 52 else 38.2
    th[:, :, 0, 0], th[:, :, 0, 1] = d, -d            # one diagonal tap per layer
    got = _gpu(torch_cuda, img, maps, axes, th, angle)
    assert rel_err(got, _oracle(img, maps, axes, th, angle)) <= TOL32


def test_device_status_clean_after_filtering(torch_cuda):
    from paper_2512_04556_gb300 import disk
    img, maps, axes, th, angle = _case(64, 96, 2, 3, 6, 2.0, 23)
    _gpu(torch_cuda, img, maps, axes, th, angle)
    disk.device_status()


def test_bounded_wait_reports_timeout_and_context_survives(torch_cuda):
    """A tile-copy wait that runs out (a barrier nothing completes) records
    DISK_ERR_TIMEOUT, the status clears once read, and the context keeps
    working: the filter still matches the oracle afterwards."""
    from paper_2512_04556_gb300 import disk
    disk.device_status()
    disk.selftest_bounded_wait(2000)
    with pytest.raises(disk.DiskError) as e:
        disk.device_status()
    assert e.value.code == -6
    disk.device_status()
    img, maps, axes, th, angle = _case(40, 50, 2, 3, 6, 2.0, 29)
    got = _gpu(torch_cuda, img, maps, axes, th, angle)
    assert rel_err(got, _oracle(img, maps, axes, th, angle)) <= TOL32
