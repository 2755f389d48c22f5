"""Parity at the full benchmark sizes, in the launch configuration the
benchmark times, on sampled outputs the FP64 oracle computes one by one.

An output pixel of the L-layer cascade depends only on the input within
R = sum_l (ceil(max |o_l|) + 1) of it, so the oracle filters the crop of
radius R around each sampled pixel (clipped at the true image border, where
clamp-to-edge then reads exactly what the full frame reads) and the GPU's
full-frame output is compared there.  The image gradient is sampled the same
way (its dependency cone has the same radius).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import basis_io, mlp
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASES = os.path.join(ROOT, "tests", "golden", "bases")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _samples(H, W, n, seed):
    g = np.random.default_rng(seed)
    pts = [(0, 0), (H - 1, W - 1), (0, W - 1), (H - 1, 0), (H // 2, 3), (5, W // 2)]
    pts += [(int(g.integers(0, H)), int(g.integers(0, W))) for _ in range(n - len(pts))]
    return pts


def _cone(theta):
    return int(sum(np.ceil(np.abs(theta[:, l, :, :2]).max()) + 1 for l in range(theta.shape[1])))


def _crop_oracle(fn, arr, maps, y, x, R):
    H, W = arr.shape[:2]
    y0, y1, x0, x1 = max(0, y - R), min(H, y + R + 1), max(0, x - R), min(W, x + R + 1)
    out = fn(np.ascontiguousarray(arr[y0:y1, x0:x1]).astype(np.float64),
             np.ascontiguousarray(maps[:, y0:y1, x0:x1]).astype(np.float64))
    return out[y - y0, x - x0]


def _frame4k():
    H, W = wl.C4["H"], wl.C4["W"]
    img = wl.to_fp16(wl.image_rects(H, W, 3))
    m0 = wl.param_map(H, W, *wl.C4["map_range0"], sigma=wl.C4["map_sigma"], stream=0)
    m1 = wl.param_map(H, W, *wl.C4["map_range1"], sigma=wl.C4["map_sigma"], stream=1)
    return img, np.stack([m0, m1])


def test_4k_fp16_2d_filter_sampled(torch_cuda):
    """The benchmark frame (3840 x 2160 FP16, 8 x 8 fitted ellipses, L=4,
    T=24), filtered exactly as bench.py does, against the oracle on crops."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    img, maps = _frame4k()
    path = os.path.join(BASES, "ellipse8x8_L4T24.dkb")
    b = disk.Basis.load(path)
    out = disk.sv_filter(b, torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()).cpu().numpy()
    axes, th = basis_io.read(path)
    th = th.astype(np.float64)
    R = _cone(th)
    nn, nv = [len(a) for a in axes], np.concatenate(axes).astype(np.float64)
    fn = lambda a, m: oracle.sv_filter(a, m, nn, nv, th)
    got, want = [], []
    for (y, x) in _samples(*img.shape[:2], 24, 0):
        want.append(np.float16(_crop_oracle(fn, img, maps, y, x, R)).astype(np.float64))
        got.append(out[y, x].astype(np.float64))
    got, want = np.array(got), np.array(want)
    assert np.abs(got - want).max() / np.abs(want).max() <= 2e-3


def test_4k_fp16_2d_image_gradient_sampled(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    img, maps = _frame4k()
    path = os.path.join(BASES, "ellipse8x8_L4T24.dkb")
    b = disk.Basis.load(path)
    go = wl.to_fp16(np.random.default_rng(9).uniform(-1, 1, img.shape).astype(np.float32))
    gi = disk.sv_filter_backward_image(b, torch.from_numpy(go).cuda(),
                                       torch.from_numpy(maps).cuda()).cpu().numpy()
    axes, th = basis_io.read(path)
    th = th.astype(np.float64)
    R = _cone(th)
    nn, nv = [len(a) for a in axes], np.concatenate(axes).astype(np.float64)
    fn = lambda a, m: oracle.sv_filter_adjoint(a, m, nn, nv, th)
    got, want = [], []
    for (y, x) in _samples(*img.shape[:2], 12, 1):
        want.append(_crop_oracle(fn, go, maps, y, x, R))
        got.append(gi[y, x].astype(np.float64))
    got, want = np.array(got), np.array(want)
    assert np.abs(got - want).max() / np.abs(want).max() <= 1e-5


def test_4k_fp16_gaussian_tilt_shift_sampled(torch_cuda):
    """3840 x 2160 FP16 under a tilt-shift sigma map (1..11 px), 11 fitted
    Gaussians, L=6, T=8, autotuned tiles as the benchmark's Gaussian leg."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    g = wl.G
    H, W = g["H"], g["W"]
    img = wl.to_fp16(wl.image_rects(H, W, 3))
    maps = wl.tilt_shift_map(H, W, *g["map_range"])[None]
    path = os.path.join(BASES, "gauss11_L6T8.dkb")
    b = disk.Basis.load(path)
    di, dm = torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()
    disk.sv_filter_autotune(b, di, dm)
    out = disk.sv_filter(b, di, dm).cpu().numpy()
    axes, th = basis_io.read(path)
    th = th.astype(np.float64)
    R = _cone(th)
    fn = lambda a, m: oracle.sv_filter(a, m, [len(axes[0])], axes[0].astype(np.float64), th)
    pts = _samples(H, W, 20, 3)
    pts += [(int(0.55 * H), 100), (int(0.55 * H) + 120, 2000)]      # in and at the edge of focus
    got, want = [], []
    for (y, x) in pts:
        want.append(np.float16(_crop_oracle(fn, img, maps, y, x, R)).astype(np.float64))
        got.append(out[y, x].astype(np.float64))
    got, want = np.array(got), np.array(want)
    assert np.abs(got - want).max() / np.abs(want).max() <= 2e-3


def _cone_rot(theta):
    return int(sum(np.ceil(np.hypot(theta[:, l, :, 0], theta[:, l, :, 1]).max()) + 1
                   for l in range(theta.shape[1])))


@pytest.mark.parametrize("preset,fname,tangential", [
    (wl.RM, "line12_L3T8.dkb", False), (wl.RB, "cateye12_L4T16.dkb", True)])
def test_4k_fp16_rotated_sampled(torch_cuda, preset, fname, tangential):
    """3840 x 2160 FP16, radial motion blur (segments 2..40 px, L=3, T=8) and
    rotational bokeh (aspect-2 ellipses 2..24 px, L=4, T=16): a 1-D basis
    over strength turned per pixel by the radial / tangential angle map,
    autotuned tiles as the benchmark's legs."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    H, W = preset["H"], preset["W"]
    img = wl.to_fp16(wl.image_rects(H, W, 3))
    strength, angle = wl.radial_maps(H, W, *preset["map_range"], tangential=tangential)
    maps = strength[None]
    path = os.path.join(BASES, fname)
    b = disk.Basis.load(path)
    di, dm, da = (torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda(),
                  torch.from_numpy(angle).cuda())
    disk.sv_filter_rotated_autotune(b, di, dm, da)
    out = disk.sv_filter_rotated(b, di, dm, da).cpu().numpy()
    axes, th = basis_io.read(path)
    th = th.astype(np.float64)
    R = _cone_rot(th)
    nv = axes[0].astype(np.float64)
    got, want = [], []
    for (y, x) in _samples(H, W, 20, 4):
        y0, y1, x0, x1 = max(0, y - R), min(H, y + R + 1), max(0, x - R), min(W, x + R + 1)
        o = oracle.sv_filter_rotated(img[y0:y1, x0:x1].astype(np.float64),
                                     maps[:, y0:y1, x0:x1].astype(np.float64),
                                     angle[y0:y1, x0:x1].astype(np.float64), [len(nv)], nv, th)
        want.append(np.float16(o[y - y0, x - x0]).astype(np.float64))
        got.append(out[y, x].astype(np.float64))
    got, want = np.array(got), np.array(want)
    assert np.abs(got - want).max() / np.abs(want).max() <= 2e-3


def test_1080p_fp32_1d_filter_sampled(torch_cuda):
    """1920 x 1080 FP32, 16 fitted disks (radius 1..32), L=4, T=16."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    H, W = 1080, 1920
    img = wl.image_rects(H, W, 3)
    maps = wl.param_map(H, W, 1.0, 32.0, sigma=96.0)[None]
    path = os.path.join(BASES, "disk16_L4T16.dkb")
    b = disk.Basis.load(path)
    out = disk.sv_filter(b, torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()).cpu().numpy()
    axes, th = basis_io.read(path)
    th = th.astype(np.float64)
    R = _cone(th)
    fn = lambda a, m: oracle.sv_filter(a, m, [16], axes[0].astype(np.float64), th)
    got, want = [], []
    for (y, x) in _samples(H, W, 24, 2):
        want.append(_crop_oracle(fn, img, maps, y, x, R))
        got.append(out[y, x].astype(np.float64))
    got, want = np.array(got), np.array(want)
    assert np.abs(got - want).max() / np.abs(want).max() <= 1e-5


def test_full_fit_batch_sampled_targets(torch_cuda):
    """The 256-target batch fitted in one launch as the benchmark does (sparse
    sampling, 500 steps, 512 threads x 4-CTA clusters); the oracle fits two of
    its smallest targets and its largest alone.  The loss histories agree to
    2 % after 500 steps (FP32 vs FP64 paths)."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = wl.shape_batch(256)
    packed, sizes = disk.pack_targets(tg)
    disk.fit_set_config(4, 16, max(sizes), 512, 4)
    _, _, hist = disk.fit(packed, sizes, 4, 16, 500, init=disk.INIT_SS, seed=7, loss_hist=True)
    hist = hist.cpu().numpy()
    for b in list(np.argsort(sizes)[:2]) + [int(np.argmax(sizes))]:
        _, wh = oracle.fit(tg[b], 4, 16, 500, init=oracle.INIT_SS, seed=7)
        np.testing.assert_allclose(hist[b, [0, 100, 500]], wh[[0, 100, 500]], rtol=2e-2)


def test_mlp_full_shape_forward(torch_cuda):
    """The learned initializer's network at its full shape (4096-512-512-512-192,
    batch 256) against the FP64 oracle."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    net = disk.MLP(4096, 512, 3, 192, seed=3)
    x = np.random.default_rng(4).random((256, 4096)).astype(np.float32)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = mlp.forward(net.params.cpu().numpy().astype(np.float64), x.astype(np.float64),
                          4096, 512, 3, 192)
    assert np.abs(y - want).max() <= 1e-5 * np.abs(want).max()
