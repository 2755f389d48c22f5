"""GPU parity of the image gradient of the spatially varying filter against
the oracle's transpose, and the forward/backward dot-product identity."""
import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _case(H, W, dims, seed, spread=1.5, L=3, T=5):
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
    th[..., 2] = g.normal(0.2, 0.3, th[..., 2].shape)   # signed weights
    return axes, th.astype(np.float32), maps.astype(np.float32)


def _oracle_adjoint(gout, maps, axes, th):
    return oracle.sv_filter_adjoint(gout.astype(np.float64), maps.astype(np.float64),
                                    [len(a) for a in axes], np.concatenate(axes).astype(np.float64),
                                    th.astype(np.float64))


@pytest.mark.parametrize("dims,H,W,C,dtype", [(1, 37, 45, 3, "f32"), (2, 40, 33, 3, "f32"),
                                             (1, 5, 70, 4, "f32"), (2, 31, 29, 3, "f16"),
                                             (1, 64, 96, 3, "f16")])
def test_image_gradient_matches_oracle_transpose(torch_cuda, dims, H, W, C, dtype):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    axes, th, maps = _case(H, W, dims, H * 7 + W)
    gout = np.random.default_rng(W).standard_normal((H, W, C)).astype(np.float32)
    if dtype == "f16":
        gout = gout.astype(np.float16)
    b = disk.Basis.from_arrays(axes, th)
    got = disk.sv_filter_backward_image(b, torch.from_numpy(gout).cuda(), torch.from_numpy(maps).cuda())
    torch.cuda.synchronize()
    want = _oracle_adjoint(gout, maps, axes, th)
    err = np.abs(got.cpu().numpy() - want).max() / np.abs(want).max()
    assert err <= TOL, err


def test_backward_is_transpose_of_forward_on_gpu(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    H, W = 70, 90
    axes, th, maps = _case(H, W, 2, 3, spread=3.0)
    b = disk.Basis.from_arrays(axes, th)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((H, W, 3), device="cuda", generator=g)
    y = torch.randn((H, W, 3), device="cuda", generator=g)
    dm = torch.from_numpy(maps).cuda()
    lhs = (disk.sv_filter(b, x, dm).double() * y.double()).sum().item()
    rhs = (x.double() * disk.sv_filter_backward_image(b, y, dm).double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_autograd_function_image_gradient(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import autograd, disk
    H, W = 33, 47
    axes, th, maps = _case(H, W, 1, 9)
    b = disk.Basis.from_arrays(axes, th)
    img = torch.rand((H, W, 3), device="cuda", requires_grad=True)
    dm = torch.from_numpy(maps).cuda()
    w = torch.rand((H, W, 3), device="cuda")
    (autograd.sv_filter(img, dm, b) * w).sum().backward()
    want = _oracle_adjoint(w.cpu().numpy(), maps, axes, th)
    err = np.abs(img.grad.cpu().numpy() - want).max() / np.abs(want).max()
    assert err <= TOL


def test_autograd_function_image_gradient_fp16_storage(torch_cuda):
    """FP16 image: the incoming FP16 gradient reaches the library unchanged,
    the library's FP32 image gradient matches the FP64 transpose at the FP32
    gate, and autograd rounds it to FP16 once (within one FP16 unit of the
    rounded oracle)."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import autograd, disk
    H, W = 37, 52
    axes, th, maps = _case(H, W, 2, 19)
    b = disk.Basis.from_arrays(axes, th)
    img = torch.rand((H, W, 3), device="cuda").half().requires_grad_()
    dm = torch.from_numpy(maps).cuda()
    w = torch.rand((H, W, 3), device="cuda").half()
    (autograd.sv_filter(img, dm, b) * w).sum().backward()
    want = _oracle_adjoint(w.float().cpu().numpy(), maps, axes, th)
    g32 = disk.sv_filter_backward_image(b, w, dm).cpu().numpy()
    assert np.abs(g32 - want).max() / np.abs(want).max() <= TOL
    assert img.grad.dtype == torch.float16
    want16 = want.astype(np.float16).astype(np.float64)
    err = np.abs(img.grad.cpu().numpy().astype(np.float64) - want16).max() / np.abs(want).max()
    assert err <= 2.0 ** -10


@pytest.mark.parametrize("dims,H,W,C", [(1, 29, 41, 3), (2, 35, 30, 3), (1, 20, 64, 4)])
def test_theta_gradient_matches_oracle(torch_cuda, dims, H, W, C):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    axes, th, maps = _case(H, W, dims, 40 + H)
    rng = np.random.default_rng(41)
    img = rng.random((H, W, C)).astype(np.float32)
    gout = rng.standard_normal((H, W, C)).astype(np.float32)
    b = disk.Basis.from_arrays(axes, th)
    gi, gt = disk.sv_filter_backward(b, torch.from_numpy(img).cuda(), torch.from_numpy(gout).cuda(),
                                     torch.from_numpy(maps).cuda())
    torch.cuda.synchronize()
    nn = [len(a) for a in axes]
    nv = np.concatenate(axes).astype(np.float64)
    want_t = oracle.sv_filter_grad_theta(img.astype(np.float64), gout.astype(np.float64),
                                         maps.astype(np.float64), nn, nv, th.astype(np.float64))
    err_t = np.abs(gt.cpu().numpy() - want_t).max() / np.abs(want_t).max()
    assert err_t <= 1e-4, err_t
    want_i = _oracle_adjoint(gout, maps, axes, th)
    assert np.abs(gi.cpu().numpy() - want_i).max() / np.abs(want_i).max() <= TOL


def test_theta_gradient_fp16_storage(torch_cuda):
    """FP16 images keep FP16 activations: the gradient stays within the FP16 gate."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    H, W = 32, 48
    axes, th, maps = _case(H, W, 2, 50)
    rng = np.random.default_rng(51)
    img = rng.random((H, W, 3)).astype(np.float16)
    gout = rng.standard_normal((H, W, 3)).astype(np.float16)
    b = disk.Basis.from_arrays(axes, th)
    _, gt = disk.sv_filter_backward(b, torch.from_numpy(img).cuda(), torch.from_numpy(gout).cuda(),
                                    torch.from_numpy(maps).cuda(), grad_img=False)
    torch.cuda.synchronize()
    want = oracle.sv_filter_grad_theta(img.astype(np.float64), gout.astype(np.float64),
                                       maps.astype(np.float64), [3, 4],
                                       np.concatenate(axes).astype(np.float64), th.astype(np.float64))
    assert np.abs(gt.cpu().numpy() - want).max() / np.abs(want).max() <= 2e-3


def test_theta_gradient_central_differences_on_gpu(torch_cuda):
    """Central differences of the GPU forward (FP32) agree with the GPU
    gradient on a sample of weights and offsets."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    H, W = 40, 40
    axes, th, maps = _case(H, W, 1, 60)
    rng = np.random.default_rng(61)
    img = torch.from_numpy(rng.random((H, W, 3)).astype(np.float32)).cuda()
    gout = torch.from_numpy(rng.standard_normal((H, W, 3)).astype(np.float32)).cuda()
    dm = torch.from_numpy(maps).cuda()
    _, gt = disk.sv_filter_backward(disk.Basis.from_arrays(axes, th), img, gout, dm, grad_img=False)
    gt = gt.cpu().numpy()

    def loss(t):
        out = disk.sv_filter(disk.Basis.from_arrays(axes, t), img, dm)
        return float((out.double() * gout.double()).sum().item())

    # weights enter linearly (any step is exact); offsets use a small step so
    # that few pixels see a bilinear kink between the two evaluations
    for idx in [(0, 0, 0, 2), (1, 1, 2, 2), (2, 2, 4, 0), (3, 0, 1, 1), (1, 2, 3, 0)]:
        h = 1e-2 if idx[3] == 2 else 1e-3
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(fd - gt[idx]) <= 2e-2 * max(abs(fd), 1e-2 * np.abs(gt).max()), (idx, fd, gt[idx])


def test_autograd_cascade_theta_and_image(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import autograd
    H, W = 30, 37
    axes, th, maps = _case(H, W, 2, 70)
    rng = np.random.default_rng(71)
    img = torch.from_numpy(rng.random((H, W, 3)).astype(np.float32)).cuda().requires_grad_()
    theta = torch.from_numpy(th).cuda().requires_grad_()
    w = torch.from_numpy(rng.standard_normal((H, W, 3)).astype(np.float32)).cuda()
    (autograd.sv_cascade(img, torch.from_numpy(maps).cuda(), theta, axes) * w).sum().backward()
    want_t = oracle.sv_filter_grad_theta(img.detach().cpu().numpy().astype(np.float64),
                                         w.cpu().numpy().astype(np.float64), maps.astype(np.float64),
                                         [3, 4], np.concatenate(axes).astype(np.float64),
                                         th.astype(np.float64))
    assert np.abs(theta.grad.cpu().numpy() - want_t).max() / np.abs(want_t).max() <= 1e-4
    want_i = _oracle_adjoint(w.cpu().numpy(), maps, axes, th)
    assert np.abs(img.grad.cpu().numpy() - want_i).max() / np.abs(want_i).max() <= TOL
