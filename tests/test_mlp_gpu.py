"""GPU parity of the learned initializer's kernels (forward, training step
with its hand-written backward and Adam, area resampling) against the FP64
oracle."""
import numpy as np
import pytest

from oracle import mlp
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def test_forward_and_train_step_match_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    shape = (70, 33, 3, 21)                 # ragged against the 64 x 64 GEMM tiles
    net = disk.MLP(*shape, seed=5)
    p0 = net.params.cpu().numpy().astype(np.float64)
    lim = np.sqrt(6 / 70)
    w0 = p0[:70 * 33]                        # He-uniform: U(-lim, lim), std lim / sqrt(3)
    assert np.abs(w0).max() <= lim and abs(w0.std() - lim / np.sqrt(3)) < 0.05 * lim
    g = np.random.default_rng(1)
    x = g.random((37, 70)).astype(np.float32)
    t = g.normal(0, 1, (37, 21)).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(dx).cpu().numpy()
    want, _ = mlp.forward(p0, x.astype(np.float64), *shape)
    assert np.abs(y - want).max() <= 1e-5 * np.abs(want).max()
    loss = net.train_step(dx, dt, lr=1e-3)
    torch.cuda.synchronize()
    wl_, wg = mlp.loss_and_grad(p0, x.astype(np.float64), t.astype(np.float64), *shape)
    assert abs(loss.item() - wl_) <= 1e-5 * wl_
    wp, _, _ = mlp.adam(p0, np.zeros_like(p0), np.zeros_like(p0), wg, 1, 1e-3)
    got = net.params.cpu().numpy()
    # first Adam step: lr * sign(g) wherever |g| >> eps; compare the update
    upd, wupd = got - p0, wp - p0
    big = np.abs(wg) > 1e-6
    assert np.abs(upd[big] - wupd[big]).max() <= 1e-5


def test_full_size_network_on_tensor_cores_matches_oracle(torch_cuda):
    """The benchmark network (4096-512-512-512-192, batch 256): every product
    runs on the tensor cores (four TF32 hi/lo products per FP32 product, split-K
    over the SMs); forward, loss and gradient against the FP64 oracle at the
    FP32 gate."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    shape = (4096, 512, 3, 192)
    net = disk.MLP(*shape, seed=11)
    p0 = net.params.cpu().numpy().astype(np.float64)
    g = np.random.default_rng(12)
    x = g.random((256, 4096)).astype(np.float32)
    t = (0.5 * g.standard_normal((256, 192))).astype(np.float32)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(dx).cpu().numpy()
    want, _ = mlp.forward(p0, x.astype(np.float64), *shape)
    assert np.abs(y - want).max() <= 1e-5 * np.abs(want).max()
    loss, grad = net.grad(dx, dt)
    wl_, wg = mlp.loss_and_grad(p0, x.astype(np.float64), t.astype(np.float64), *shape)
    assert abs(loss.item() - wl_) <= 1e-5 * wl_
    gg = grad.cpu().numpy()
    for (lo, hi) in _layer_ranges(shape):
        ref = wg[lo:hi]
        assert np.abs(gg[lo:hi] - ref).max() <= 1e-5 * np.abs(ref).max(), (lo, hi)


def _layer_ranges(shape):
    dims = mlp.layer_dims(*shape)
    out, off = [], 0
    for a, b in dims:
        out.append((off, off + a * b))          # weights
        out.append((off + a * b, off + a * b + b))  # biases
        off += a * b + b
    return out


def test_area_resampling_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = wl.shape_batch(5, kmin=33, kmax=129, first=300) + [wl.disk(31.5)]
    packed, sizes = disk.pack_targets(tg)
    out = disk.downsample_targets(packed, sizes, 64).cpu().numpy()
    for b, t in enumerate(tg):
        want = mlp.downsample(t.astype(np.float64), 64)
        assert np.abs(out[b] - want).max() <= 1e-5, b


def test_learned_initializer_gains_over_the_radial_start(torch_cuda, capsys):
    """A small learned initializer (training pairs from the project's own
    fitter) reaches the plain fitter's final loss in fewer Adam steps on
    held-out targets than the paper's radial start needs (its full run)."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk, learned_init as li
    L, T, steps = 3, 8, 200
    train_t = wl.shape_batch(8000, kmin=17, kmax=33, first=0)
    held_t = wl.shape_batch(128, kmin=17, kmax=33, first=5_000_000)
    th, _ = li.fit_pairs(train_t, L, T, steps)
    X = li.features(train_t)
    Y = li.to_labels(th, [t.shape[0] for t in train_t], T)
    net = disk.MLP(li.SIDE * li.SIDE, 512, 2, L * T * 3, seed=1)
    li.train(net, X, Y, epochs=30, batch=128)
    res = li.evaluate(net, held_t, L, T, steps)
    with capsys.disabled():
        print("\nlearned-init gain (toy config):", res)
    # this small configuration (8,000 pairs of 17..33 px targets, L = 3,
    # T = 8, 200 steps, a 4096-512-512-72 network) gains about 3.8x on
    # GB300; the floor is 2.5x fewer steps
    assert res["speedup"] >= 2.5, res
    assert res["median_start_loss_ratio"] < 1.0, res


def test_grad_matches_oracle_and_halves_average_to_full_batch(torch_cuda):
    """disk_mlp_grad against the FP64 gradient; the mean of two half-batch
    gradients is the full-batch gradient (what the data-parallel all-reduce
    relies on), and applying it equals one train_step on the full batch."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    shape = (64, 48, 2, 12)
    g = np.random.default_rng(31)
    x = g.random((40, 64)).astype(np.float32)
    t = g.normal(size=(40, 12)).astype(np.float32)
    a = disk.MLP(*shape, seed=9)
    b = disk.MLP(*shape, seed=9)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss, grad = a.grad(xd, td)
    wl_, wg = mlp.loss_and_grad(a.params.cpu().numpy().astype(np.float64), x, t, *shape)
    assert abs(loss.item() - wl_) <= 1e-5 * abs(wl_)
    assert np.abs(grad.cpu().numpy() - wg).max() <= 1e-5 * np.abs(wg).max()
    _, g1 = a.grad(xd[:20], td[:20])
    _, g2 = a.grad(xd[20:], td[20:])
    avg = (g1 + g2) / 2
    assert (avg - grad).abs().max().item() <= 1e-5 * grad.abs().max().item()
    a.apply(avg, 1e-3)
    b.train_step(xd, td, 1e-3)
    assert (a.params - b.params).abs().max().item() <= 1e-6


def _composed_learned_start(torch, net, packed, sizes, L, T):
    """The learned start assembled from the other entry points and torch
    arithmetic: resample, forward, network units -> pixels, Eq. 6 start, the
    fitted loss of both, the lower one kept (network on a tie)."""
    from paper_2512_04556_gb300 import disk
    X = disk.downsample_targets(packed, sizes, 64).reshape(len(sizes), -1)
    y = net.forward(X).reshape(-1, L, T, 3)
    s = torch.tensor([max(1.0, (k - 1) / 2) for k in sizes], dtype=torch.float32,
                     device=y.device)[:, None, None]
    th_net = torch.stack([y[..., 0].clamp(-1, 1) * s, y[..., 1].clamp(-1, 1) * s, y[..., 2] / T],
                         dim=-1).contiguous()
    th_ir = disk.fit(packed, sizes, L, T, 0, init=disk.INIT_IR)[0]
    l_net, _ = disk.fit_loss_grad(packed, sizes, th_net)
    l_ir, _ = disk.fit_loss_grad(packed, sizes, th_ir)
    keep = l_net <= l_ir
    return torch.where(keep[:, None, None, None], th_net, th_ir), keep


def test_learned_init_entry_point_equals_its_steps(torch_cuda):
    """disk_learned_init (all steps on the device behind the C ABI) gives the
    composed pipeline's starts bit for bit, for a random network and for one
    whose output is the single-point complex (all taps at 0, weights 1/T):
    that start is exact on a one-pixel target and worse than the Eq. 6 ring
    on broad ones, so both branches of the choice are taken."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    L, T = 2, 4
    point = np.zeros((17, 17), np.float32)
    point[8, 8] = 1.0
    tg = wl.shape_batch(30, kmin=17, kmax=45, first=900) + [point, wl.disk(9.0)]
    packed, sizes = disk.pack_targets(tg)
    rand_net = disk.MLP(64 * 64, 64, 2, L * T * 3, seed=3)
    point_net = disk.MLP(64 * 64, 64, 2, L * T * 3, seed=3)
    point_net.params.zero_()
    bias = torch.zeros((L, T, 3), device="cuda")
    bias[..., 2] = 1.0                       # weight label w * T = 1
    point_net.params[-L * T * 3:] = bias.reshape(-1)
    for net in (rand_net, point_net):
        got, used = disk.learned_init(net, packed, sizes, L, T)
        want, keep = _composed_learned_start(torch, net, packed, sizes, L, T)
        assert torch.equal(used, keep)
        assert torch.equal(got, want)
    assert bool(used[-2]) and not bool(used[-1])
