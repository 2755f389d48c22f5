"""GPU parity of the fitter (Eq. 4 objective, its hand-written backward,
Eq. 6 / Eq. 7 initialisations and the Adam loop) against the FP64 oracle,
through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _targets(n, kmin=7, kmax=25, first=0):
    return wl.shape_batch(n, seed=wl.SEED_SHAPE, kmin=kmin, kmax=kmax, first=first)


def _theta_away_from_integers(targets, L, T, seed):
    """Random complexes within each target's clamp box, fractions in [0.05, 0.95]."""
    g = np.random.default_rng(seed)
    out = []
    for t in targets:
        s = max(1.0, (t.shape[0] - 1) / 2)
        th = np.zeros((L, T, 3))
        o = g.uniform(-0.6 * s, 0.6 * s, (L, T, 2))
        o = np.floor(o) + np.clip(o - np.floor(o), 0.05, 0.95)
        th[..., :2] = o
        th[..., 2] = g.normal(1.0 / T, 0.3 / T, (L, T))
        out.append(th.astype(np.float32))
    return np.stack(out)


@pytest.mark.parametrize("loss,eps", [(0, 0.0), (1, 1e-4)])
@pytest.mark.parametrize("L,T", [(1, 8), (2, 5), (3, 8), (4, 16), (6, 12)])
def test_loss_and_gradient_match_oracle(torch_cuda, loss, eps, L, T):
    """The first layer's closed-form gradients (four pixels per tap; from
    dL/dI_1 directly at L = 1, through the second layer's adjoint otherwise),
    the second layer's (sums over the first layer's splats) and the swept
    layers' against the FP64 gradient."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = _targets(6, 7, 31)
    th = _theta_away_from_integers(tg, L, T, 1)
    packed, sizes = disk.pack_targets(tg)
    l, g = disk.fit_loss_grad(packed, sizes, torch.from_numpy(th).cuda(), loss=loss, eps=eps)
    torch.cuda.synchronize()
    l, g = l.cpu().numpy(), g.cpu().numpy()
    for b, t in enumerate(tg):
        wl_, wg = oracle.fit_loss(th[b].astype(np.float64), t, loss, eps, grad=True)
        assert abs(l[b] - wl_) <= 1e-4 * abs(wl_), (b, l[b], wl_)
        err = np.abs(g[b] - wg).max() / np.abs(wg).max()
        assert err <= 1e-4, (b, err)


@pytest.mark.parametrize("init", [1, 2, 3])
def test_initialisation_matches_oracle(torch_cuda, init):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = _targets(7, 9, 41, first=10)
    packed, sizes = disk.pack_targets(tg)
    th, _, _ = disk.fit(packed, sizes, 4, 16, 0, init=init, seed=77)
    torch.cuda.synchronize()
    th = th.cpu().numpy()
    for b, t in enumerate(tg):
        if init == 1:
            want = oracle.init_ir(t, 4, 16)
        elif init == 2:
            want, _ = oracle.init_ss(t, 4, 16, 77)
        else:
            want = oracle.init_rand(t.shape[0], 4, 16, 77)
        s = max(1.0, (t.shape[0] - 1) / 2)
        want[..., :2] = np.clip(want[..., :2], -s, s)
        if init == 2:   # dart-throwing decisions are exact: identical sample positions
            assert np.array_equal(th[b, 0, :, :2], want[0, :, :2].astype(np.float32))
        assert np.abs(th[b] - want).max() <= 1e-5 * s, (b, np.abs(th[b] - want).max())


def test_adam_trajectory_matches_oracle(torch_cuda):
    """20 Adam steps from the radial init: the parameter paths agree."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = _targets(4, 9, 21, first=20)
    packed, sizes = disk.pack_targets(tg)
    th, final, hist = disk.fit(packed, sizes, 3, 8, 20, init=1, loss_hist=True)
    torch.cuda.synchronize()
    th, hist = th.cpu().numpy(), hist.cpu().numpy()
    for b, t in enumerate(tg):
        want, whist = oracle.fit(t, 3, 8, 20, init=oracle.INIT_IR)
        s = max(1.0, (t.shape[0] - 1) / 2)
        assert np.abs(th[b] - want).max() <= 2e-3 * s, (b, np.abs(th[b] - want).max())
        np.testing.assert_allclose(hist[b], whist, rtol=2e-3)


def test_batched_fit_lowers_the_loss(torch_cuda):
    """A batch of uneven non-convex targets: every loss falls, and sparse
    sampling beats random offsets on the median."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = _targets(24, 15, 51, first=40)
    packed, sizes = disk.pack_targets(tg)
    res = {}
    for init in (2, 3):
        th, final, hist = disk.fit(packed, sizes, 3, 12, 150, init=init, seed=5, loss_hist=True)
        torch.cuda.synchronize()
        hist = hist.cpu().numpy()
        assert np.all(hist[:, -1] < hist[:, 0])
        res[init] = np.median(hist[:, -1] / hist[:, 0])
    assert res[2] < res[3]


def test_fit_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    packed, sizes = disk.pack_targets(_targets(2))
    with pytest.raises(disk.DiskError):
        disk.fit(packed, [8, 9], 3, 8, 5)                 # even size
    with pytest.raises(disk.DiskError):
        disk.fit(packed, sizes, 16, 64, 5)                # L * T > 512


def test_autotune_and_cuda_graph_replay(torch_cuda):
    """The autotuner picks one of its CTA sizes, and a whole fit (plan
    upload, sparse-sampling init, persistent kernel) captured in a CUDA graph
    replays to exactly the eager result."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = _targets(12, 9, 41, first=60)
    packed, sizes = disk.pack_targets(tg)
    assert disk.fit_autotune(packed, sizes, 3, 8) in {(256, 1), (512, 1), (1024, 1), (512, 2),
                                                      (1024, 2), (512, 4), (1024, 4)}
    eager, eager_loss, _ = disk.fit(packed, sizes, 3, 8, 30, init=2, seed=3)
    theta = torch.zeros_like(eager)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        disk.fit(packed, sizes, 3, 8, 1, init=2, seed=3, theta=theta)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        _, loss, _ = disk.fit(packed, sizes, 3, 8, 30, init=2, seed=3, theta=theta)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(theta, eager)
        assert torch.equal(loss, eager_loss)


@pytest.mark.parametrize("threads,ctas", [(256, 1), (512, 1), (1024, 1), (512, 2), (1024, 2),
                                          (512, 4), (1024, 4)])
def test_fit_launch_configurations_match_oracle(torch_cuda, threads, ctas):
    """Every launch configuration -- including a target split over a cluster
    of 2 or 4 CTAs, whose loss and tap gradients are summed through
    distributed shared memory -- follows the FP64 oracle's loss history."""
    from paper_2512_04556_gb300 import disk
    tg = [wl.ring(40.0, 6.0, 97), wl.star(6, 30.0, 14.0, 0.3, 65), wl.disk(12.0, 33)]
    packed, sizes = disk.pack_targets(tg)
    disk.fit_set_config(4, 16, max(sizes), threads, ctas)
    _, _, hist = disk.fit(packed, sizes, 4, 16, 60, init=disk.INIT_SS, seed=5, loss_hist=True)
    hist = hist.cpu().numpy()
    for b in range(len(tg)):
        want = _oracle_hist(tg[b], b)
        np.testing.assert_allclose(hist[b, [0, 30, 60]], want[[0, 30, 60]], rtol=2e-2)


_ORACLE_CACHE = {}


def _oracle_hist(t, key):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle.fit(t, 4, 16, 60, init=oracle.INIT_SS, seed=5)[1]
    return _ORACLE_CACHE[key]


@pytest.mark.parametrize("K,L,T", [(257, 4, 16), (33, 8, 64), (21, 16, 32), (1, 2, 4), (3, 1, 1)])
def test_fit_at_the_size_limits(torch_cuda, K, L, T):
    """The largest target (K = 257), the largest complexes (L * T = 512, up to
    16 layers; the splat list then fills 256 threads) and degenerate ones
    (K = 1, T = 1): loss and gradient against the FP64 oracle, and five Adam
    steps against the oracle's trajectory."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    t = wl.ring(max(1.0, (K - 1) / 2 - 2.0), max(1.5, K / 12), K) if K >= 9 else wl.disk(1.0, K)
    th = _theta_away_from_integers([t], L, T, K + L)
    packed, sizes = disk.pack_targets([t])
    l, g = disk.fit_loss_grad(packed, sizes, torch.from_numpy(th).cuda())
    torch.cuda.synchronize()
    wl_, wg = oracle.fit_loss(th[0].astype(np.float64), t, 0, 0.0, grad=True)
    assert abs(float(l[0]) - wl_) <= 1e-4 * abs(wl_)
    err = np.abs(g.cpu().numpy()[0] - wg).max() / max(np.abs(wg).max(), 1e-30)
    assert err <= 1e-4, err
    got, _, hist = disk.fit(packed, sizes, L, T, 5, init=disk.INIT_GIVEN,
                            theta=torch.from_numpy(th).cuda(), loss_hist=True)
    want, whist = oracle.fit(t, L, T, 5, init=oracle.INIT_GIVEN, theta0=th[0].astype(np.float64))
    np.testing.assert_allclose(hist.cpu().numpy()[0], whist, rtol=2e-3)
    s = max(1.0, (K - 1) / 2)
    assert np.abs(got.cpu().numpy()[0] - want).max() <= 2e-3 * s
