"""GPU tests of the checkpointed fit (disk_fit_resume) and of the network
checkpoint: a fit of n Adam steps cut into segments, with the optimiser state
carried between calls or through a checkpoint file, returns bit for bit what
the unbroken disk_fit returns (same launch configuration), and the unbroken
fit follows the FP64 oracle."""
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


def _batch():
    return [wl.ring(9.0, 2.5, 27), wl.star(5, 8.0, 4.0, 0.3, 21), wl.disk(4.0, 11),
            wl.ring(3.0, 1.5, 9)]


def _start(tg, L, T, seed):
    g = np.random.default_rng(seed)
    th = np.zeros((len(tg), L, T, 3), np.float32)
    for b, t in enumerate(tg):
        s = max(1.0, (t.shape[0] - 1) / 2)
        th[b, ..., :2] = g.uniform(-0.7 * s, 0.7 * s, (L, T, 2))
        th[b, ..., 2] = g.normal(1.0 / T, 0.2 / T, (L, T))
    return th


@pytest.mark.parametrize("init,loss,threads,ctas", [
    (1, 0, 512, 1), (2, 0, 1024, 2), (0, 1, 512, 4), (3, 0, 256, 1)])
def test_split_fit_equals_unbroken_fit(torch_cuda, init, loss, threads, ctas):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = _batch()
    L, T, n, k, eps = 3, 8, 40, 15, (1e-4 if loss else 0.0)
    packed, sizes = disk.pack_targets(tg)
    disk.fit_set_config(L, T, max(sizes), threads, ctas)
    th0 = torch.from_numpy(_start(tg, L, T, 11)).cuda()
    full, full_loss, hist = disk.fit(packed, sizes, L, T, n, init=init, loss=loss, eps=eps,
                                     seed=9, theta=th0.clone(), loss_hist=True)
    state = torch.full((len(tg), 3, L * T * 3), float("nan"), device="cuda")
    theta = th0.clone()
    _, h1 = disk.fit_resume(packed, sizes, state, theta, 0, k, n, init=init, loss=loss, eps=eps,
                            seed=9, loss_hist=True)
    mid_theta, mid_state = theta.clone(), state.clone()
    theta.fill_(float("nan"))                       # ignored when step0 > 0
    _, h2 = disk.fit_resume(packed, sizes, state, theta, k, 0, n, loss=loss, eps=eps,
                            loss_hist=True)
    assert torch.equal(theta, mid_theta) and torch.equal(state, mid_state)
    fin, h3 = disk.fit_resume(packed, sizes, state, theta, k, n - k, n, loss=loss, eps=eps,
                              loss_hist=True)
    torch.cuda.synchronize()
    assert torch.equal(theta, full) and torch.equal(fin, full_loss)
    assert torch.equal(h1, hist[:, :k + 1]) and torch.equal(h3, hist[:, k:])
    assert torch.equal(h2[:, 0], hist[:, k])
    # the state's layout: offsets / s_b (clamped), raw weights, then the moments
    st, th = state.cpu().numpy(), theta.cpu().numpy()
    for b, t in enumerate(tg):
        s = np.float32(max(1.0, (t.shape[0] - 1) / 2))
        q = st[b, 0].reshape(L, T, 3)
        assert np.abs(q[..., :2]).max() <= 1.0
        np.testing.assert_array_equal(q[..., :2] * s, th[b, ..., :2])
        np.testing.assert_array_equal(q[..., 2], th[b, ..., 2])
        assert (st[b, 2] >= 0).all() and np.isfinite(st[b, 1:]).all()
    if init == 1 and loss == 0:
        for b, t in enumerate(tg):
            want, whist = oracle.fit(t, L, T, n, init=oracle.INIT_IR)
            s = max(1.0, (t.shape[0] - 1) / 2)
            assert np.abs(th[b] - want).max() <= 2e-3 * s
            np.testing.assert_allclose(hist[b].cpu().numpy(), whist, rtol=2e-3)


def test_checkpoint_file_survives_an_interrupted_run(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2512_04556_gb300 import checkpoint as ck
    from paper_2512_04556_gb300 import disk
    tg = _batch()
    L, T, n = 3, 8, 50
    packed, sizes = disk.pack_targets(tg)
    disk.fit_set_config(L, T, max(sizes), 512, 1)
    want, want_loss, _ = disk.fit(packed, sizes, L, T, n, init=disk.INIT_SS, seed=4)
    path = str(tmp_path / "fit.ckpt")
    _, _, step = ck.fit_with_checkpoints(path, packed, sizes, L, T, n, 12, init=disk.INIT_SS,
                                         seed=4, stop_after=2)
    assert step == 24
    theta, loss, step = ck.fit_with_checkpoints(path, packed, sizes, L, T, n, 12,
                                                init=disk.INIT_SS, seed=4)
    torch.cuda.synchronize()
    assert step == n and torch.equal(theta, want) and torch.equal(loss, want_loss)
    assert ck.load_fit(path)[0]["step"] == n
    other = packed.clone()
    other[0] += 1.0
    with pytest.raises(ck.CheckpointError, match="another fit"):
        ck.fit_with_checkpoints(path, other, sizes, L, T, n, 12, init=disk.INIT_SS, seed=4)
    with pytest.raises(ck.CheckpointError, match="another fit"):
        ck.fit_with_checkpoints(path, packed, sizes, L, T, n + 1, 12, init=disk.INIT_SS, seed=4)


def test_a_corrupted_state_keeps_every_tap_inside_its_box(torch_cuda):
    """Offsets of a resumed state are clamped again, so a state with huge or
    NaN offsets still samples inside the canvases."""
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    tg = _batch()
    L, T = 2, 6
    packed, sizes = disk.pack_targets(tg)
    disk.fit_set_config(L, T, max(sizes), 512, 1)
    g = np.random.default_rng(5)
    st = g.standard_normal((len(tg), 3, L * T * 3)).astype(np.float32)
    st[:, 0, 0::3] = 1e30
    st[:, 0, 1::3] = np.nan
    st[:, 2] = np.abs(st[:, 2])
    state = torch.from_numpy(st).cuda()
    theta = torch.zeros((len(tg), L, T, 3), device="cuda")
    disk.fit_resume(packed, sizes, state, theta, 3, 4, 10)
    disk.device_status()  # raises if a bounded wait gave up
    th = theta.cpu().numpy()
    for b, t in enumerate(tg):
        s = max(1.0, (t.shape[0] - 1) / 2)
        assert np.abs(th[b, ..., :2]).max() <= s


def test_resume_rejects_bad_schedules(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    packed, sizes = disk.pack_targets(_batch())
    state = torch.zeros((4, 3, 2 * 4 * 3), device="cuda")
    theta = torch.zeros((4, 2, 4, 3), device="cuda")
    for step0, steps, total in ((5, 6, 10), (-1, 1, 10), (0, 1, 2_000_000)):
        with pytest.raises(disk.DiskError):
            disk.fit_resume(packed, sizes, state, theta, step0, steps, total)
    with pytest.raises(ValueError):
        disk.fit_resume(packed, sizes, state[:, :2].contiguous(), theta, 0, 1, 1)


def test_network_checkpoint_resumes_training_exactly(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    g = np.random.default_rng(8)
    x = torch.from_numpy(g.standard_normal((64, 256)).astype(np.float32)).cuda()
    y = torch.from_numpy(g.standard_normal((64, 24)).astype(np.float32)).cuda()
    net = disk.MLP(256, 64, 2, 24, seed=3)
    for _ in range(3):
        net.train_step(x, y, 1e-3)
    path = str(tmp_path / "net.ckpt")
    net.save(path)
    back = disk.MLP.load(path)
    assert back.shape == net.shape and back.step == 3
    for _ in range(2):
        la = net.train_step(x, y, 1e-3).clone()
        lb = back.train_step(x, y, 1e-3).clone()
        assert torch.equal(la, lb)
    torch.cuda.synchronize()
    assert torch.equal(net.params, back.params) and torch.equal(net.m, back.m)
    assert torch.equal(net.v, back.v) and back.step == 5
