"""Data-parallel step of the learned initializer on two gloo ranks (CPU):
the all-reduce average of the ranks' half-batch gradients -- here the FP64
oracle's, standing in for the GPU kernels -- equals the full-batch gradient,
and every rank ends with the same parameters as one full-batch step."""
import os
import socket

import numpy as np

from oracle import mlp
from paper_2512_04556_gb300 import dp

SHAPE = (16, 12, 2, 6)


class _OracleNet:
    """The MLP interface dp_train_step uses, computed by the FP64 oracle."""

    def __init__(self, params):
        import torch
        self.params = torch.from_numpy(params.copy())
        self.m = np.zeros_like(params)
        self.v = np.zeros_like(params)
        self.step = 0
        self.torch = torch

    def grad(self, x, target, stream=None):
        loss, g = mlp.loss_and_grad(self.params.numpy(), x.numpy(), target.numpy(), *SHAPE)
        return self.torch.tensor([loss]), self.torch.from_numpy(g)

    def apply(self, grad, lr, stream=None):
        self.step += 1
        p, self.m, self.v = mlp.adam(self.params.numpy(), self.m, self.v, grad.numpy(), self.step, lr)
        self.params = self.torch.from_numpy(p)


def _data():
    g = np.random.default_rng(5)
    params = g.normal(scale=0.3, size=mlp.param_count(*SHAPE))
    return params, g.random((24, 16)), g.normal(size=(24, 6))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    params, x, t = _data()
    net = _OracleNet(params)
    h = x.shape[0] // world
    sl = slice(rank * h, (rank + 1) * h)
    for _ in range(3):
        dp.dp_train_step(net, torch.from_numpy(x[sl]), torch.from_numpy(t[sl]), 1e-2, dist)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), net.params.numpy())
    dist.destroy_process_group()


def test_dp_two_ranks_equal_full_batch(tmp_path):
    import torch
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    params, x, t = _data()
    ref = _OracleNet(params)
    for _ in range(3):
        dp.dp_train_step(ref, torch.from_numpy(x), torch.from_numpy(t), 1e-2, None)
    for r in range(2):
        np.testing.assert_allclose(np.load(tmp_path / f"r{r}.npy"), ref.params.numpy(), rtol=1e-12,
                                   atol=1e-13)
