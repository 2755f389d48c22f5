"""Data-parallel training step of the learned initializer's network.

Each rank computes the loss and gradient of its own batch with the
hand-written backward pass (`MLP.grad`), the ranks average the gradients with
one all-reduce (torch.distributed: NCCL on GPUs, gloo on CPUs), and every
rank applies the same Adam update (`MLP.apply`), so the parameters stay
identical on all ranks.  With equal local batches this is the step on the
union of the batches, because the loss is a mean over the batch.
"""
from __future__ import annotations


def average_gradient(grad, dist=None):
    """All-reduce (sum) the gradient in place and divide by the world size;
    unchanged without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return grad
    dist.all_reduce(grad)
    grad /= dist.get_world_size()
    return grad


def dp_train_step(net, x, target, lr: float, dist=None, stream=None):
    """One data-parallel step; returns this rank's loss (device tensor)."""
    loss, g = net.grad(x, target, stream=stream)
    average_gradient(g, dist)
    net.apply(g, lr, stream=stream)
    return loss
