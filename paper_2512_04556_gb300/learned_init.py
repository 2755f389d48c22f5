"""Learned initializer for the fit (a project addition to Sec. 4.1-4.2).

Pipeline, every numeric step in the library's CUDA kernels:
1. pairs: the batched fitter (disk_fit, Eq. 6 radial init, Adam, 500 steps)
   turns seeded non-convex targets into fitted complexes theta*;
2. features: each target area-resampled to 64 x 64 and scaled to max 1;
   labels: theta* with offsets in units of the half-width s = max(1, (K-1)/2)
   and weights times T (both of order one);
3. training: MSE regression with Adam (disk_mlp_train_step);
4. use: the network's complex starts the fit; the fitted loss judges it --
   per target, the start with the lower loss (network or Eq. 6) is kept;
5. evaluation: on held-out targets, the Adam steps the refined fit needs to
   reach the loss the plain fitter (Eq. 6 start) reaches after its full run.

`python -m paper_2512_04556_gb300.learned_init` runs the full configuration
(50k training pairs, 2k held-out targets) and prints a JSON summary.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import disk
from . import workloads as wl

SIDE = 64


def _scales(sizes):
    return np.array([max(1.0, (k - 1) / 2) for k in sizes], dtype=np.float32)


def fit_pairs(targets, L, T, steps, batch=1024, init=disk.INIT_IR, seed=0):
    """Fitted complexes theta* [n, L, T, 3] (pixels, device) and final losses."""
    import torch
    thetas, losses = [], []
    for i in range(0, len(targets), batch):
        packed, sizes = disk.pack_targets(targets[i:i + batch])
        if i == 0:
            disk.fit_autotune(packed, sizes, L, T)  # launch configuration for this batch shape
        th, fl, _ = disk.fit(packed, sizes, L, T, steps, init=init, seed=seed)
        thetas.append(th)
        losses.append(fl)
    return torch.cat(thetas), torch.cat(losses)


def features(targets, batch=2048):
    """Area-resampled, max-scaled targets [n, SIDE*SIDE] (device)."""
    import torch
    out = []
    for i in range(0, len(targets), batch):
        packed, sizes = disk.pack_targets(targets[i:i + batch])
        out.append(disk.downsample_targets(packed, sizes, SIDE).reshape(len(sizes), -1))
    return torch.cat(out)


def to_labels(theta, sizes, T):
    """Pixels -> network units: offsets / s, weights * T."""
    import torch
    s = torch.from_numpy(_scales(sizes)).to(theta.device)[:, None, None]
    y = theta.clone()
    y[..., 0] /= s
    y[..., 1] /= s
    y[..., 2] *= T
    return y.reshape(theta.shape[0], -1)


def train(net, X, Y, epochs=30, batch=256, lr0=1e-3, lr1=1e-5, seed=0, log=None):
    """Adam on shuffled mini-batches, lr decayed geometrically lr0 -> lr1."""
    import torch
    n = X.shape[0]
    steps = epochs * max(1, n // batch)
    g = torch.Generator(device=X.device).manual_seed(seed)
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device=X.device, generator=g)
        for j in range(0, n - batch + 1, batch):
            idx = perm[j:j + batch]
            lr = lr0 * (lr1 / lr0) ** (k / max(1, steps - 1))
            loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr)
            k += 1
        if log is not None:
            log.append(float(loss.item()))
    return net


def network_start(net, targets, L, T, loss=disk.LOSS_MSE):
    """The network's complexes [n, L, T, 3] (pixels), each replaced by the
    Eq. 6 radial start where that has the lower fitted loss
    (disk_learned_init, every step on the device)."""
    packed, sizes = disk.pack_targets(targets)
    return disk.learned_init(net, packed, sizes, L, T, SIDE, loss=loss)


def iterations_to_reach(hist, ref):
    """First step index t at which the loss before step t is <= ref (steps + 1
    when never reached)."""
    ok = hist <= ref[:, None]
    first = np.where(ok.any(1), ok.argmax(1), hist.shape[1])
    return first


def evaluate(net, targets, L, T, steps=500):
    """Median iterations of the network-started fit to reach the plain
    fitter's final loss, and related figures."""
    packed, sizes = disk.pack_targets(targets)
    _, _, h_plain = disk.fit(packed, sizes, L, T, steps, init=disk.INIT_IR, loss_hist=True)
    th0, used = network_start(net, targets, L, T)
    _, _, h_net = disk.fit(packed, sizes, L, T, steps, init=disk.INIT_GIVEN, theta=th0,
                           loss_hist=True)
    hp, hn = h_plain.cpu().numpy(), h_net.cpu().numpy()
    it = iterations_to_reach(hn, hp[:, -1])
    med = float(np.median(it))
    return {"median_iterations": med, "plain_iterations": steps,
            "speedup": steps / max(med, 1.0),
            "reached_fraction": float((it <= steps).mean()),
            "network_start_used": float(used.float().mean().item()),
            "median_start_loss_ratio": float(np.median(hn[:, 0] / hp[:, 0])),
            "median_final_loss_ratio": float(np.median(hn[:, -1] / hp[:, -1])),
            "heldout": len(targets)}


def run(n_train=50000, n_heldout=2000, epochs=30, steps=500, kmin=33, kmax=129, hidden=512,
        depth=3, seed=0, return_net=False):
    """Full learned-initializer experiment; returns a summary dict (and the
    trained network with ``return_net``)."""
    import torch
    L, T = wl.C5["L"], wl.C5["T"]
    t0 = time.perf_counter()
    train_t = wl.shape_batch(n_train, kmin=kmin, kmax=kmax, first=0)
    held_t = wl.shape_batch(n_heldout, kmin=kmin, kmax=kmax, first=10_000_000)
    th, _ = fit_pairs(train_t, L, T, steps)
    sizes = [t.shape[0] for t in train_t]
    X = features(train_t)
    Y = to_labels(th, sizes, T)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    net = disk.MLP(SIDE * SIDE, hidden, depth, L * T * 3, seed=seed)
    log = []
    t1 = time.perf_counter()
    train(net, X, Y, epochs=epochs, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    res = evaluate(net, held_t, L, T, steps)
    res.update({"train_pairs": n_train, "epochs": epochs, "pair_generation_s": t_pairs,
                "training_s": t_train, "final_train_loss": log[-1] if log else None,
                "network": f"{SIDE * SIDE}-{'-'.join([str(hidden)] * depth)}-{L * T * 3}"})
    return (res, net) if return_net else res


if __name__ == "__main__":
    print(json.dumps(run()))
