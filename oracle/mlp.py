"""FP64 oracle of the learned initializer -- test infrastructure only.

The learned initializer maps a dense target kernel to the L x T x 3 sparse
parameters of a complex: the target is area-resampled to side x side and
scaled to a maximum of 1, then a multilayer perceptron (ReLU hidden layers)
regresses the parameters (offsets in units of the target half-width,
weights raw).  The paper has no learned initializer; this follows the
project's own definition, written plainly with numpy matrix products.

Parameter layout (shared by name with the CUDA library, not by code): for
each layer i in order, W_i [n_in][n_out] row-major then b_i [n_out].
"""
from __future__ import annotations

import numpy as np


def area_weights(K: int, side: int) -> np.ndarray:
    """A [side][K]: A[j][i] = length of input pixel i ([i, i+1)) inside output
    cell j ([j K/side, (j+1) K/side)), divided by the cell length K/side, so
    each row sums to 1 (area averaging)."""
    A = np.zeros((side, K))
    s = K / side
    for j in range(side):
        lo, hi = j * s, (j + 1) * s
        for i in range(int(np.floor(lo)), min(K, int(np.ceil(hi)))):
            A[j, i] = max(0.0, min(hi, i + 1) - max(lo, i)) / s
    return A


def downsample(target: np.ndarray, side: int = 64) -> np.ndarray:
    """Area resampling to side x side, then scaled to a maximum of 1."""
    A = area_weights(target.shape[0], side)
    out = A @ np.asarray(target, np.float64) @ A.T
    m = out.max()
    return out / m if m > 0 else out


def layer_dims(n_in: int, hidden: int, depth: int, n_out: int):
    dims = [n_in] + [hidden] * depth + [n_out]
    return list(zip(dims[:-1], dims[1:]))


def param_count(n_in, hidden, depth, n_out) -> int:
    return sum(a * b + b for a, b in layer_dims(n_in, hidden, depth, n_out))


def unpack(params, n_in, hidden, depth, n_out):
    out, off = [], 0
    for a, b in layer_dims(n_in, hidden, depth, n_out):
        W = params[off:off + a * b].reshape(a, b)
        off += a * b
        bb = params[off:off + b]
        off += b
        out.append((W, bb))
    return out


def forward(params, x, n_in, hidden, depth, n_out):
    """Returns (y, activations): h_0 = x, h_i = relu(h_{i-1} W_i + b_i) for the
    hidden layers, y = h_depth W + b (no activation)."""
    layers = unpack(np.asarray(params, np.float64), n_in, hidden, depth, n_out)
    h = np.asarray(x, np.float64)
    acts = [h]
    for i, (W, b) in enumerate(layers):
        z = h @ W + b
        h = np.maximum(z, 0.0) if i < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grad(params, x, target, n_in, hidden, depth, n_out):
    """Mean squared error over the batch and outputs, and its gradient with
    respect to every parameter (same flat layout)."""
    y, acts = forward(params, x, n_in, hidden, depth, n_out)
    t = np.asarray(target, np.float64)
    n = y.size
    loss = float(((y - t) ** 2).sum() / n)
    layers = unpack(np.asarray(params, np.float64), n_in, hidden, depth, n_out)
    grads = []
    d = 2.0 * (y - t) / n
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        h_in = acts[i]
        grads.append((h_in.T @ d, d.sum(0)))
        if i > 0:
            d = (d @ W.T) * (acts[i] > 0)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam(params, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), step counted from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
