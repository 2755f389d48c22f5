"""Pins for the FP64 learned-initializer oracle (numpy): central differences,
a hand-derived forward case, the first Adam step, and exact special cases of
area resampling."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_central_differences():
    shape = (6, 5, 2, 3)
    g = np.random.default_rng(0)
    p = g.normal(0, 0.5, mlp.param_count(*shape))
    x = g.normal(0, 1, (4, 6))
    t = g.normal(0, 1, (4, 3))
    _, grad = mlp.loss_and_grad(p, x, t, *shape)
    h = 1e-6
    fd = np.zeros_like(p)
    for i in range(p.size):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd[i] = (mlp.loss_and_grad(pp, x, t, *shape)[0] - mlp.loss_and_grad(pm, x, t, *shape)[0]) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-5, atol=1e-9)


def test_forward_identity_and_relu_case():
    """W1 = I, b1 = 0 (ReLU passes positives, zeroes negatives), W2 = 2 I, b2 = 1:
    y = 2 relu(x) + 1, derived by hand."""
    p = np.concatenate([np.eye(3).ravel(), np.zeros(3), (2 * np.eye(3)).ravel(), np.ones(3)])
    x = np.array([[0.5, -1.0, 2.0]])
    y, _ = mlp.forward(p, x, 3, 3, 1, 3)
    np.testing.assert_allclose(y, [[2.0, 1.0, 5.0]])


def test_first_adam_step_moves_by_lr_times_sign():
    g = np.array([3.0, -0.2, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-4)


@pytest.mark.parametrize("K", [64, 128, 32])
def test_area_resampling_special_cases(K):
    g = np.random.default_rng(K)
    t = g.random((K, K))
    out = mlp.downsample(t, 64) * (mlp.area_weights(K, 64) @ t @ mlp.area_weights(K, 64).T).max()
    if K == 64:
        np.testing.assert_allclose(out, t, atol=1e-14)
    elif K == 128:
        box = 0.25 * (t[0::2, 0::2] + t[1::2, 0::2] + t[0::2, 1::2] + t[1::2, 1::2])
        np.testing.assert_allclose(out, box, atol=1e-14)
    else:
        np.testing.assert_allclose(out, np.kron(t, np.ones((2, 2))), atol=1e-14)
    # area averaging preserves the integral: sum(out) * (K/64)^2 = sum(t)
    assert abs(out.sum() * (K / 64) ** 2 - t.sum()) < 1e-9
    np.testing.assert_allclose(mlp.downsample(np.full((K, K), 0.3), 64), 1.0)
