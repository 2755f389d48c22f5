"""Pins for the oracle's fitter (Eq. 4 with Adam and the Sec. 5.1 schedule)
and its random start, against facts that do not come from the oracle.

* Adam (Kingma & Ba 2015): with bias correction, the first update of every
  coordinate is lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps; and
  under a constant gradient every update is lr_t * sign(g), whatever t.
* Sec. 5.1: the learning rate falls linearly from lr0 at the first step to
  lr1 at the last, so step t of n uses lr0 + (lr1 - lr0) t / (n - 1).
* The canvas bound: offsets stay within one target half-width s per axis,
  from the start and after every step.
* The random start draws offsets uniform in [-s/L, s/L] per axis from the
  published SplitMix64 stream (Steele, Lea & Flood 2014), dx then dy per tap.

Each construction makes one of these checkable by hand: a plausible slip in
the fitter (a dropped bias correction, an off-by-one schedule, a missing
clamp) changes the numbers these tests read by far more than their
tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

LR0, LR1 = 1e-3, 1e-4


def _away_from_integers(th, margin=0.05):
    o = th[..., :2]
    f = np.clip(o - np.floor(o), margin, 1 - margin)
    th = th.copy()
    th[..., :2] = np.floor(o) + f
    return th


@pytest.mark.parametrize("loss,eps", [(oracle.LOSS_MSE, 0.0), (oracle.LOSS_CHARB, 1e-3)])
def test_first_adam_step_is_lr0_times_sign_of_gradient(loss, eps):
    """One step from a given start moves each weight by -lr0 sign(g) and each
    offset by -s lr0 sign(g) (offsets are stepped in half-width units)."""
    K = 11
    s = (K - 1) / 2
    tgt = wl.star(5, 4.5, 2.0, 0.3, K)
    th0 = _away_from_integers(wl.complex_random(2, 4, 1.8, 31))
    assert np.abs(th0[..., :2]).max() < s
    _, g = oracle.fit_loss(th0, tgt, loss, eps, grad=True)
    th1, _ = oracle.fit(tgt, 2, 4, 1, LR0, LR1, init=oracle.INIT_GIVEN, loss=loss, eps=eps,
                        theta0=th0)
    # gradient in the optimiser's own units: offsets per half-width
    gq = g.copy()
    gq[..., :2] *= s
    step = th1 - th0
    step[..., :2] /= s
    big = np.abs(gq) > 1e-4
    assert big.sum() >= 0.8 * big.size
    np.testing.assert_allclose(step[big], -LR0 * np.sign(gq[big]), rtol=2e-4, atol=0)


def _clamped_corner_case(C):
    """K = 5 (s = 2), one layer of one tap, target -C everywhere in its box.
    The tap starts beyond the canvas bound at (4, 4) and is clamped to (2, 2),
    where its response sits on the box's corner pixel.  Moving it outward
    moves response off the box (where the loss gradient is zero), so the
    offset gradient points outward and the clamp holds it at (2, 2).  The
    weight's gradient is 2 (w + C) / 25: positive and, for C >> 1, constant
    to ~1e-6 over a few steps, so Adam steps the weight by -lr_t exactly."""
    K = 5
    tgt = -C * np.ones((K, K))
    th0 = np.array([[[4.0, 4.0, 0.5]]])
    return K, tgt, th0


@pytest.mark.parametrize("steps", [1, 2, 3, 5])
def test_schedule_and_clamp_under_a_constant_gradient(steps):
    C = 1e3
    K, tgt, th0 = _clamped_corner_case(C)
    th, hist = oracle.fit(tgt, 1, 1, steps, LR0, LR1, init=oracle.INIT_GIVEN,
                          loss=oracle.LOSS_MSE, theta0=th0)
    # offsets held at the bound s = 2 from the start and after every step
    assert th[0, 0, 0] == 2.0 and th[0, 0, 1] == 2.0
    # the loss with the tap on the corner is ((w + C)^2 + 24 C^2) / 25, so
    # every logged loss gives back the weight it was taken at
    w = np.sqrt(25.0 * hist - 24.0 * C * C) - C
    assert abs(w[0] - 0.5) < 1e-8
    assert abs(w[-1] - th[0, 0, 2]) < 1e-8
    lr = [LR0] if steps == 1 else [LR0 + (LR1 - LR0) * t / (steps - 1) for t in range(steps)]
    np.testing.assert_allclose(w[:-1] - w[1:], lr, rtol=0, atol=1e-8)
    assert abs(th[0, 0, 2] - (0.5 - sum(lr))) < 1e-8


def test_clamp_after_a_step_that_would_cross_it():
    """A tap a quarter step inside the bound, pulled outward by the gradient,
    ends on the bound instead of crossing it.  Target: -C in the 5 x 5 box
    except +C on the corner pixel; the tap's response sits almost wholly on
    that corner, so moving it further out lowers the loss."""
    C = 1e3
    K = 5
    tgt = -C * np.ones((K, K))
    tgt[0, 0] = C
    th0 = np.array([[[2.0 - 0.25 * LR0 * 2.0, 2.0 - 0.25 * LR0 * 2.0, 0.5]]])
    _, g = oracle.fit_loss(th0, tgt, grad=True)
    assert g[0, 0, 0] < 0 and g[0, 0, 1] < 0  # outward
    th, _ = oracle.fit(tgt, 1, 1, 1, LR0, LR1, init=oracle.INIT_GIVEN,
                       loss=oracle.LOSS_MSE, theta0=th0)
    assert th[0, 0, 0] == 2.0 and th[0, 0, 1] == 2.0


def test_offsets_beyond_the_bound_are_clamped_before_the_first_loss():
    """With zero steps the fit returns the given start clamped to the bound, and
    the one logged loss is that of the clamped start."""
    C = 1e3
    K, tgt, th0 = _clamped_corner_case(C)
    th, hist = oracle.fit(tgt, 1, 1, 0, LR0, LR1, init=oracle.INIT_GIVEN,
                          loss=oracle.LOSS_MSE, theta0=th0)
    np.testing.assert_array_equal(th, [[[2.0, 2.0, 0.5]]])
    assert abs(hist[0] - ((0.5 + C) ** 2 + 24 * C * C) / 25) < 1e-9 * C * C


def test_random_start_from_published_splitmix64_outputs():
    """Seed 0: the first three published outputs give dx, dy of tap 0 and dx of
    tap 1 through u = (x >> 11) / 2^53 and o = (2u - 1) s / L."""
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = [(x >> 11) / 2.0 ** 53 for x in published]
    K, L, T = 13, 2, 3
    s = (K - 1) / 2 / L
    th = oracle.init_rand(K, L, T, seed=0)
    want = [(2 * v - 1) * s for v in u]
    got = [th[0, 0, 0], th[0, 0, 1], th[0, 1, 0]]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    assert np.abs(th[..., :2]).max() <= s
    np.testing.assert_array_equal(th[..., 2], np.full((L, T), 1.0 / T))
    # a different seed is a different stream
    assert not np.array_equal(th, oracle.init_rand(K, L, T, seed=1))
