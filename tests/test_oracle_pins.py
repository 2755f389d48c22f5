"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-worked
fixtures, textbook filters that special cases reduce to, brute-force dense
expansion, closed-form moments, central finite differences and the
dot-product adjoint identity.  A dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage, signal

import oracle
from paper_2512_04556_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_blocks(name):
    blocks, cur = [], None
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line:
            continue
        if line.startswith("#"):
            if cur:
                blocks.append(np.array(cur, dtype=np.float64))
            cur = []
            continue
        cur.append([float(v) for v in line.split()])
    if cur:
        blocks.append(np.array(cur, dtype=np.float64))
    return blocks


# ---------------------------------------------------------------- goldens

def test_golden_box_layer():
    """Hand-worked 2x2 box (one tap at (1/2, 1/2)) with clamp-to-edge."""
    *_, img, want = _read_blocks("layer_box_3x3.txt")
    got = oracle.layer(img[:, :, None], np.array([[0.5, 0.5, 1.0]]))[:, :, 0]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_golden_synth_two_layers():
    """Hand-worked impulse response of a two-layer complex (Eq. 10)."""
    *_, theta, want = _read_blocks("synth_two_layers.txt")
    got = oracle.synth(theta.reshape(2, 2, 3), 3)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_splitmix64_published_vector():
    """SplitMix64 from state 0: published first outputs."""
    assert oracle.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ---------------------------------------------------------------- special cases

def _img(H, W, C, seed):
    return np.random.default_rng(seed).random((H, W, C))


def test_integer_offset_is_pure_shift():
    img = _img(9, 11, 3, 1)
    for dx, dy in [(2, 0), (0, -3), (-1, 4), (5, 5)]:
        got = oracle.layer(img, np.array([[dx, dy, 1.0]]))
        v = np.clip(np.arange(9)[:, None] + dy, 0, 8)
        u = np.clip(np.arange(11)[None, :] + dx, 0, 10)
        np.testing.assert_allclose(got, img[v, u], rtol=0, atol=1e-15)


def test_half_offset_is_2x2_box():
    img = _img(8, 10, 2, 2)
    got = oracle.layer(img, np.array([[0.5, 0.5, 1.0]]))
    p = np.pad(img, ((0, 1), (0, 1), (0, 0)), mode="edge")
    want = 0.25 * (p[:-1, :-1] + p[:-1, 1:] + p[1:, :-1] + p[1:, 1:])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_four_half_taps_are_binomial_and_two_layers_five_tap():
    img = _img(16, 17, 1, 3)
    taps = np.array([[sx * 0.5, sy * 0.5, 0.25] for sx in (-1, 1) for sy in (-1, 1)])
    b3 = np.outer([1, 2, 1], [1, 2, 1]) / 16.0
    one = oracle.layer(img, taps)
    want1 = ndimage.correlate(img[:, :, 0], b3, mode="nearest")
    np.testing.assert_allclose(one[:, :, 0], want1, rtol=0, atol=1e-14)
    two = oracle.layer(one, taps)
    b5 = np.outer([1, 4, 6, 4, 1], [1, 4, 6, 4, 1]) / 256.0
    want2 = ndimage.correlate(img[:, :, 0], b5, mode="nearest")
    # cascaded clamps equal one clamp away from the border
    np.testing.assert_allclose(two[2:-2, 2:-2, 0], want2[2:-2, 2:-2], rtol=0, atol=1e-14)


# ---------------------------------------------------------------- (a) impulse = dense expansion

def _dense_stencil(taps):
    """Brute-force expansion of one layer into integer taps: correlation stencil
    D with out[x] = sum_m D[m] in[x + m]; returned with its half-width."""
    r = int(np.ceil(np.abs(taps[:, :2]).max())) + 1
    D = np.zeros((2 * r + 1, 2 * r + 1))
    for dx, dy, w in taps:
        fx, fy = math.floor(dx), math.floor(dy)
        ax, ay = dx - fx, dy - fy
        for ox, bx in ((0, 1 - ax), (1, ax)):
            for oy, by in ((0, 1 - ay), (1, ay)):
                D[r + fy + oy, r + fx + ox] += w * bx * by
    return D, r


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_a_impulse_equals_dense_expansion(seed):
    th = wl.complex_random(3, 5, 3.3, seed)
    D, r = _dense_stencil(th[0])
    for l in range(1, 3):
        Dl, rl = _dense_stencil(th[l])
        D = signal.convolve2d(D, Dl, mode="full")
        r += rl
    K = 2 * r + 1
    want = D[::-1, ::-1]                      # K_syn[c + m] = D[-m]
    got = oracle.synth(th, K)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    assert abs(got.sum() - np.prod(th[:, :, 2].sum(1))) < 1e-12


# ---------------------------------------------------------------- (b) linearity

def _sv_case(H, W, seed, dims=1):
    g = np.random.default_rng(100 + seed)
    if dims == 1:
        nodes = [1.0, 2.0, 4.0, 8.0]
        n_nodes = [4]
        th = wl.basis_random(nodes, 3, 5, spread=1.0, seed=seed).astype(np.float64)
        maps = g.uniform(0.5, 9.0, (1, H, W))
    else:
        n0, n1 = 3, 4
        nodes = list(np.linspace(1, 3, n0)) + list(np.linspace(0, 1, n1))
        n_nodes = [n0, n1]
        th = wl.basis_random(np.repeat(np.linspace(1, 3, n0), n1), 2, 4, spread=1.0,
                             seed=seed).astype(np.float64)
        maps = np.stack([g.uniform(0.8, 3.2, (H, W)), g.uniform(-0.1, 1.1, (H, W))])
    th[..., 2] /= th[..., 2].sum(-1, keepdims=True)   # exact unit sums in FP64
    return maps, n_nodes, np.array(nodes), th


@pytest.mark.parametrize("dims", [1, 2])
def test_b_linearity(dims):
    maps, nn, nv, th = _sv_case(13, 17, 4, dims)
    I, J = _img(13, 17, 3, 5), _img(13, 17, 3, 6)
    a, b = 0.7, -1.9
    lhs = oracle.sv_filter(a * I + b * J, maps, nn, nv, th)
    rhs = a * oracle.sv_filter(I, maps, nn, nv, th) + b * oracle.sv_filter(J, maps, nn, nv, th)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- (c) constants

@pytest.mark.parametrize("dims", [1, 2])
def test_c_constant_preserved(dims):
    maps, nn, nv, th = _sv_case(11, 14, 7, dims)
    assert np.allclose(th[..., 2].sum(-1), 1.0)
    out = oracle.sv_filter(np.full((11, 14, 3), 0.375), maps, nn, nv, th)
    np.testing.assert_allclose(out, 0.375, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- (d) node reproduction

def test_alpha_weights():
    nodes = [1.0, 2.0, 4.0, 8.0]
    assert oracle.locate(2.0, nodes) == (0, 1.0)
    assert oracle.locate(3.0, nodes) == (1, 0.5)
    assert oracle.locate(0.2, nodes) == (0, 0.0)
    assert oracle.locate(99.0, nodes) == (2, 1.0)
    assert oracle.locate(float("nan"), nodes) == (0, 0.0)
    np.testing.assert_allclose(oracle.alpha([6.0], [4], nodes), [0, 0, 0.5, 0.5])
    a = oracle.alpha([1.5, 0.25], [2, 3], [1.0, 2.0, 0.0, 0.5, 1.0])
    want = np.outer([0.5, 0.5], [0.5, 0.5, 0.0]).ravel()
    np.testing.assert_allclose(a, want)
    for k, p in enumerate(nodes):
        np.testing.assert_allclose(oracle.alpha([p], [4], nodes), np.eye(4)[k])


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_d_node_reproduction(k):
    maps, nn, nv, th = _sv_case(20, 22, 8, 1)
    img = _img(20, 22, 3, 9)
    out = oracle.sv_filter(img, np.full((1, 20, 22), nv[k]), nn, nv, th)
    # the cascade of the node's own complex, layer by layer (shift invariant)
    ref = img
    for l in range(th.shape[1]):
        ref = oracle.layer(ref, th[k, l])
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13)
    # and, away from the border, the brute-force dense composite
    D, r = _dense_stencil(th[k, 0])
    for l in range(1, th.shape[1]):
        Dl, rl = _dense_stencil(th[k, l])
        D = signal.convolve2d(D, Dl, mode="full")
        r += rl
    for c in range(3):
        want = ndimage.correlate(img[:, :, c], D, mode="nearest")
        np.testing.assert_allclose(out[r:-r, r:-r, c], want[r:-r, r:-r], rtol=0, atol=1e-12)


def test_sv_between_nodes_is_convex_blend_of_taps():
    """One layer, one tap per node: halfway between nodes the tap is the mean
    of the two node taps (Eq. 9 interpolates offsets and weights)."""
    nv = np.array([0.0, 1.0])
    th = np.zeros((2, 1, 1, 3))
    th[0, 0, 0] = [0.0, 0.0, 1.0]
    th[1, 0, 0] = [1.0, 0.0, 0.5]
    img = _img(6, 7, 1, 10)
    out = oracle.sv_filter(img, np.full((1, 6, 7), 0.5), [2], nv, th)
    want = oracle.layer(img, np.array([[0.5, 0.0, 0.75]]))
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- moments

def test_moment_invariant_of_impulse_response():
    """Normalised non-negative layers: the impulse response's mean is minus the
    sum of the layer means; its covariance is the sum of layer covariances,
    each tap contributing o o^T plus the bilinear tent variance f(1-f) per axis."""
    th = wl.complex_random(3, 6, 2.7, 21, nonneg=True)
    R = oracle.support_radius(th)
    K = 2 * R + 1
    Ks = oracle.synth(th, K)
    c = np.arange(K) - R
    yy, xx = np.meshgrid(c, c, indexing="ij")
    mx, my = (Ks * xx).sum(), (Ks * yy).sum()
    cxx = (Ks * (xx - mx) ** 2).sum()
    cyy = (Ks * (yy - my) ** 2).sum()
    cxy = (Ks * (xx - mx) * (yy - my)).sum()
    mu = np.zeros(2)
    cov = np.zeros((2, 2))
    for l in range(3):
        o, w = th[l, :, :2], th[l, :, 2]
        f = o - np.floor(o)
        m = (w[:, None] * o).sum(0)
        mu += m
        cov += (w[:, None, None] * (o[:, :, None] * o[:, None, :])).sum(0) - np.outer(m, m)
        cov += np.diag((w[:, None] * f * (1 - f)).sum(0))
    np.testing.assert_allclose([mx, my], -mu, atol=1e-12)
    np.testing.assert_allclose([[cxx, cxy], [cxy, cyy]], cov, atol=1e-11)


# ---------------------------------------------------------------- initialisation

def test_ir_init_ring_of_eq6():
    """Two-point target at (+-2, 0): per-axis variance (4 + 0)/2 = 2; with L=1
    the moment-matching step is sigma * sqrt(2) = 2."""
    tgt = np.zeros((5, 5))
    tgt[2, 0] = tgt[2, 4] = 0.5
    th = oracle.init_ir(tgt, 1, 7)
    ang = 2 * np.pi * np.arange(1, 8) / 7
    np.testing.assert_allclose(th[0, :, 0], 2 * np.cos(ang), atol=1e-14)
    np.testing.assert_allclose(th[0, :, 1], 2 * np.sin(ang), atol=1e-14)
    np.testing.assert_allclose(th[0, :, 2], 1 / 7)
    th4 = oracle.init_ir(tgt, 4, 7)
    dr = math.sqrt(2) * math.sqrt(12 / (4 * 5 * 9))
    np.testing.assert_allclose(np.hypot(th4[:, 0, 0], th4[:, 0, 1]), dr * np.arange(1, 5), atol=1e-13)


def test_ss_init_samples_the_support():
    tgt = wl.star(5, 14.0, 6.0, 0.3, 31)
    K, h, T = 31, 15, 16
    th, draws = oracle.init_ss(tgt, 4, T, seed=1234)
    q = -th[0, :, :2]
    nz = tgt > 0
    assert np.all(q == np.round(q))
    for x, y in q:
        assert nz[int(y) + h, int(x) + h]
    S = nz.sum()
    r2 = S / (T * np.pi)
    d2 = ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1) + np.eye(T) * 1e9
    # samples are separated by at least the (possibly shrunk) radius
    n_shrinks = 0
    while d2.min() < r2 * 0.81 ** n_shrinks - 1e-9:
        n_shrinks += 1
    assert n_shrinks <= 3
    assert draws >= T
    np.testing.assert_allclose(th[0, :, 2], 1 / T)
    # deterministic under the seed
    th2, _ = oracle.init_ss(tgt, 4, T, seed=1234)
    np.testing.assert_array_equal(th, th2)


# ---------------------------------------------------------------- gradients

def _away_from_integers(th, margin=0.05):
    o = th[..., :2]
    f = o - np.floor(o)
    f = np.clip(f, margin, 1 - margin)
    th = th.copy()
    th[..., :2] = np.floor(o) + f
    return th


@pytest.mark.parametrize("loss,eps", [(oracle.LOSS_MSE, 0.0), (oracle.LOSS_CHARB, 1e-3)])
def test_fit_gradient_matches_central_differences(loss, eps):
    tgt = wl.disk(4.5, 11)
    th = _away_from_integers(wl.complex_random(2, 4, 2.2, 5))
    v, g = oracle.fit_loss(th, tgt, loss, eps, grad=True)
    h = 1e-6
    fd = np.zeros_like(th)
    for idx in np.ndindex(*th.shape):
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        fd[idx] = (oracle.fit_loss(tp, tgt, loss, eps) - oracle.fit_loss(tm, tgt, loss, eps)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9 * np.abs(fd).max())


def test_mse_is_plane_sum_over_K2():
    tgt = wl.disk(3.0, 9)
    th = wl.complex_random(2, 3, 1.5, 6)
    R = oracle.support_radius(th) + 4
    Ks = oracle.synth_canvas(th, R)
    pad = np.zeros_like(Ks)
    pad[R - 4:R + 5, R - 4:R + 5] = tgt
    assert abs(oracle.fit_loss(th, tgt) - ((Ks - pad) ** 2).sum() / 81) < 1e-15


@pytest.mark.parametrize("dims", [1, 2])
def test_sv_adjoint_dot_product(dims):
    """<F x, y> = <x, F^T y> for the spatially varying filter with clamp."""
    maps, nn, nv, th = _sv_case(12, 15, 11, dims)
    x, y = _img(12, 15, 3, 12) - 0.5, _img(12, 15, 3, 13) - 0.5
    lhs = (oracle.sv_filter(x, maps, nn, nv, th) * y).sum()
    rhs = (x * oracle.sv_filter_adjoint(y, maps, nn, nv, th)).sum()
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_uniform_adjoint_zero_boundary_is_negated_offsets():
    """Tent symmetry: on a zero-bounded canvas the transpose of a shift-invariant
    layer is the same layer with every offset negated."""
    th = wl.complex_random(1, 5, 2.6, 14)[0]
    x = _img(14, 14, 1, 15)
    y = _img(14, 14, 1, 16)
    neg = th.copy()
    neg[:, :2] *= -1
    lhs = (oracle.layer(x, th, "zero") * y).sum()
    rhs = (x * oracle.layer(y, neg, "zero")).sum()
    assert abs(lhs - rhs) < 1e-12


# ---------------------------------------------------------------- fitting

def test_fit_decreases_and_init_ordering():
    """The fit lowers the loss, and the paper's initialisations beat random
    offsets on a non-convex target (Sec. 5.4 ordering: SS, IR ahead of Rand)."""
    tgt = wl.star(5, 10.0, 4.0, 0.2, 23)
    res = {}
    for name, init in [("ir", oracle.INIT_IR), ("ss", oracle.INIT_SS), ("rand", oracle.INIT_RAND)]:
        finals = []
        for seed in range(3):
            _, hist = oracle.fit(tgt, 2, 8, 150, init=init, seed=seed)
            assert hist[-1] < hist[0]
            finals.append(hist[-1])
        res[name] = np.median(finals)
    assert res["ss"] < res["rand"]
    assert res["ir"] < res["rand"]


# ---------------------------------------------------------------- dense SV reference

def test_dense_sv_delta_kernels_shift_and_blend():
    img = _img(9, 10, 3, 17)
    lut = np.zeros((2, 3, 3))
    lut[0, 1, 1] = 1.0                       # identity
    lut[1, 1, 2] = 1.0                       # m = (+1, 0): out[x] = I[x - (1, 0)]
    out0 = oracle.dense_sv(img, np.full((1, 9, 10), 0.0), [2], [0.0, 1.0], lut)
    np.testing.assert_allclose(out0, img, atol=1e-15)
    out1 = oracle.dense_sv(img, np.full((1, 9, 10), 1.0), [2], [0.0, 1.0], lut)
    u = np.clip(np.arange(10) - 1, 0, 9)
    np.testing.assert_allclose(out1, img[:, u], atol=1e-15)
    outh = oracle.dense_sv(img, np.full((1, 9, 10), 0.25), [2], [0.0, 1.0], lut)
    np.testing.assert_allclose(outh, 0.75 * img + 0.25 * img[:, u], atol=1e-15)


def test_fitted_complex_reproduces_dense_convolution():
    """A complex whose impulse response equals K makes the filter equal true
    convolution with K (away from the border)."""
    th = wl.complex_random(2, 4, 2.0, 18)
    R = oracle.support_radius(th)
    Ks = oracle.synth(th, 2 * R + 1)
    img = _img(24, 25, 1, 19)
    out = oracle.sv_filter(img, np.zeros((1, 24, 25)), [1], [0.0], th[None])
    dense = oracle.dense_sv(img, np.zeros((1, 24, 25)), [1], [0.0], Ks[None])
    np.testing.assert_allclose(out[R:-R, R:-R], dense[R:-R, R:-R], atol=1e-13)


@pytest.mark.parametrize("dims", [1, 2])
def test_sv_theta_gradient_matches_central_differences(dims):
    """d<g, F(img)>/d theta of the spatially varying cascade against central
    differences of the oracle's own forward (offsets kept off integers)."""
    H, W = 9, 11
    maps, nn, nv, th = _sv_case(H, W, 31, dims)
    th = _away_from_integers(th, 0.1)
    g = np.random.default_rng(32)
    img = g.random((H, W, 2))
    go = g.standard_normal((H, W, 2))
    got = oracle.sv_filter_grad_theta(img, go, maps, nn, nv, th)
    h = 1e-6
    fd = np.zeros_like(th)
    for idx in np.ndindex(*th.shape):
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        fd[idx] = ((oracle.sv_filter(img, maps, nn, nv, tp) - oracle.sv_filter(img, maps, nn, nv, tm)) * go).sum() / (2 * h)
    np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-8 * np.abs(fd).max())
