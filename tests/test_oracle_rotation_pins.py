"""Pins of the oracle's rotated spatially varying filter (per-pixel rotation
of every blended tap offset, the runtime form of the rotational and radial
blur effects of Sec. 5.3), against facts fixed by geometry:

* a zero angle is the plain filter;
* a quarter turn of every offset equals filtering the image turned by a
  quarter turn (maps turned with it) and turning the result back: the pixel
  grid, clamp-to-edge and bilinear sampling are all invariant under it;
* a half turn is the same with a half turn of the image;
* a ring of N equally weighted, equally spaced taps is unchanged by a turn of
  2 pi / N (the tap set maps onto itself);
* for one layer, each pixel's output is the shift-invariant layer with that
  pixel's rotated taps (a transposed or shifted angle map fails).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl


def _case(H=23, W=19, dims=1, L=2, T=5, seed=0):
    g = np.random.default_rng(seed)
    img = g.random((H, W, 3))
    if dims == 1:
        nn, nv = [3], np.array([1.0, 2.0, 4.0])
        maps = g.uniform(0.5, 4.5, (1, H, W))
    else:
        nn, nv = [2, 3], np.array([0.0, 1.0, 0.0, 0.5, 1.0])
        maps = np.stack([g.uniform(0, 1, (H, W)), g.uniform(0, 1, (H, W))])
    B = int(np.prod(nn))
    th = np.stack([wl.complex_random(L, T, 3.3, seed + 10 + k) for k in range(B)])
    return img, maps, nn, nv, th


@pytest.mark.parametrize("dims", [1, 2])
def test_zero_angle_is_plain_filter(dims):
    img, maps, nn, nv, th = _case(dims=dims)
    a = oracle.sv_filter_rotated(img, maps, np.zeros(img.shape[:2]), nn, nv, th)
    b = oracle.sv_filter(img, maps, nn, nv, th)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dims", [1, 2])
def test_quarter_turn_conjugates_rot90(dims):
    """(dx, dy) -> (-dy, dx): out = rot90^-1(F(rot90(img), rot90(maps)))."""
    img, maps, nn, nv, th = _case(dims=dims, seed=3)
    H, W = img.shape[:2]
    got = oracle.sv_filter_rotated(img, maps, np.full((H, W), math.pi / 2), nn, nv, th)
    r_img = np.ascontiguousarray(np.rot90(img, 1, axes=(0, 1)))
    r_maps = np.ascontiguousarray(np.rot90(maps, 1, axes=(1, 2)))
    want = np.rot90(oracle.sv_filter(r_img, r_maps, nn, nv, th), -1, axes=(0, 1))
    assert np.abs(got - want).max() <= 1e-12
    # the opposite turn is a different filter
    other = np.rot90(oracle.sv_filter(np.ascontiguousarray(np.rot90(img, -1, axes=(0, 1))),
                                      np.ascontiguousarray(np.rot90(maps, -1, axes=(1, 2))),
                                      nn, nv, th), 1, axes=(0, 1))
    assert np.abs(got - other).max() > 1e-3


def test_half_turn_conjugates_rot180():
    img, maps, nn, nv, th = _case(seed=5)
    H, W = img.shape[:2]
    got = oracle.sv_filter_rotated(img, maps, np.full((H, W), math.pi), nn, nv, th)
    want = oracle.sv_filter(img[::-1, ::-1].copy(), maps[:, ::-1, ::-1].copy(), nn, nv, th)[::-1, ::-1]
    assert np.abs(got - want).max() <= 1e-12


@pytest.mark.parametrize("N", [5, 8])
def test_symmetric_ring_invariant_under_its_turn(N):
    H, W = 21, 17
    img = np.random.default_rng(7).random((H, W, 3))
    r = 3.7
    ang = 0.3 + 2 * math.pi * np.arange(N) / N
    th = np.zeros((1, 1, N, 3))
    th[0, 0, :, 0], th[0, 0, :, 1], th[0, 0, :, 2] = r * np.cos(ang), r * np.sin(ang), 1.0 / N
    maps = np.zeros((1, H, W))
    a = oracle.sv_filter_rotated(img, maps, np.full((H, W), 2 * math.pi / N), [1], [0.0], th)
    b = oracle.sv_filter(img, maps, [1], [0.0], th)
    assert np.abs(a - b).max() <= 1e-12
    c = oracle.sv_filter_rotated(img, maps, np.full((H, W), math.pi / N), [1], [0.0], th)
    assert np.abs(c - b).max() > 1e-3


def test_single_layer_per_pixel_definition():
    img, maps, nn, nv, th = _case(H=9, W=11, L=1, T=4, seed=9)
    H, W = img.shape[:2]
    angle = np.random.default_rng(1).uniform(-4, 4, (H, W))
    got = oracle.sv_filter_rotated(img, maps, angle, nn, nv, th)
    for v in range(H):
        for u in range(W):
            al = oracle.alpha([maps[0, v, u]], nn, nv)
            taps = np.tensordot(al, th, axes=(0, 0))[0]          # [T][3] at this pixel
            c, s = math.cos(angle[v, u]), math.sin(angle[v, u])
            rt = taps.copy()
            rt[:, 0] = taps[:, 0] * c - taps[:, 1] * s
            rt[:, 1] = taps[:, 0] * s + taps[:, 1] * c
            want = oracle.layer(img, rt)[v, u]
            assert np.abs(got[v, u] - want).max() <= 1e-12


def test_non_finite_angle_acts_as_zero():
    img, maps, nn, nv, th = _case(seed=11)
    H, W = img.shape[:2]
    angle = np.full((H, W), 0.7)
    angle[3, 4], angle[10, 2] = np.nan, np.inf
    got = oracle.sv_filter_rotated(img, maps, angle, nn, nv, th)
    zero = angle.copy()
    zero[3, 4] = zero[10, 2] = 0.0
    np.testing.assert_array_equal(got, oracle.sv_filter_rotated(img, maps, zero, nn, nv, th))
    assert np.isfinite(got).all()
