"""Seeded synthetic inputs for the DISK workloads.

This module holds only input recipes (images, parameter maps, random bases,
dense target kernels); none of the filtering, interpolation or fitting
arithmetic lives here.  Both the CUDA path and the FP64 oracle consume the
arrays it returns, so the two see identical bytes.

Seeds (numpy PCG64): 0 images, 1 maps, 2 bases, 3 target shapes; train and
held-out target sets use disjoint seed ranges.

The paper's own inputs (five photographs, its kernel suite of silhouettes and
optical PSFs) are not available; these recipes stand in for them with the
shapes, sizes and value ranges of the paper's workloads (Sec. 5.1, Sec. 5.3).
"""
from __future__ import annotations

import math

import numpy as np

SEED_IMAGE, SEED_MAP, SEED_BASIS, SEED_SHAPE = 0, 1, 2, 3


def rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, *stream]))


# --------------------------------------------------------------------------
# Images
# --------------------------------------------------------------------------

def image_uniform(H: int, W: int, C: int = 3, seed: int = SEED_IMAGE) -> np.ndarray:
    """H x W x C float32, uniform in [0, 1)."""
    return rng(seed).random((H, W, C), dtype=np.float32)


def image_rects(H: int, W: int, C: int = 3, seed: int = SEED_IMAGE,
                n_rects: int | None = None, noise: float = 0.1) -> np.ndarray:
    """Random axis-aligned rectangles of uniform colour over a grey background,
    plus uniform noise of amplitude ``noise``; float32 in [0, 1]."""
    g = rng(seed, 1)
    img = np.full((H, W, C), 0.5, dtype=np.float32)
    if n_rects is None:
        n_rects = max(8, (H * W) // 20000)
    for _ in range(n_rects):
        h = int(g.integers(4, max(5, H // 4)))
        w = int(g.integers(4, max(5, W // 4)))
        y0 = int(g.integers(0, max(1, H - h)))
        x0 = int(g.integers(0, max(1, W - w)))
        img[y0:y0 + h, x0:x0 + w, :] = g.random(C, dtype=np.float32)
    img = (1.0 - noise) * img + noise * g.random((H, W, C), dtype=np.float32)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def to_fp16(img: np.ndarray) -> np.ndarray:
    """Round to IEEE half (round to nearest even), the storage type of the 4K
    workload."""
    return img.astype(np.float16)


# --------------------------------------------------------------------------
# Parameter maps
# --------------------------------------------------------------------------

def smooth_field(H: int, W: int, sigma: float, seed: int = SEED_MAP, stream: int = 0) -> np.ndarray:
    """White noise smoothed with a Gaussian of ``sigma`` px (reflect border),
    min-max normalised to [0, 1]; float64.  For large sigma the noise is drawn
    on a grid coarsened by sigma/4 and smoothed there, then resampled
    bilinearly, which keeps the generator fast at 4K."""
    from scipy import ndimage
    g = rng(seed, 100 + stream)
    if sigma <= 16 or H * W <= 512 * 512:
        f = ndimage.gaussian_filter(g.standard_normal((H, W)), sigma, mode="reflect")
    else:
        step = sigma / 4.0
        h = int(math.ceil(H / step)) + 2
        w = int(math.ceil(W / step)) + 2
        coarse = ndimage.gaussian_filter(g.standard_normal((h, w)), 4.0, mode="reflect")
        ys = np.arange(H) / step + 0.5
        xs = np.arange(W) / step + 0.5
        yy, xx = np.meshgrid(ys, xs, indexing="ij")
        f = ndimage.map_coordinates(coarse, [yy, xx], order=1, mode="nearest")
    lo, hi = f.min(), f.max()
    return (f - lo) / max(hi - lo, 1e-30)


def param_map(H: int, W: int, lo: float, hi: float, sigma: float,
              seed: int = SEED_MAP, stream: int = 0) -> np.ndarray:
    """Smooth random per-pixel parameter map in [lo, hi], float32."""
    return (lo + (hi - lo) * smooth_field(H, W, sigma, seed, stream)).astype(np.float32)


# --------------------------------------------------------------------------
# Random complexes and bases (theta [B][L][T][3] = dx, dy, w in pixels)
# --------------------------------------------------------------------------

def basis_random(node_vals, L: int, T: int, spread: float = 3.0,
                 seed: int = SEED_BASIS) -> np.ndarray:
    """One complex per node value s: offsets uniform in [-spread*s, spread*s]
    px per axis, each layer's weights Dirichlet(1) (they sum to 1)."""
    g = rng(seed, 7)
    B = len(node_vals)
    th = np.zeros((B, L, T, 3), dtype=np.float32)
    for k, s in enumerate(node_vals):
        th[k, :, :, 0:2] = g.uniform(-spread * s, spread * s, size=(L, T, 2))
        th[k, :, :, 2] = g.dirichlet(np.ones(T), size=L)
    return th


def complex_random(L: int, T: int, reach: float, seed: int, nonneg: bool = False) -> np.ndarray:
    """A single complex [L][T][3] with offsets uniform in [-reach, reach] and
    weights ~ N(1/T, 0.5/T) (or Dirichlet(1) when ``nonneg``)."""
    g = rng(seed, 11)
    th = np.zeros((L, T, 3), dtype=np.float64)
    th[:, :, 0:2] = g.uniform(-reach, reach, size=(L, T, 2))
    if nonneg:
        th[:, :, 2] = g.dirichlet(np.ones(T), size=L)
    else:
        th[:, :, 2] = g.normal(1.0 / T, 0.5 / T, size=(L, T))
    return th


# --------------------------------------------------------------------------
# Dense target kernels, rasterised with 4 x 4 supersampled area coverage and
# normalised to unit sum; odd size K, centre at index (K-1)/2.
# --------------------------------------------------------------------------

_SS = (np.arange(4) - 1.5) / 4.0


def _axis(K: int) -> np.ndarray:
    """The 4K supersample coordinates along one axis."""
    h = (K - 1) / 2.0
    c = np.arange(K) - h
    return (c[:, None] + _SS[None, :]).reshape(-1)


def _grid(K: int):
    """(xx, yy) as a row [1, 4K] and a column [4K, 1] that broadcast to the
    supersample grid: every grid expression below is evaluated per element
    exactly as on full arrays, without materialising them."""
    s = _axis(K)
    return s[None, :], s[:, None]


def _coverage(inside: np.ndarray, K: int) -> np.ndarray:
    # the mean of each pixel's 16 samples: an integer count / 16, exact
    cov = inside.reshape(K, 4, K, 4).sum(axis=(1, 3), dtype=np.int32) / 16.0
    s = cov.sum()
    if s <= 0:
        cov = np.zeros((K, K))
        cov[(K - 1) // 2, (K - 1) // 2] = 1.0
        return cov
    return cov / s


def kernel_size_for(radius: float) -> int:
    return 2 * int(math.ceil(radius)) + 1


def disk(radius: float, K: int | None = None) -> np.ndarray:
    K = K or kernel_size_for(radius)
    xx, yy = _grid(K)
    return _coverage(xx * xx + yy * yy <= radius * radius, K)


def ellipse(radius: float, ratio: float, angle: float, K: int | None = None) -> np.ndarray:
    """Semi-major ``radius``, semi-minor radius/ratio, major axis at ``angle``."""
    K = K or kernel_size_for(radius)
    xx, yy = _grid(K)
    c, s = math.cos(angle), math.sin(angle)
    a, b = radius, radius / ratio
    xr = c * xx + s * yy
    yr = -s * xx + c * yy
    return _coverage((xr / a) ** 2 + (yr / b) ** 2 <= 1.0, K)


def gaussian(sigma: float, K: int | None = None) -> np.ndarray:
    """Isotropic Gaussian of standard deviation sigma px, 4 x 4 supersampled
    over each pixel, unit sum, odd size 2 ceil(3 sigma) + 1."""
    K = K or 2 * int(math.ceil(3.0 * sigma)) + 1
    xx, yy = _grid(K)
    g = np.exp(-(xx * xx + yy * yy) / (2.0 * sigma * sigma))  # [4K, 4K] by broadcasting
    g = g.reshape(K, 4, K, 4).mean(axis=(1, 3))
    return g / g.sum()


def gaussian_lut(sigmas, K: int) -> np.ndarray:
    return np.stack([gaussian(s, K) for s in sigmas]).astype(np.float32)


def tilt_shift_map(H: int, W: int, lo: float, hi: float, focus: float = 0.55,
                   band: float = 0.05, ramp: float = 0.4, seed: int = SEED_MAP) -> np.ndarray:
    """Tilt-shift blur map: sharp (lo) inside a horizontal focus band around
    row focus*H, rising linearly to hi over ramp*H, plus a faint smooth
    perturbation; float32 [H][W]."""
    y = np.arange(H)[:, None] / H
    t = np.clip((np.abs(y - focus) - band) / ramp, 0.0, 1.0)
    pert = 0.05 * (smooth_field(H, W, 96.0, seed, stream=7) - 0.5)
    return np.clip(lo + (hi - lo) * (t + pert), lo, hi).astype(np.float32)


def ellipse_params(radius: float, u: float) -> tuple[float, float, float]:
    """The 2-D kernel-space axis u in [0,1] couples anisotropy ratio 1+3u with
    rotation pi*u."""
    return radius, 1.0 + 3.0 * u, math.pi * u


def line(length: float, K: int | None = None, angle: float = 0.0, width: float = 1.0) -> np.ndarray:
    """Motion-blur segment: |along| <= length / 2, |across| <= width / 2, the
    long axis at ``angle`` (x right, y down); size 2 ceil(length / 2) + 1."""
    K = K or kernel_size_for(length / 2.0)
    xx, yy = _grid(K)
    c, s = math.cos(angle), math.sin(angle)
    along = c * xx + s * yy
    across = -s * xx + c * yy
    return _coverage((np.abs(along) <= length / 2.0) & (np.abs(across) <= width / 2.0), K)


def cat_eye(radius: float, K: int | None = None, angle: float = 0.0) -> np.ndarray:
    """Rotational-bokeh kernel: an ellipse of semi-major radius and
    semi-minor radius / 2, major axis at ``angle``."""
    return ellipse(radius, 2.0, angle, K)


def radial_maps(H: int, W: int, lo: float, hi: float, tangential: bool = False,
                seed: int = SEED_MAP) -> tuple[np.ndarray, np.ndarray]:
    """Strength and angle maps of the radial effects: strength grows from lo
    at the frame centre to hi at the corners (plus a faint smooth
    perturbation); the angle (radians, x right, y down) points away from the
    centre (radial motion blur) or across that direction (rotational bokeh).
    Returns float32 [H][W] strength and float32 [H][W] angle."""
    y = np.arange(H)[:, None] - (H - 1) / 2.0
    x = np.arange(W)[None, :] - (W - 1) / 2.0
    r = np.sqrt(x * x + y * y)
    t = r / r.max()
    pert = 0.05 * (smooth_field(H, W, 96.0, seed, stream=9) - 0.5)
    strength = np.clip(lo + (hi - lo) * (t + pert), lo, hi).astype(np.float32)
    ang = np.arctan2(np.broadcast_to(y, (H, W)), np.broadcast_to(x, (H, W)))
    if tangential:
        ang = ang + np.pi / 2
    return strength, ang.astype(np.float32)


def ring(radius: float, width: float, K: int | None = None) -> np.ndarray:
    K = K or kernel_size_for(radius)
    xx, yy = _grid(K)
    r = np.sqrt(xx * xx + yy * yy)
    return _coverage((r <= radius) & (r >= radius - width), K)


def polygon(verts: np.ndarray, K: int) -> np.ndarray:
    """Even-odd fill of a closed polygon with vertices [n][2] (x, y) about the
    kernel centre."""
    # A sample (x, y) is inside when an odd number of edges cross its row y
    # at some xint > x.  Per edge, the rows it crosses and where; the samples
    # of a row left of a crossing are a prefix (the axis is ascending), so the
    # count per sample is a running sum of the crossings' prefix lengths.
    s = _axis(K)
    M = len(s)
    at = np.zeros((M, M + 1), dtype=np.int32)  # crossings per (row, prefix length)
    n = len(verts)
    for i in range(n):
        x1, y1 = verts[i]
        x2, y2 = verts[(i + 1) % n]
        rows = np.nonzero((y1 > s) != (y2 > s))[0]
        if rows.size == 0:
            continue
        xint = (x2 - x1) * (s[rows] - y1) / (y2 - y1) + x1
        np.add.at(at, (rows, np.searchsorted(s, xint, side="left")), 1)
    count = np.cumsum(at[:, ::-1], axis=1)[:, ::-1]  # crossings with prefix length >= m
    return _coverage((count[:, 1:] & 1).astype(bool), K)


def star(points: int, r_out: float, r_in: float, phase: float, K: int) -> np.ndarray:
    ang = phase + np.pi * np.arange(2 * points) / points
    rad = np.where(np.arange(2 * points) % 2 == 0, r_out, r_in)
    return polygon(np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1), K)


def random_shape(K: int, g: np.random.Generator) -> tuple[str, np.ndarray]:
    """One non-convex target of odd size K: random star-shaped polygon, ring,
    5-8 point star or annulus, all inside the K x K box."""
    h = (K - 1) / 2.0
    kind = int(g.integers(0, 4))
    if kind == 0:
        n = int(g.integers(6, 13))
        ang = np.sort(g.uniform(0, 2 * np.pi, n))
        rad = g.uniform(0.35, 1.0, n) * (h - 0.5)
        return "polygon", polygon(np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1), K)
    if kind == 1:
        r = g.uniform(0.6, 1.0) * (h - 0.5)
        return "ring", ring(r, max(1.5, g.uniform(0.06, 0.12) * r), K)
    if kind == 2:
        p = int(g.integers(5, 9))
        ro = g.uniform(0.75, 1.0) * (h - 0.5)
        return "star", star(p, ro, ro * g.uniform(0.35, 0.6), g.uniform(0, 2 * np.pi), K)
    r = g.uniform(0.6, 1.0) * (h - 0.5)
    return "annulus", ring(r, g.uniform(0.3, 0.55) * r, K)


def shape_batch(n: int, seed: int = SEED_SHAPE, kmin: int = 33, kmax: int = 129,
                first: int = 0) -> list[np.ndarray]:
    """n seeded non-convex targets of odd sizes uniform over {kmin..kmax},
    unit sum.  Target j of a batch depends only on (seed, first + j), so train
    and held-out sets drawn from disjoint index ranges never overlap."""
    out = []
    for j in range(first, first + n):
        g = rng(seed, 1000 + j)
        K = int(g.integers(kmin // 2, kmax // 2 + 1)) * 2 + 1
        out.append(random_shape(K, g)[1])
    return out


def ring_batch(n: int, seed: int = SEED_SHAPE, kmin: int = 33, kmax: int = 81,
               first: int = 0) -> list[np.ndarray]:
    """n seeded ring kernels (the layer/sample ablation's target family):
    odd size uniform over {kmin..kmax}, outer radius 0.6..1.0 of the
    half-width, width 0.06..0.25 of the radius (at least 1.5 px)."""
    out = []
    for j in range(first, first + n):
        g = rng(seed, 50000 + j)
        K = int(g.integers(kmin // 2, kmax // 2 + 1)) * 2 + 1
        r = g.uniform(0.6, 1.0) * ((K - 1) / 2.0 - 0.5)
        out.append(ring(r, max(1.5, g.uniform(0.06, 0.25) * r), K))
    return out


# --------------------------------------------------------------------------
# The five workload presets (sizes and node sets of the benchmark configs)
# --------------------------------------------------------------------------

C1 = dict(name="sv_256_fp32_1d", H=256, W=256, C=3, L=3, T=8, nodes=[1.0, 2.0, 4.0, 8.0],
          map_range=(1.0, 8.0), map_sigma=16.0)
C2 = dict(name="sv_bokeh_1080p_fp32_1d", H=1080, W=1920, C=3, L=4, T=16,
          nodes=list(np.linspace(1.0, 32.0, 16)), map_range=(1.0, 32.0), map_sigma=96.0,
          dense_K=65)
C3 = dict(name="fit_batch_256", batch=256, L=4, T=16, steps=500, kmin=33, kmax=129)
C4 = dict(name="sv_4k_fp16_2d", H=2160, W=3840, C=3, L=4, T=24,
          nodes0=list(np.linspace(2.0, 40.0, 8)), nodes1=list(np.linspace(0.0, 1.0, 8)),
          map_range0=(2.0, 40.0), map_range1=(0.0, 1.0), map_sigma=192.0, dense_K=81)
G = dict(name="sv_4k_fp16_gaussian_tilt_shift", H=2160, W=3840, C=3, L=6, T=8,
         nodes=list(np.linspace(1.0, 11.0, 11)), map_range=(1.0, 11.0), dense_K=67)
RM = dict(name="sv_4k_fp16_radial_motion", H=2160, W=3840, C=3, L=3, T=8,
          nodes=list(np.linspace(2.0, 40.0, 12)), map_range=(2.0, 40.0), dense_K=41,
          dense_angles=37)
RB = dict(name="sv_4k_fp16_rotational_bokeh", H=2160, W=3840, C=3, L=4, T=16,
          nodes=list(np.linspace(2.0, 24.0, 12)), map_range=(2.0, 24.0), dense_K=49,
          dense_angles=37)
C5 = dict(name="mlp_init", train=50000, heldout=2000, L=4, T=16, hidden=512, depth=3, side=64)


def c1_inputs(H: int | None = None, W: int | None = None):
    """Config 1: uniform image, smooth s-map in [1, 8], random 4-node basis."""
    H = H or C1["H"]
    W = W or C1["W"]
    img = image_uniform(H, W, 3)
    m = param_map(H, W, *C1["map_range"], sigma=C1["map_sigma"])
    th = basis_random(C1["nodes"], C1["L"], C1["T"])
    return img, m[None], [len(C1["nodes"])], np.array(C1["nodes"], np.float32), th


def disk_lut(node_vals, K: int) -> np.ndarray:
    """Dense disk kernels of the given radii, all padded to K x K."""
    return np.stack([disk(r, K) for r in node_vals]).astype(np.float32)


def ellipse_lut(nodes0, nodes1, K: int) -> np.ndarray:
    """Dense ellipse kernels on the (radius, u) grid, node (a, b) at a*n1 + b."""
    return np.stack([ellipse(*ellipse_params(r, u), K) for r in nodes0 for u in nodes1]
                    ).astype(np.float32)
