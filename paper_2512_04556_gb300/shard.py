"""Row-band sharding of the spatially varying filter across ranks.

An output pixel of the L-layer cascade depends only on input rows within
R = sum_l (ceil(reach_l) + 1) of it (each layer reads at most ceil(reach) + 1
rows away, clamped to the image).  So rank r can filter output rows
[y0, y1) exactly from the input rows [max(0, y0 - R), min(H, y1 + R)):
inside the band the halo rows stand in for the rest of the image, and at the
true image border clamp-to-edge reads the same rows the full frame reads.
No collective is needed on the data path; gathering the bands (if the caller
wants the whole frame on one rank) is the only exchange.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Band:
    out_y0: int   # first output row of the band
    out_y1: int   # one past the last output row
    in_y0: int    # first input row the band reads
    in_y1: int    # one past the last input row

    @property
    def crop(self) -> slice:
        """Rows of the band's filtered input that are its output rows."""
        return slice(self.out_y0 - self.in_y0, self.out_y1 - self.in_y0)


def cascade_reach(theta) -> int:
    """R = sum over layers of ceil(max per-axis |offset|) + 1 for a basis
    theta [B][L][T][3] (pixels); rotated filtering uses the Euclidean length
    (rotated=True in row_bands)."""
    th = np.asarray(theta, dtype=np.float64)
    return int(sum(math.ceil(float(np.abs(th[:, l, :, :2]).max())) + 1 for l in range(th.shape[1])))


def cascade_reach_rotated(theta) -> int:
    th = np.asarray(theta, dtype=np.float64)
    return int(sum(math.ceil(float(np.hypot(th[:, l, :, 0], th[:, l, :, 1]).max())) + 1
                   for l in range(th.shape[1])))


def row_bands(H: int, world: int, R: int) -> list[Band]:
    """world contiguous output bands of near-equal height (the first H % world
    get one extra row), each with the input rows it needs."""
    if world < 1 or H < 1 or R < 0:
        raise ValueError("H >= 1, world >= 1 and R >= 0 required")
    base, extra = divmod(H, world)
    bands, y = [], 0
    for r in range(world):
        h = base + (1 if r < extra else 0)
        y0, y1 = y, y + h
        bands.append(Band(y0, y1, max(0, y0 - R), min(H, y1 + R)))
        y = y1
    return bands


def filter_band(filter_fn, img, maps, band: Band):
    """Apply filter_fn(img_rows, maps_rows) -> filtered rows to the band's
    input rows and keep its output rows.  img [H][W][C] and maps [dims][H][W]
    may be numpy arrays or tensors (any that slice like numpy)."""
    out = filter_fn(img[band.in_y0:band.in_y1], maps[:, band.in_y0:band.in_y1])
    return out[band.crop]


def balance_targets(sizes, world: int) -> list[list[int]]:
    """Split a batch of fitting targets over ranks (the fitter shards by
    target, with no exchange): longest-processing-time greedy on a target's
    work, taken as the area of its canvas (its size squared), so each rank's
    total work is within one target's work of the others'."""
    if world < 1:
        raise ValueError("world >= 1 required")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 2, i))
    loads = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += int(sizes[i]) ** 2
    return parts
