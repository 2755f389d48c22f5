"""Row-band sharding on the GPU: the 4K FP16 benchmark frame filtered as
three bands with their halo rows, stacked, equals the full-frame filter bit
for bit (every output pixel is computed by the same arithmetic)."""
import os

import numpy as np
import pytest

from paper_2512_04556_gb300 import shard
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASES = os.path.join(ROOT, "tests", "golden", "bases")


def test_bands_equal_full_frame_4k():
    import torch
    from oracle import basis_io
    from paper_2512_04556_gb300 import disk
    H, W = wl.C4["H"], wl.C4["W"]
    img = torch.from_numpy(wl.to_fp16(wl.image_rects(H, W, 3))).cuda()
    m0 = wl.param_map(H, W, *wl.C4["map_range0"], sigma=wl.C4["map_sigma"], stream=0)
    m1 = wl.param_map(H, W, *wl.C4["map_range1"], sigma=wl.C4["map_sigma"], stream=1)
    maps = torch.from_numpy(np.stack([m0, m1])).cuda()
    path = os.path.join(BASES, "ellipse8x8_L4T24.dkb")
    b = disk.Basis.load(path)
    full = disk.sv_filter(b, img, maps)
    R = shard.cascade_reach(basis_io.read(path)[1])
    fn = lambda a, m: disk.sv_filter(b, a.contiguous(), m.contiguous())
    parts = [shard.filter_band(fn, img, maps, band) for band in shard.row_bands(H, 3, R)]
    assert torch.equal(torch.cat(parts), full)
