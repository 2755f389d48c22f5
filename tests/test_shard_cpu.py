"""Row-band sharding of the filter (host logic, no GPU): filtering the bands
with the FP64 oracle and stacking them reproduces the full-frame oracle
exactly, for one rank and for two gloo ranks that gather their bands."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import shard
from paper_2512_04556_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _case():
    img, maps, nn, nv, th = wl.c1_inputs(61, 37)
    return img.astype(np.float64), maps.astype(np.float64), nn, nv.astype(np.float64), th.astype(np.float64)


def test_bands_cover_rows_once():
    for H, world, R in [(61, 1, 5), (61, 2, 30), (61, 3, 7), (5, 4, 100)]:
        bands = shard.row_bands(H, world, R)
        rows = np.concatenate([np.arange(b.out_y0, b.out_y1) for b in bands])
        np.testing.assert_array_equal(rows, np.arange(H))
        for b in bands:
            assert b.in_y0 == max(0, b.out_y0 - R) and b.in_y1 == min(H, b.out_y1 + R)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_banded_oracle_equals_full_frame(world):
    img, maps, nn, nv, th = _case()
    fn = lambda a, m: oracle.sv_filter(np.ascontiguousarray(a), np.ascontiguousarray(m), nn, nv, th)
    full = fn(img, maps)
    R = shard.cascade_reach(th)
    parts = [shard.filter_band(fn, img, maps, b) for b in shard.row_bands(img.shape[0], world, R)]
    np.testing.assert_array_equal(np.concatenate(parts), full)


def test_band_too_thin_halo_differs():
    """With a halo one row short the band edge reads clamped rows that the
    full frame does not: the reach is needed in full."""
    img, maps, nn, nv, th = _case()
    fn = lambda a, m: oracle.sv_filter(np.ascontiguousarray(a), np.ascontiguousarray(m), nn, nv, th)
    full = fn(img, maps)
    R = shard.cascade_reach(th)
    parts = [shard.filter_band(fn, img, maps, b) for b in shard.row_bands(img.shape[0], 2, R // 3)]
    assert np.abs(np.concatenate(parts) - full).max() > 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    img, maps, nn, nv, th = _case()
    fn = lambda a, m: oracle.sv_filter(np.ascontiguousarray(a), np.ascontiguousarray(m), nn, nv, th)
    bands = shard.row_bands(img.shape[0], world, shard.cascade_reach(th))
    mine = torch.from_numpy(shard.filter_band(fn, img, maps, bands[rank]))
    # gather: pad every band to the tallest, all-gather, trim
    hmax = max(b.out_y1 - b.out_y0 for b in bands)
    pad = torch.zeros((hmax,) + tuple(mine.shape[1:]), dtype=mine.dtype)
    pad[:mine.shape[0]] = mine
    got = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(got, pad)
    frame = torch.cat([g[:b.out_y1 - b.out_y0] for g, b in zip(got, bands)]).numpy()
    np.save(os.path.join(out_dir, f"r{rank}.npy"), frame)
    dist.destroy_process_group()


def test_two_ranks_gather_bands_gloo(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    img, maps, nn, nv, th = _case()
    full = oracle.sv_filter(img, maps, nn, nv, th)
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"r{r}.npy"), full)


def test_balance_targets_covers_and_balances():
    sizes = [int(s) for s in np.random.default_rng(2).integers(16, 65, 257) * 2 + 1]
    for world in (1, 2, 3, 8):
        parts = shard.balance_targets(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] ** 2 for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(s ** 2 for s in sizes)
