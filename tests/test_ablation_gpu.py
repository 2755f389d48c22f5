"""Layer/sample ablation on rings with the batched fitter: every grid cell's
loss history agrees with the FP64 oracle's fit of the same ring, and the
sweep reproduces the trends of Fig. 6 and Fig. 7."""
import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GRID = [(1, 8), (2, 8), (4, 4), (4, 16)]


@pytest.fixture(scope="module")
def rings():
    import torch
    assert torch.cuda.is_available()
    return wl.ring_batch(12, kmax=49)


@pytest.mark.parametrize("L,T", GRID)
def test_grid_cell_matches_oracle(rings, L, T):
    from paper_2512_04556_gb300 import disk
    packed, sizes = disk.pack_targets(rings)
    _, _, hist = disk.fit(packed, sizes, L, T, 200, init=disk.INIT_SS, seed=4, loss_hist=True)
    hist = hist.cpu().numpy()
    j = int(np.argmin(sizes))
    _, want = oracle.fit(rings[j], L, T, 200, init=oracle.INIT_SS, seed=4)
    np.testing.assert_allclose(hist[j, [0, 50, 200]], want[[0, 50, 200]], rtol=2e-2)


def test_sweep_trends(rings):
    """More taps give lower median error (Fig. 7); SS beats IR beats random
    starts after the same number of steps (Fig. 6)."""
    from paper_2512_04556_gb300 import ablation, disk
    packed, sizes = disk.pack_targets(rings)
    rel = {}
    for L, T in [(1, 8), (4, 16)]:
        r = ablation.fit_config(packed, sizes, rings, L, T, 300, disk.INIT_SS)
        rel[(L, T)] = r["median_rel_mse"]
        assert r["curve"][0] >= r["curve"][300]
    assert rel[(4, 16)] < rel[(1, 8)]
    inits = {k: ablation.fit_config(packed, sizes, rings, 4, 16, 300, c)["median_rel_mse"]
             for k, c in ablation.INITS.items()}
    assert inits["ss"] < inits["ir"] < inits["rand"]


def test_filter_cost_grows_with_taps(rings):
    from paper_2512_04556_gb300 import ablation, disk
    packed, sizes = disk.pack_targets(rings)
    ms = {}
    for L, T in [(2, 8), (4, 16)]:
        th = ablation.fit_config(packed, sizes, rings, L, T, 50, disk.INIT_SS)["theta"]
        ms[(L, T)] = ablation.filter_cost(th, sizes, H=540, W=960, reps=3)
    assert ms[(4, 16)] > ms[(2, 8)]
