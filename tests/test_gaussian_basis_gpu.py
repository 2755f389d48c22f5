"""The Gaussian sigma basis fitted on the GPU by the batched fitter (one
launch, all 11 nodes, L=6, T=8, Eq. 6 radial start, 1000 Adam steps of the
Sec. 5.1 schedule) against the FP64 oracle's fitter, and filtering with it."""
import numpy as np
import pytest

import oracle
from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SIGMAS = np.linspace(1.0, 11.0, 11)


@pytest.fixture(scope="module")
def gpu_basis():
    import torch
    from paper_2512_04556_gb300 import disk
    assert torch.cuda.is_available()
    tg = [wl.gaussian(float(s)) for s in SIGMAS]
    packed, sizes = disk.pack_targets(tg)
    th, final, hist = disk.fit(packed, sizes, 6, 8, 1000, init=disk.INIT_IR, loss_hist=True)
    return tg, th.cpu().numpy(), final.cpu().numpy(), hist.cpu().numpy()


@pytest.mark.parametrize("node", [1, 5])
def test_batched_gaussian_fit_matches_oracle(gpu_basis, node):
    tg, _, _, hist = gpu_basis
    _, want = oracle.fit(tg[node], 6, 8, 1000, init=oracle.INIT_IR)
    np.testing.assert_allclose(hist[node, [0, 100, 1000]], want[[0, 100, 1000]], rtol=2e-2)


def test_batched_gaussian_basis_quality(gpu_basis):
    """Every node reaches a relative MSE below 2e-3 (the oracle's own fits from
    the radial start reach 1.6e-4 at sigma 1 to 1.5e-3 at sigma 11), checked
    on the oracle's impulse response of the GPU-fitted complex."""
    tg, th, final, _ = gpu_basis
    for b, t in enumerate(tg):
        ir = oracle.synth(th[b].astype(np.float64), t.shape[0])
        assert ((ir - t) ** 2).sum() / (t ** 2).sum() <= 2e-3


def test_gpu_fitted_basis_filters_like_oracle(gpu_basis):
    """The GPU-fitted basis, loaded as a 1-D basis over sigma, filters a
    tilt-shift frame exactly as the oracle does with the same complexes."""
    import torch
    from paper_2512_04556_gb300 import disk
    _, th, _, _ = gpu_basis
    b = disk.Basis.from_arrays([SIGMAS], th)
    H, W = 200, 136
    img = wl.image_rects(H, W, 3, seed=5)
    maps = wl.tilt_shift_map(H, W, 1.0, 11.0)[None]
    out = disk.sv_filter(b, torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()).cpu().numpy()
    want = oracle.sv_filter(img.astype(np.float64), maps.astype(np.float64), [11], SIGMAS,
                            th.astype(np.float64))
    assert np.abs(out - want).max() / np.abs(want).max() <= 1e-5
