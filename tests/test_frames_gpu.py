"""Host-frame pipeline (disk_sv_filter_frames): frames copied in, filtered
and copied out with the copies overlapping the filtering of other frames.
Every output must equal the device-resident filter on the same frame."""
import numpy as np
import pytest

from paper_2512_04556_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.mark.parametrize("fp16,dims,n", [(True, 2, 5), (False, 1, 4), (True, 1, 1), (False, 2, 2)])
def test_frames_match_device_filter(torch_cuda, fp16, dims, n):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    H, W = 97, 150
    nodes = [[1.0, 2.0, 4.0]] if dims == 1 else [[1.0, 3.0], [0.0, 0.5, 1.0]]
    B = int(np.prod([len(a) for a in nodes]))
    b = disk.Basis.from_arrays(nodes, wl.basis_random([1.0] * B, 3, 6, 2.0, 21))
    imgs, maps, outs = [], [], []
    for i in range(n):
        im = wl.image_uniform(H, W, 3, seed=100 + i)
        im = wl.to_fp16(im) if fp16 else im
        imgs.append(torch.from_numpy(im).pin_memory())
        m = np.stack([wl.param_map(H, W, 0.5, 4.5, 8.0, 200 + i + 7 * d) for d in range(dims)])
        if dims == 2:
            m[1] = np.clip(m[1] / 4.5, 0, 1)
        maps.append(torch.from_numpy(np.ascontiguousarray(m, dtype=np.float32)).pin_memory())
        outs.append(torch.empty_like(imgs[-1]).pin_memory())
    disk.sv_filter_frames(b, imgs, maps, outs)
    torch.cuda.synchronize()
    for i in range(n):
        want = disk.sv_filter(b, imgs[i].cuda(), maps[i].cuda()).cpu()
        assert torch.equal(outs[i], want), f"frame {i}"


def test_frames_empty_and_mismatch(torch_cuda):
    torch = torch_cuda
    from paper_2512_04556_gb300 import disk
    b = disk.Basis.from_arrays([[1.0, 2.0]], wl.basis_random([1.0, 2.0], 2, 4, 1.0, 3))
    assert disk.sv_filter_frames(b, [], [], []) == []
    im = torch.rand((8, 8, 3))
    with pytest.raises(ValueError):
        disk.sv_filter_frames(b, [im], [], [im.clone()])
