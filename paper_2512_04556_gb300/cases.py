"""Named workloads, run once each through the public API (for profiling and
quick checks): ``python -m paper_2512_04556_gb300.cases <name> [--reps N]``.

  filter4k      4K RGB FP16, 8 x 8 fitted ellipse basis, L=4, T=24 (the benchmark frame,
                autotuned tiles as the benchmark uses)
  pair4k        the same frame with layers 1 and 2 fused into one launch (sv_pair_kernel),
                layers 3 and 4 single (32 x 16, 32 x 32)
  backward4k    full backward (image and basis gradients) on the same frame
  dense4k       dense spatially varying convolution on the same frame
  gauss4k       4K RGB FP16 under a tilt-shift sigma map, 11 fitted Gaussians, L=6, T=8
  radial4k      4K RGB FP16 radial motion blur: 12 fitted segments (L=3, T=8) turned per pixel
  bokeh4k       4K RGB FP16 rotational bokeh: 12 fitted aspect-2 ellipses (L=4, T=16) turned
  filter1080p   1080p RGB FP32, 16 fitted disks, L=4, T=16
  fit           64 uneven targets, L=4, T=16, 100 steps (sparse-sampling init)
  fit256        the benchmark's 256 uneven targets, L=4, T=16, 100 steps, 512 threads x
                4-CTA clusters per target (the benchmark's launch configuration)
  mlp           one training step of the learned initializer, batch 256
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASES = os.path.join(ROOT, "tests", "golden", "bases")


def _frame4k():
    from . import workloads as wl
    H, W = wl.C4["H"], wl.C4["W"]
    img = wl.to_fp16(wl.image_rects(H, W, 3))
    m0 = wl.param_map(H, W, *wl.C4["map_range0"], sigma=wl.C4["map_sigma"], stream=0)
    m1 = wl.param_map(H, W, *wl.C4["map_range1"], sigma=wl.C4["map_sigma"], stream=1)
    return img, np.stack([m0, m1])


def main(argv=None):
    import torch

    from . import disk
    from . import workloads as wl
    p = argparse.ArgumentParser()
    p.add_argument("name")
    p.add_argument("--reps", type=int, default=1)
    a = p.parse_args(argv)
    run = None
    if a.name in ("filter4k", "pair4k", "backward4k", "dense4k"):
        img, maps = _frame4k()
        di, dm = torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()
        if a.name == "dense4k":
            n0, n1 = np.linspace(2.0, 40.0, 16), np.linspace(0.0, 1.0, 16)
            lut = torch.from_numpy(wl.ellipse_lut(n0, n1, 81)).cuda()
            run = lambda: disk.dense_sv([n0, n1], lut, di, dm)
        else:
            b = disk.Basis.load(os.path.join(BASES, "ellipse8x8_L4T24.dkb"))
            if a.name == "filter4k":
                disk.sv_filter_autotune(b, di, dm)      # the benchmark's tile choice
                run = lambda: disk.sv_filter(b, di, dm)
            elif a.name == "pair4k":
                disk.sv_filter_set_layers(b, di, [8, 0, 2, 4])
                run = lambda: disk.sv_filter(b, di, dm)
            else:
                go = torch.empty_like(di).uniform_(-1, 1)
                run = lambda: disk.sv_filter_backward(b, di, go, dm)
    elif a.name == "gauss4k":
        g = wl.G
        img = wl.to_fp16(wl.image_rects(g["H"], g["W"], 3))
        maps = wl.tilt_shift_map(g["H"], g["W"], *g["map_range"])[None]
        b = disk.Basis.load(os.path.join(BASES, "gauss11_L6T8.dkb"))
        di, dm = torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()
        disk.sv_filter_autotune(b, di, dm)
        run = lambda: disk.sv_filter(b, di, dm)
    elif a.name in ("radial4k", "bokeh4k"):
        pre, fname = (wl.RM, "line12_L3T8.dkb") if a.name == "radial4k" else (wl.RB, "cateye12_L4T16.dkb")
        img = wl.to_fp16(wl.image_rects(pre["H"], pre["W"], 3))
        st, ang = wl.radial_maps(pre["H"], pre["W"], *pre["map_range"], tangential=a.name == "bokeh4k")
        b = disk.Basis.load(os.path.join(BASES, fname))
        di, dm, da = (torch.from_numpy(img).cuda(), torch.from_numpy(st[None]).cuda(),
                      torch.from_numpy(ang).cuda())
        disk.sv_filter_rotated_autotune(b, di, dm, da)
        run = lambda: disk.sv_filter_rotated(b, di, dm, da)
    elif a.name == "filter1080p":
        img = wl.image_rects(1080, 1920, 3)
        maps = wl.param_map(1080, 1920, 1.0, 32.0, sigma=96.0)[None]
        b = disk.Basis.load(os.path.join(BASES, "disk16_L4T16.dkb"))
        di, dm = torch.from_numpy(img).cuda(), torch.from_numpy(maps).cuda()
        run = lambda: disk.sv_filter(b, di, dm)
    elif a.name == "fit":
        packed, sizes = disk.pack_targets(wl.shape_batch(64))
        run = lambda: disk.fit(packed, sizes, 4, 16, 100, init=disk.INIT_SS, seed=1)
    elif a.name == "fit256":
        tg = wl.shape_batch(256)
        packed, sizes = disk.pack_targets(tg)
        disk.fit_set_config(4, 16, max(sizes), 512, 4)
        run = lambda: disk.fit(packed, sizes, 4, 16, 100, init=disk.INIT_SS, seed=7)
    elif a.name == "mlp":
        net = disk.MLP(4096, 512, 3, 192, seed=0)
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.rand((256, 4096), device="cuda", generator=g)
        t = torch.randn((256, 192), device="cuda", generator=g)
        run = lambda: net.train_step(x, t, 1e-3)
    else:
        sys.exit(f"unknown case {a.name}")
    for _ in range(a.reps):
        run()
    torch.cuda.synchronize()
    print(f"{a.name}: ok ({a.reps} run(s))")


if __name__ == "__main__":
    main()
