"""Fits the bases of the two full-size filtering workloads with the FP64
oracle's fitter and writes them as basis files (calls only ``oracle/``).

Offline stage of Sec. 4.3: every node's complex is fitted to its own dense
target with the Eq. 4 objective, Adam and the Sec. 5.1 schedule (1000 steps,
lr 1e-3 -> 1e-4).  Nodes are fitted in order along the radius axis, each
warm-started from its neighbour with offsets scaled by the ratio of target
half-widths, so that tap i means the same tap across nodes and blending them
(Eq. 9) is meaningful; the first node of each chain starts from the Eq. 6
radial initialisation.

  bases/disk16_L4T16.dkb    16 disks, radius 1..32 px, L=4, T=16 (1-D)
  bases/gauss11_L6T8.dkb    11 Gaussians, sigma 1..11 px, L=6, T=8 (1-D; the paper's
                            6-layer, 8-sample configuration)
  bases/line12_L3T8.dkb     12 motion-blur segments, length 2..40 px, along x, L=3, T=8 (1-D;
                            turned per pixel at run time for radial motion blur)
  bases/cateye12_L4T16.dkb  12 ellipses of aspect 2, semi-major 2..24 px, along x, L=4, T=16
                            (1-D; turned per pixel at run time for rotational bokeh)
  bases/ellipse8x8_L4T24.dkb  8 x 8 ellipses, radius 2..40 px x u in [0,1]
                            (anisotropy 1+3u, rotation pi u), L=4, T=24 (2-D)

Usage: python tests/golden/make_bases.py [--steps N] [--only disk|ellipse|gauss|line|cateye]
"""
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "bases")


def _chain(args):
    kind, radii, u, L, T, steps = args
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_2512_04556_gb300 import workloads as wl
    thetas, losses, prev = [], [], None
    for r in radii:
        if kind == "disk":
            tgt = wl.disk(r)
        elif kind == "gauss":
            tgt = wl.gaussian(r)
        elif kind == "line":
            tgt = wl.line(r)
        elif kind == "cateye":
            tgt = wl.cat_eye(r)
        else:
            tgt = wl.ellipse(*wl.ellipse_params(r, u))
        K = tgt.shape[0]
        hw = max(1.0, (K - 1) / 2)
        if prev is None:
            th, hist = oracle.fit(tgt, L, T, steps, init=oracle.INIT_IR)
        else:
            th0 = prev[0].copy()
            th0[..., :2] *= hw / prev[1]
            th0[..., :2] = np.clip(th0[..., :2], -hw, hw)
            th, hist = oracle.fit(tgt, L, T, steps, init=oracle.INIT_GIVEN, theta0=th0)
        rel = hist[-1] * K * K / float((tgt ** 2).sum())
        thetas.append(th)
        losses.append(dict(radius=float(r), u=u, K=K, mse=float(hist[-1]), rel_mse=float(rel),
                           mse0=float(hist[0])))
        prev = (th, hw)
    return kind, u, thetas, losses


def main(steps=1000, only=None):
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import basis_io
    from paper_2512_04556_gb300 import workloads as wl
    os.makedirs(OUT, exist_ok=True)
    c2, c4 = wl.C2, wl.C4
    g = wl.G
    jobs = [("disk", list(c2["nodes"]), 0.0, c2["L"], c2["T"], steps)]
    jobs += [("ellipse", list(c4["nodes0"]), float(u), c4["L"], c4["T"], steps) for u in c4["nodes1"]]
    jobs += [("gauss", list(g["nodes"]), 0.0, g["L"], g["T"], steps)]
    jobs += [("line", list(wl.RM["nodes"]), 0.0, wl.RM["L"], wl.RM["T"], steps)]
    jobs += [("cateye", list(wl.RB["nodes"]), 0.0, wl.RB["L"], wl.RB["T"], steps)]
    if only:
        jobs = [j for j in jobs if j[0] in only.split(",")]
    os.environ["OMP_NUM_THREADS"] = "1"
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 4)) as pool:
        res = pool.map(_chain, jobs)
    rpath = os.path.join(OUT, "fit_report.json")
    report = json.load(open(rpath)) if os.path.exists(rpath) else {}
    report["steps"] = steps
    kinds = {r[0] for r in res}
    if "disk" in kinds:
        disk_th = [r for r in res if r[0] == "disk"][0]
        basis_io.write(os.path.join(OUT, "disk16_L4T16.dkb"), [c2["nodes"]], np.stack(disk_th[2]))
        report["disk"] = disk_th[3]
    if "gauss" in kinds:
        gth = [r for r in res if r[0] == "gauss"][0]
        basis_io.write(os.path.join(OUT, "gauss11_L6T8.dkb"), [g["nodes"]], np.stack(gth[2]))
        report["gauss"] = gth[3]
    for kind, preset, fname in (("line", wl.RM, "line12_L3T8.dkb"),
                                ("cateye", wl.RB, "cateye12_L4T16.dkb")):
        if kind in kinds:
            th = [r for r in res if r[0] == kind][0]
            basis_io.write(os.path.join(OUT, fname), [preset["nodes"]], np.stack(th[2]))
            report[kind] = th[3]
    if "ellipse" in kinds:
        ell = {r[1]: r for r in res if r[0] == "ellipse"}
        th = np.zeros((8, 8, c4["L"], c4["T"], 3))
        losses = []
        for b, u in enumerate(c4["nodes1"]):
            for a in range(8):
                th[a, b] = ell[float(u)][2][a]
            losses += ell[float(u)][3]
        basis_io.write(os.path.join(OUT, "ellipse8x8_L4T24.dkb"), [c4["nodes0"], c4["nodes1"]],
                       th.reshape(64, c4["L"], c4["T"], 3))
        report["ellipse"] = losses
    with open(rpath, "w") as f:
        json.dump(report, f, indent=1)
    print(f"wrote bases in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    n = 1000
    if "--steps" in sys.argv:
        n = int(sys.argv[sys.argv.index("--steps") + 1])
    only = sys.argv[sys.argv.index("--only") + 1] if "--only" in sys.argv else None
    main(n, only)
