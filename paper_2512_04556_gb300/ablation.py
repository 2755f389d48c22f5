"""Layer/sample and initialisation ablations on ring kernels (Sec. 5.4,
Fig. 6 and Fig. 7), run with the batched GPU fitter, and the quality/cost
table built from them.

For every (L, T) of a grid the whole ring batch is fitted in one launch; the
result per configuration is the median (and 90th percentile) relative MSE
sum (K_syn - K_tgt)^2 / sum K_tgt^2 over the batch, its convergence curve, the
fit time, and the cost of filtering a 4K FP16 frame with a basis of those
fitted complexes (the per-pixel cost grows with the tap count L*T, Sec. 4.2).
``choose`` then picks the cheapest configuration that meets a quality target,
the trade-off Sec. 4.3 leaves to the user.

  python -m paper_2512_04556_gb300.ablation [--rings N] [--steps S] [--json out.json]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import disk
from . import workloads as wl

GRID_L = (1, 2, 3, 4, 6, 8)
GRID_T = (4, 8, 12, 16, 24, 32)
INITS = {"rand": disk.INIT_RAND, "ir": disk.INIT_IR, "ss": disk.INIT_SS}


def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def relative(hist, targets) -> np.ndarray:
    """Loss history [batch, steps+1] (mean over the K x K target) to the
    relative MSE per target and step."""
    scale = np.array([t.size / float((t ** 2).sum()) for t in targets])
    return hist * scale[:, None]


def fit_config(packed, sizes, targets, L: int, T: int, steps: int, init: int, seed: int = 0,
               stream=None) -> dict:
    import torch
    stream = stream or torch.cuda.current_stream()
    a, b = _events(stream)
    a.record(stream)
    th, _, hist = disk.fit(packed, sizes, L, T, steps, init=init, seed=seed, loss_hist=True,
                           stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    rel = relative(hist.cpu().numpy().astype(np.float64), targets)
    marks = sorted({0, steps // 10, steps // 4, steps // 2, steps})
    return {"L": L, "T": T, "taps": L * T, "steps": steps,
            "median_rel_mse": float(np.median(rel[:, -1])),
            "p90_rel_mse": float(np.percentile(rel[:, -1], 90)),
            "curve": {int(m): float(np.median(rel[:, m])) for m in marks},
            "fit_ms": a.elapsed_time(b), "theta": th}


def filter_cost(theta, sizes, H: int = 2160, W: int = 3840, reps: int = 5, stream=None) -> float:
    """Median time (ms) of one autotuned FP16 pass over an H x W frame with a
    1-D basis of up to 16 of the fitted complexes (nodes in order of target
    size) under a smooth map over the node range."""
    import torch
    stream = stream or torch.cuda.current_stream()
    order = np.argsort(sizes, kind="stable")
    pick = order[np.linspace(0, len(order) - 1, min(16, len(order))).round().astype(int)]
    nodes = np.arange(len(pick), dtype=np.float32)
    b = disk.Basis.from_arrays([nodes], theta.cpu().numpy()[pick])
    img = torch.from_numpy(wl.to_fp16(wl.image_rects(H, W, 3))).cuda()
    maps = torch.from_numpy(wl.param_map(H, W, 0.0, float(len(pick) - 1), sigma=192.0)[None]).cuda()
    out = torch.empty_like(img)
    disk.sv_filter_autotune(b, img, maps, out=out, stream=stream)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    ts = []
    for _ in range(reps):
        flush.fill_(1)
        e0, e1 = _events(stream)
        e0.record(stream)
        disk.sv_filter(b, img, maps, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def sweep(n_rings: int = 64, steps: int = 500, grid=None, init: int = disk.INIT_SS,
          seed: int = 0, cost: bool = True) -> list[dict]:
    targets = wl.ring_batch(n_rings)
    packed, sizes = disk.pack_targets(targets)
    grid = grid or [(L, T) for L in GRID_L for T in GRID_T]
    rows = []
    for L, T in grid:
        r = fit_config(packed, sizes, targets, L, T, steps, init, seed)
        th = r.pop("theta")
        if cost:
            ms = filter_cost(th, sizes)
            r["filter_4k_ms"] = ms
            r["filter_4k_gpix_s"] = 2160 * 3840 / (ms * 1e-3) / 1e9
        rows.append(r)
    return rows


def init_sweep(n_rings: int = 64, steps: int = 500, L: int = 4, T: int = 16, seed: int = 0) -> dict:
    targets = wl.ring_batch(n_rings)
    packed, sizes = disk.pack_targets(targets)
    out = {}
    for name, code in INITS.items():
        r = fit_config(packed, sizes, targets, L, T, steps, code, seed)
        r.pop("theta")
        out[name] = r
    return out


def choose(rows: list[dict], tol: float, cost_key: str = "taps") -> dict | None:
    """The cheapest configuration (by cost_key) whose median relative MSE is
    at most tol; None if none reaches it.  Ties go to the better quality."""
    ok = [r for r in rows if r["median_rel_mse"] <= tol]
    if not ok:
        return None
    return min(ok, key=lambda r: (r[cost_key], r["median_rel_mse"]))


def pareto(rows: list[dict], cost_key: str = "filter_4k_ms") -> list[dict]:
    """Configurations not beaten on both cost and quality by another one,
    in order of cost."""
    rs = sorted(rows, key=lambda r: (r[cost_key], r["median_rel_mse"]))
    front, best = [], float("inf")
    for r in rs:
        if r["median_rel_mse"] < best:
            front.append(r)
            best = r["median_rel_mse"]
    return front


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--rings", type=int, default=64)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--json", default=None)
    a = p.parse_args(argv)
    rows = sweep(a.rings, a.steps)
    inits = init_sweep(a.rings, a.steps)
    res = {"rings": a.rings, "steps": a.steps, "grid": rows, "inits": inits,
           "pareto": [(r["L"], r["T"]) for r in pareto(rows)],
           "choose": {str(t): (lambda c: c and (c["L"], c["T"]))(choose(rows, t, "filter_4k_ms"))
                      for t in (1e-1, 5e-2, 2e-2, 1e-2)}}
    txt = json.dumps(res, indent=1)
    if a.json:
        with open(a.json, "w") as f:
            f.write(txt)
    print(f"{'L':>2} {'T':>3} {'taps':>4} {'median':>9} {'p90':>9} {'fit ms':>8} {'4K ms':>7}")
    for r in rows:
        print(f"{r['L']:>2} {r['T']:>3} {r['taps']:>4} {r['median_rel_mse']:9.3e} "
              f"{r['p90_rel_mse']:9.3e} {r['fit_ms']:8.1f} {r.get('filter_4k_ms', 0):7.3f}")
    for k, r in inits.items():
        print(f"init {k}: median {r['median_rel_mse']:.3e} curve {r['curve']}")
    print("pareto", res["pareto"])
    print("choose", res["choose"])


if __name__ == "__main__":
    main()
