"""Measure the five workload configurations through the C-ABI on cuda:0.

  python benchmarks/run_configs.py [--only C1,C4] [--reps 3]

C1  32^3 top-hat (delta 10 in radius 4 cells), r_V = 8 cells, FP64
C2  128^3 lognormal (sigma 1.5), r_V = 2, 8, 32 cells x both signs, FP64
C3  256^3 lognormal + 8^3 patches over delta > 20 (then > 80): sigma 2.0 and 1.0 at r_V = 8 cells
    and sigma 1.0 at r_V = 8 cells, FP64
C4  512^3 lognormal (sigma 2.0), r_V = 16 cells: mixed vs FP64
C5  64 independent solves of 32..128^3, mixed, batched
Every solve goes to max|d - lambda| < 1e-8 from phi = 0.  Each config prints one
JSON line: device times (CUDA events inside the library), cycles and launch
counts.  Correctness at these sizes is the business of the GPU tests
(tests/test_gpu_fullsize.py and the others), which compare with the CPU oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TOL = 1e-8


def _rel(a, b):
    import numpy as np
    return float(np.abs(a - b).max() / np.abs(b).max())


def _solve(mg, delta, alpha, kappa, reps, **opt):
    import numpy as np
    import torch
    n = delta.shape[0]
    g = mg.mg_create_grid(n, mg.options(**opt))
    try:
        mg.mg_set_stream(g, torch.cuda.current_stream())
        d = torch.from_numpy(delta).cuda()
        mg.mg_set_density(g, 0, -1, d)
        zero = torch.zeros_like(d)
        times = []
        for _ in range(reps):
            mg.mg_set_field(g, 0, -1, zero)
            st = mg.mg_solve(g, 0, alpha, kappa, TOL)
            times.append(st["wall_s"])
        phi = np.empty_like(delta)
        mg.mg_get_field(g, 0, -1, phi)
        force = np.empty((3,) + delta.shape)
        mg.mg_get_force(g, 0, -1, force)
    finally:
        mg.mg_destroy_grid(g)
    st["wall_s_min"] = min(times)
    return st, phi, force


def c1(mg, I, reps):
    w = I.workload_tophat(32)
    st, phi, force = _solve(mg, w["delta"], w["alpha"], w["kappa"], reps)
    return {"config": "C1", "solves_per_s": 1.0 / st["wall_s_min"], "cycles": st["cycles"],
            "res": st["res"], "launches": st["launches"]}


def c2(mg, I, reps):
    w = I.workload_lognormal_sweep(128)
    out = []
    for s in w["solves"]:
        st, phi, _ = _solve(mg, w["delta"], s["alpha"], s["kappa"], reps)
        out.append({"r_v": s["r_v"], "sign": s["kappa"], "ms": 1e3 * st["wall_s_min"],
                    "cycles": st["cycles"], "floored_cells": st["guard_hits"]})
    total = sum(x["ms"] for x in out)
    return {"config": "C2", "solves_per_s": 1e3 * len(out) / total, "solves": out,
            "cell_updates": 128 ** 3}


def c3(mg, I, reps):
    import numpy as np
    import torch
    res = {"config": "C3", "variants": []}
    for sigma, alpha in ((2.0, I.alpha_kappa_for_rv(8.0)), (1.0, I.alpha_kappa_for_rv(8.0))):
        h = I.refined_hierarchy(256, sigma, 1303)
        levels = [L for L in h["levels"] if len(L["origins"])]
        g = mg.mg_create_grid(256, mg.options())
        v = {"sigma": sigma, "alpha_kappa": alpha, "patches": [len(L["origins"]) for L in levels]}
        try:
            mg.mg_set_stream(g, torch.cuda.current_stream())
            mg.mg_set_density(g, 0, -1, h["delta0"])
            for lvl, L in enumerate(levels, start=1):
                mg.mg_add_patches(g, lvl, L["origins"])
                mg.mg_set_density(g, lvl, -1, np.ascontiguousarray(L["delta"]))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = mg.mg_solve(g, 0, alpha, 1.0, TOL)
            torch.cuda.synchronize()
            v["seconds_all_levels"] = time.perf_counter() - t0
            v["domain_ms"] = 1e3 * st["wall_s"]
            v["domain_cycles"] = st["cycles"]
            v["level_cycles"] = [mg.mg_get_level_stats(g, lvl)["cycles"]
                                 for lvl in range(1, len(levels) + 1)]
            v["level_ms"] = [1e3 * mg.mg_get_level_stats(g, lvl)["wall_s"]
                             for lvl in range(1, len(levels) + 1)]
        finally:
            mg.mg_destroy_grid(g)
        res["variants"].append(v)
    return res


def c4(mg, I, reps):
    delta = I.lognormal_delta(512, 2.0, 1304)
    alpha = I.alpha_kappa_for_rv(16.0)
    stm, phim, fm = _solve(mg, delta, alpha, 1.0, reps, prec=1)
    st64, phi64, f64 = _solve(mg, delta, alpha, 1.0, 1, prec=0)
    return {"config": "C4", "mixed_ms": 1e3 * stm["wall_s_min"], "fp64_ms": 1e3 * st64["wall_s_min"],
            "speedup": st64["wall_s_min"] / stm["wall_s_min"], "mixed_outer": stm["outer"],
            "mixed_inner_cycles": stm["cycles"], "fp64_cycles": st64["cycles"],
            "floored_cells": stm["guard_hits"],
            "phi_rel_diff_mixed_vs_fp64": _rel(phim, phi64),
            "force_rel_diff_mixed_vs_fp64": _rel(fm, f64)}


def c5(mg, I, reps):
    import numpy as np
    import torch
    w = I.workload_batch(64)
    specs = [dict(s, delta=I.lognormal_delta(s["n"], s["sigma"], s["seed"])) for s in w]
    g = mg.mg_create_batch([s["n"] for s in specs], mg.options(prec=1))
    try:
        mg.mg_set_stream(g, torch.cuda.current_stream())
        for k, s in enumerate(specs):
            mg.mg_set_density(g, 0, k, s["delta"])
        times = []
        for _ in range(reps):
            zeros = [np.zeros((s["n"],) * 3) for s in specs]
            for k, z in enumerate(zeros):
                mg.mg_set_field(g, 0, k, z)
            rc, stats = mg.mg_solve_batch(g, [s["branch"] for s in specs],
                                          [s["alpha"] for s in specs],
                                          [s["kappa"] for s in specs], TOL)
            times.append(stats[0]["wall_s"])
    finally:
        mg.mg_destroy_grid(g)
    return {"config": "C5", "batch_seconds": min(times), "solves_per_s": 64 / min(times),
            "launches": stats[0]["launches"],
            "max_outer": max(x["outer"] for x in stats),
            "sizes": {str(n): [s["n"] for s in specs].count(n) for n in (32, 64, 96, 128)}}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--only", default="C1,C2,C3,C4,C5")
    p.add_argument("--reps", type=int, default=3)
    args = p.parse_args(argv)
    from paper_1303_0008_gb300 import inputs as I
    from paper_1303_0008_gb300 import mg
    fns = {"C1": c1, "C2": c2, "C3": c3, "C4": c4, "C5": c5}
    for name in args.only.split(","):
        t0 = time.perf_counter()
        out = fns[name](mg, I, args.reps)
        out["wall_clock_s"] = time.perf_counter() - t0
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
