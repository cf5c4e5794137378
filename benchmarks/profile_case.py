"""One solve of a lognormal workload through the C-ABI, for profiling a kernel.

  python benchmarks/profile_case.py --n 256 --prec fp64 --rv 8
  python benchmarks/profile_case.py --six --prec fp64

Runs a single periodic solve (default sigma 1.5, seed 1302) to 1e-8 on cuda:0, or with
--six the six solves of one step of the benchmark, and prints the statistics of
each solve as one JSON line.  --case selects the other kernel families: a
refined hierarchy, the batched solves, or particle assignment with refinement.  Meant to be run under a profiler with a kernel
filter (for instance `ncu -k regex:k_smooth_colour64 -s 4 -c 3 ...`): at n = 256
every FP64 array of the finest level is 134 MB, larger than the 126 MB L2, so
DRAM counters describe HBM traffic.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--prec", choices=["fp64", "mixed"], default="fp64")
    p.add_argument("--rv", type=float, default=8.0)
    p.add_argument("--sigma", type=float, default=1.5)
    p.add_argument("--seed", type=int, default=1302)
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--six", action="store_true",
                   help="run the six solves of one benchmark step (128^3 lognormal, "
                        "r_V = 2, 8, 32 cells, both signs) instead of a single solve")
    p.add_argument("--sweep32", type=int, default=0)
    p.add_argument("--opt", default="",
                   help="further options of the solve, 'name=value,...' (e.g. half32=1)")
    p.add_argument("--reps", type=int, default=1, help="solves of the case (solve case)")
    p.add_argument("--galerkin", type=int, default=1,
                   help="coarse-grid correction of the refinement unions (c3 case)")
    p.add_argument("--alpha", type=float, default=None,
                   help="alpha*kappa of the c3 case (default r_V = 8 cells, 0.3)")
    p.add_argument("--variants", default=None,
                   help="';'-separated option sets 'k=v,k=v' tried one after another")
    p.add_argument("--case", choices=["solve", "refined", "batch", "particles", "c3"],
                   default="solve",
                   help="refined: a 128^3 sigma 2.0 domain with two refinement levels "
                        "(alpha*kappa 1e-3); batch: the 64-solve mixed batch; particles: "
                        "TSC assignment of 2^24 particles and the N_pc = 9 criterion at 256^3")
    args = p.parse_args(argv)

    import torch

    from paper_1303_0008_gb300 import inputs, mg

    if args.case != "solve":
        return other_case(args, torch, inputs, mg)
    prec = mg.MG_FP64 if args.prec == "fp64" else mg.MG_MIXED
    if args.six:
        w = inputs.workload_lognormal_sweep(128, 1.5, 1302)
        delta = torch.from_numpy(w["delta"]).cuda()
        solves = w["solves"]
        n = 128
    else:
        delta = torch.from_numpy(inputs.lognormal_delta(args.n, args.sigma, args.seed)).cuda()
        solves = [{"alpha": inputs.alpha_kappa_for_rv(args.rv), "kappa": 1.0, "branch": 0}]
        n = args.n
    extra = {}
    for kv in filter(None, args.opt.split(",")):
        k, v = kv.split("=")
        extra[k] = float(v) if ("." in v or "e" in v) else int(v)
    g = mg.mg_create_grid(n, mg.options(prec=prec, sweep32=args.sweep32, **extra))
    out = []
    variants = [dict(kv.split("=") for kv in v.split(",") if kv)
                for v in args.variants.split(";")] if args.variants else [{}]
    try:
        mg.mg_set_stream(g, torch.cuda.current_stream())
        mg.mg_set_density(g, 0, -1, delta)
        zero = torch.zeros_like(delta)
        base = mg.mg_get_options(g)
        for var in variants:
            opt = mg.mg_get_options(g)
            for k in mg.options_dict(base):
                setattr(opt, k, getattr(base, k))
            for k, v in var.items():
                setattr(opt, k, float(v) if ("." in v or "e" in v) else int(v))
            mg.mg_set_options(g, opt)
            for s in solves * args.reps:
                mg.mg_set_field(g, 0, -1, zero)
                st = mg.mg_solve(g, s["branch"], s["alpha"], s["kappa"], args.tol, check=False)
                st.pop("hist", None)
                st["variant"] = var
                out.append(st)
    finally:
        mg.mg_destroy_grid(g)
    for st in out:
        print(json.dumps({"n": n, "prec": args.prec, **st}))


def other_case(args, torch, inputs, mg):
    import time

    import numpy as np
    if args.case == "c3":
        # the 256^3 domain with two refinement levels (sigma 2, seed 1303)
        h = inputs.refined_hierarchy(256, 2.0, 1303)
        alpha = args.alpha if args.alpha is not None else inputs.alpha_kappa_for_rv(8.0)
        g = mg.mg_create_grid(256, mg.options(patch_galerkin=args.galerkin))
        try:
            mg.mg_set_density(g, 0, -1, h["delta0"])
            for lvl, L in enumerate(h["levels"], start=1):
                mg.mg_add_patches(g, lvl, L["origins"])
                mg.mg_set_density(g, lvl, -1, np.ascontiguousarray(L["delta"]))
            out = []
            variants = [dict(kv.split("=") for kv in v.split(",") if kv)
                        for v in args.variants.split(";")] if args.variants else [{}, {}]
            for rep, var in enumerate(variants):
                opt = mg.mg_get_options(g)
                for k, v in var.items():
                    setattr(opt, k, type(getattr(opt, k))(float(v)) if "." in v or "e" in v
                            else int(v))
                mg.mg_set_options(g, opt)
                zero = np.zeros_like(h["delta0"])
                mg.mg_set_field(g, 0, -1, zero)
                for lvl in range(1, len(h["levels"]) + 1):
                    mg.mg_set_field(g, lvl, -1, None)   # start from the level below
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = mg.mg_solve(g, 0, alpha, 1.0, args.tol, check=False)
                torch.cuda.synchronize()
                wall = time.perf_counter() - t0
                lv = [mg.mg_get_level_stats(g, lvl) for lvl in (1, 2)]
                out.append({"rep": rep, "variant": var, "rc": st["rc"], "wall_s": wall,
                            "domain": {"cycles": st["cycles"], "wall_s": st["wall_s"]},
                            "levels": [{"cycles": s["cycles"], "status": s["status"],
                                        "res": s["res"], "wall_s": s["wall_s"],
                                        "hist": s["hist"][:60]} for s in lv]})
        finally:
            mg.mg_destroy_grid(g)
        for o in out:
            print(json.dumps({"case": "c3", "galerkin": args.galerkin, "alpha": alpha,
                              "patches": [len(L["origins"]) for L in h["levels"]], **o}))
    elif args.case == "refined":
        h = inputs.refined_hierarchy(128, 2.0, 1303)
        g = mg.mg_create_grid(128)
        try:
            mg.mg_set_density(g, 0, -1, h["delta0"])
            for lvl, L in enumerate(h["levels"], start=1):
                mg.mg_add_patches(g, lvl, L["origins"])
                mg.mg_set_density(g, lvl, -1, np.ascontiguousarray(L["delta"]))
            st = mg.mg_solve(g, 0, 1e-3, 1.0, args.tol)
            levels = [mg.mg_get_level_stats(g, lvl)["cycles"] for lvl in (1, 2)]
        finally:
            mg.mg_destroy_grid(g)
        print(json.dumps({"case": "refined", "domain_cycles": st["cycles"], "level_cycles": levels,
                          "patches": [len(L["origins"]) for L in h["levels"]]}))
    elif args.case == "batch":
        w = inputs.workload_batch(64)
        g = mg.mg_create_batch([s["n"] for s in w], mg.options(prec=mg.MG_MIXED))
        try:
            for k, s in enumerate(w):
                mg.mg_set_density(g, 0, k, inputs.lognormal_delta(s["n"], s["sigma"], s["seed"]))
            rc, stats = mg.mg_solve_batch(g, [s["branch"] for s in w], [s["alpha"] for s in w],
                                          [s["kappa"] for s in w], args.tol)
        finally:
            mg.mg_destroy_grid(g)
        print(json.dumps({"case": "batch", "rc": rc, "max_outer": max(s["outer"] for s in stats)}))
    else:
        n, count = 256, 1 << 24
        gen = torch.Generator(device="cuda").manual_seed(1307)
        pos = torch.rand((3, count), generator=gen, dtype=torch.float64, device="cuda")
        pos[:, : count // 2] = torch.remainder(
            0.5 + 0.03 * torch.randn((3, count // 2), generator=gen, dtype=torch.float64,
                                     device="cuda"), 1.0)
        g = mg.mg_create_grid(n)
        try:
            mg.mg_assign_density(g, 0, pos.contiguous())
            org = mg.mg_refine_blocks(g, 0, 9.0, 1.0 / count)
            mg.mg_add_patches(g, 1, org)
            mg.mg_assign_density(g, 1, pos.contiguous())
        finally:
            mg.mg_destroy_grid(g)
        print(json.dumps({"case": "particles", "patches": int(len(org))}))


if __name__ == "__main__":
    main()
