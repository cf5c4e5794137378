"""One solve of a lognormal workload through the C-ABI, for profiling a kernel.

  python -m paper_1303_0008_gb300.profile_case --n 256 --prec fp64 --rv 8
  python -m paper_1303_0008_gb300.profile_case --six --prec fp64

Runs a single periodic solve (sigma 1.5, seed 1302) to 1e-8 on cuda:0, or with
--six the six solves of one step of the benchmark, and prints the statistics of
each solve as one JSON line.  Meant to be run under a profiler with a kernel
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
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--six", action="store_true",
                   help="run the six solves of one benchmark step (128^3 lognormal, "
                        "r_V = 2, 8, 32 cells, both signs) instead of a single solve")
    p.add_argument("--sweep32", type=int, default=0)
    args = p.parse_args(argv)

    import torch

    from paper_1303_0008_gb300 import inputs, mg

    prec = mg.MG_FP64 if args.prec == "fp64" else mg.MG_MIXED
    if args.six:
        w = inputs.workload_lognormal_sweep(128, 1.5, 1302)
        delta = torch.from_numpy(w["delta"]).cuda()
        solves = w["solves"]
        n = 128
    else:
        delta = torch.from_numpy(inputs.lognormal_delta(args.n, args.sigma, 1302)).cuda()
        solves = [{"alpha": inputs.alpha_kappa_for_rv(args.rv), "kappa": 1.0, "branch": 0}]
        n = args.n
    g = mg.mg_create_grid(n, mg.options(prec=prec, sweep32=args.sweep32))
    out = []
    try:
        mg.mg_set_stream(g, torch.cuda.current_stream())
        mg.mg_set_density(g, 0, -1, delta)
        zero = torch.zeros_like(delta)
        for s in solves:
            mg.mg_set_field(g, 0, -1, zero)
            st = mg.mg_solve(g, s["branch"], s["alpha"], s["kappa"], args.tol)
            st.pop("hist", None)
            out.append(st)
    finally:
        mg.mg_destroy_grid(g)
    for st in out:
        print(json.dumps({"n": n, "prec": args.prec, **st}))


if __name__ == "__main__":
    main()
