"""One solve of a lognormal workload through the C-ABI, for profiling a kernel.

  python -m paper_1303_0008_gb300.profile_case --n 256 --prec fp64 --rv 8

Runs a single periodic solve (sigma 1.5, seed 1302) to 1e-8 on cuda:0 and prints
its statistics as one JSON line.  Meant to be run under a profiler with a kernel
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
    args = p.parse_args(argv)

    import torch

    from paper_1303_0008_gb300 import inputs, mg

    delta = torch.from_numpy(inputs.lognormal_delta(args.n, args.sigma, 1302)).cuda()
    prec = mg.MG_FP64 if args.prec == "fp64" else mg.MG_MIXED
    g = mg.mg_create_grid(args.n, mg.options(prec=prec))
    try:
        mg.mg_set_stream(g, torch.cuda.current_stream())
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, inputs.alpha_kappa_for_rv(args.rv), 1.0, args.tol)
    finally:
        mg.mg_destroy_grid(g)
    st.pop("hist", None)
    print(json.dumps({"n": args.n, "prec": args.prec, "rv": args.rv, **st}))


if __name__ == "__main__":
    main()
