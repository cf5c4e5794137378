"""Benchmark of the DGP scalar-field FAS solver on one GB300 per rank.

Workload: the 128^3 periodic lognormal field (sigma = 1.5, P(k) ~ k^-2, seed
1302) with six (alpha, kappa) pairs: Vainshtein radius 2, 8 and 32 cells, each
with the sign of alpha (and kappa) flipped.  One step solves all six from a zero
initial guess to max|d - lambda| < 1e-8 with the FP64 path; `value` is solves
per second over all ranks (each rank solves its own copy: weak scaling, no
collective on the data path).  The mixed-precision path is timed on the same
workload and reported under "mixed".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle (one of the six solves per step, cycling)
on the host cores of rank 0 and prints the same JSON line with "impl":
"reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("smoother cell-updates/s & FAS solves/s to residual 1e-8 (FP64 vs mixed), "
          "% HBM roofline")
N = 128
SIGMA = 1.5
SEED = 1302
TOL = 1e-8
# FP64 operations of one smoother cell update (FMA counted as 2, sqrt as 1): face
# sums 3, Sigma_d 22 (A: 3 differences + 5; B: 9 cross-difference sums + 5),
# q 4, sqrt 1, root 2, update 6.
FLOP_PER_CELL_FP64 = 38
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070   # SMs x DFMA/clk x flop/DFMA x max GHz
L2_FLUSH_BYTES = 256 << 20


def workload():
    from paper_1303_0008_gb300 import inputs
    return inputs.workload_lognormal_sweep(N, SIGMA, SEED)


def world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value: float, group=None) -> float:
    """Largest `value` over the ranks of the default process group (itself if none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(value: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        mhz = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2])
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _definition(text: str, head: str) -> str:
    """The source of the function whose definition starts with `head` (to its
    matching closing brace)."""
    i = text.find(head)
    if i < 0:
        return ""
    j = text.index("{", i)
    depth = 0
    for k in range(j, len(text)):
        depth += {"{": 1, "}": -1}.get(text[k], 0)
        if depth == 0:
            return text[i:k + 1]
    return text[i:]


def kernel_source_hash():
    """Hash of the source that defines the finest-level smoother and its launch: the
    two headers its body comes from, plus the kernel, its launcher and the block-size
    rule in mg_fp64.cu (other kernels in that file do not change it)."""
    csrc = os.path.join(ROOT, "paper_1303_0008_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("mg_bodies64.cuh", "mg_common.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    fp64 = open(os.path.join(csrc, "mg_fp64.cu")).read()
    for head in ("__global__ void __launch_bounds__(256) k_smooth_colour64(",
                 "int tpb_for(long long items)", "void launch_smooth64("):
        part = _definition(fp64, head)
        assert part, head
        h.update(part.encode())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    data = json.load(open(path))
    ent = data.get(kernel)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("bytes_per_launch_full_size")


def run_ours(args):
    import numpy as np
    import torch

    from paper_1303_0008_gb300 import mg

    rank, ws, local = world()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    w = workload()
    delta_np = w["delta"]
    solves = w["solves"]
    delta = torch.from_numpy(delta_np).cuda()
    zero = torch.zeros_like(delta)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def make(prec, time_kernels):
        g = mg.mg_create_grid(N, mg.options(prec=prec, time_kernels=time_kernels))
        mg.mg_set_stream(g, stream)
        mg.mg_set_density(g, 0, -1, delta)
        return g

    def step(g, stats_out):
        for s in solves:
            mg.mg_set_field(g, 0, -1, zero)
            st = mg.mg_solve(g, s["branch"], s["alpha"], s["kappa"], TOL)
            stats_out.append(st)

    def timed(g, steps, warmup):
        for _ in range(warmup):
            step(g, [])
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        per_step = []
        stats = []
        for _ in range(steps):
            flush.zero_()                     # L2 flush: write a buffer larger than L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(g, stats)
            e1.record(stream)
            e1.synchronize()
            per_step.append(e0.elapsed_time(e1))
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        return per_step, stats

    # the finest-level smoother is timed live by events around the first colour stage
    # of every smoothing call (2 of its 16 launches per V-cycle): each event removes
    # the programmatic overlap of the two launches around it
    g64 = make(mg.MG_FP64, 2)
    with ClockSampler(local) as clk:
        per_step, stats = timed(g64, args.steps, args.warmup)
    clocks = clk.summary()
    total_ms = max_over_ranks(sum(per_step))
    solves_done = sum_over_ranks(len(solves) * args.steps)
    value = solves_done / (total_ms * 1e-3)

    # dominant kernel: the finest-level FP64 smoother (one colour stage per launch)
    k_ms = sum(s["kernel_ms"] for s in stats)
    k_n = sum(s["kernel_launches"] for s in stats)
    k_cells = sum(s["kernel_cells"] for s in stats)
    avg_ms = k_ms / max(k_n, 1)
    cells_per_launch = k_cells / max(k_n, 1)
    achieved = FLOP_PER_CELL_FP64 * cells_per_launch / (avg_ms * 1e-3) / 1e12
    launches = sum(s["launches"] for s in stats)
    cycles = [s["cycles"] for s in stats[:len(solves)]]

    # mixed precision on the same workload
    gmx = make(mg.MG_MIXED, 0)
    per_step_m, stats_m = timed(gmx, args.steps, args.warmup)
    total_m = max_over_ranks(sum(per_step_m))
    value_m = solves_done / (total_m * 1e-3)

    # end to end through the C-ABI with pinned host buffers
    host_delta = torch.from_numpy(delta_np).pin_memory()
    host_zero = torch.zeros(delta_np.shape, dtype=torch.float64).pin_memory()
    host_out = torch.empty(delta_np.shape, dtype=torch.float64).pin_memory()
    ge = mg.mg_create_grid(N, mg.options())
    mg.mg_set_stream(ge, stream)

    def e2e_step():
        mg.mg_set_density(ge, 0, -1, host_delta)
        for s in solves:
            mg.mg_set_field(ge, 0, -1, host_zero)
            mg.mg_solve(ge, s["branch"], s["alpha"], s["kappa"], TOL)
            mg.mg_get_field(ge, 0, -1, host_out)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = max_over_ranks(sum(e2e_ms))
    cell_bytes = delta_np.size * 8
    e2e = {"value": solves_done / (e2e_total * 1e-3), "unit": "solves/s",
           "h2d_bytes_per_step": cell_bytes * (1 + len(solves)),
           "d2h_bytes_per_step": cell_bytes * len(solves)}
    for h in (g64, gmx, ge):
        mg.mg_destroy_grid(h)

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "128^3 periodic lognormal delta (sigma 1.5, P(k)~k^-2, seed 1302), "
                               "6 solves: r_V = 2, 8, 32 cells x both signs of alpha, FP64, "
                               "max|d - lambda| < 1e-8 from phi = 0",
                   "n": N, "solves_per_step": len(solves), "tol": TOL, "precision": "fp64",
                   "nu_pre": 2, "nu_post": 2, "coarsest": 4,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "cycles_per_solve": cycles},
        "roofline": {"bound": "alu", "kernel": "k_smooth_colour64 (finest level)",
                     "achieved": achieved, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                     "frac": achieved / (FP64_PEAK_GFLOPS / 1e3),
                     "peak_source": "derived FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                     "flop_per_cell": FLOP_PER_CELL_FP64, "cells_per_launch": cells_per_launch,
                     "avg_launch_us": avg_ms * 1e3, "launches_timed": k_n,
                     "traffic": traffic_per_launch("k_smooth_colour64")},
        "smoother": {"fp64_cell_updates_per_s": cells_per_launch / (avg_ms * 1e-3)},
        "mixed": {"value": value_m, "unit": "solves/s", "ms_per_step": total_m / args.steps,
                  "speedup_vs_fp64": value_m / value,
                  "outer_per_solve": [s["outer"] for s in stats_m[:len(solves)]],
                  "inner_cycles_per_solve": [s["cycles"] for s in stats_m[:len(solves)]]},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# the CPU oracle
# ---------------------------------------------------------------------------
def cpu_baseline(w, count):
    """The oracle as it stands, single thread, on `count` of the six solves."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    for i in range(count):
        s = w["solves"][(2 + i) % len(w["solves"])]
        delta, _ = O.density_floor(w["delta"], s["alpha"], s["kappa"])
        O.fas_solve(delta, s["alpha"], s["kappa"], s["branch"], tol=TOL)
    dt = time.perf_counter() - t0
    return {"value": count / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{count} of the 6 solves of the 128^3 workload (r_V = 8 cells first), "
                      f"single-threaded lexicographic FAS, {dt:.1f} s"}


def run_reference(args):
    rank, ws, _ = world()
    if rank != 0:
        return
    w = workload()
    from oracle import oracle as O
    times = []
    k = 0
    for it in range(args.warmup + args.steps):
        s = w["solves"][k % len(w["solves"])]
        k += 1
        t0 = time.perf_counter()
        # the system the GPU solves: source held at the real-root bound (default guard)
        delta, _ = O.density_floor(w["delta"], s["alpha"], s["kappa"])
        O.fas_solve(delta, s["alpha"], s["kappa"], s["branch"], tol=TOL)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "128^3 periodic lognormal delta (sigma 1.5, P(k)~k^-2, "
                                   "seed 1302), 6 solves to 1e-8; one solve per step"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": "one of the six 128^3 solves per step, cycling"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    args = p.parse_args(argv)
    if args.warmup < 3:
        p.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
