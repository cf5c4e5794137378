"""Benchmark of the DGP scalar-field FAS solver on one GB300 per rank.

Workload: the 512^3 periodic lognormal field (sigma 2.0, P(k) ~ k^-2, seed 1304),
normal branch, alpha*kappa = 2.4 (Vainshtein radius 16 cells of the reference
top-hat), solved from phi = 0 to max|d - lambda| < 1e-8.  One step is one solve.
`value` is FP64 solves per second over all ranks (each rank solves its own copy:
weak scaling, no collective on the data path); the mixed-precision path (FP32
correction cycles inside FP64 defect correction) is timed on the same workload
and reported under "mixed".  The 128^3 six-solve workload (sigma 1.5, seed 1302,
r_V = 2, 8, 32 cells, both signs) is reported under "secondary".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle's four-colour OpenMP build on the host
cores of rank 0 (a bounded sample of each solve, scaled to solves/s) and prints
the same JSON line with "impl": "reference".
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
N = 512
SIGMA = 2.0
SEED = 1304
R_V = 16.0
TOL = 1e-8
WORKLOAD = ("512^3 periodic lognormal delta (sigma 2.0, P(k)~k^-2, seed 1304), normal branch, "
            "alpha*kappa = 2.4 (r_V = 16 cells), max|d - lambda| < 1e-8 from phi = 0; "
            "FP64 vs mixed precision")
# FP64 operations of one smoother cell update (FMA counted as 2, sqrt as 1): face
# sums 3, Sigma_d 22 (A: 3 differences + 5; B: 9 cross-difference sums + 5),
# q 4, sqrt 1, root 2, update 6.
FLOP_PER_CELL_FP64 = 38
# bytes of one FP32 correction-smoother cell update: e, phi0, q0 and g read, e written
BYTES_PER_CELL_FP32 = 20
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070   # SMs x DFMA/clk x flop/DFMA x max GHz
HBM_FALLBACK_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
# the secondary workload
N2, SIGMA2, SEED2 = 128, 1.5, 1302


def workload():
    from paper_1303_0008_gb300 import inputs
    return {"delta": inputs.lognormal_delta(N, SIGMA, SEED),
            "alpha": inputs.alpha_kappa_for_rv(R_V), "kappa": 1.0, "branch": 0}


def workload_secondary():
    from paper_1303_0008_gb300 import inputs
    return inputs.workload_lognormal_sweep(N2, SIGMA2, SEED2)


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


# source that determines each roofline kernel's traffic: the headers of its body
# and the definitions (kernel, launcher, block-size rule) in its translation unit
_KERNEL_SOURCES = {
    "k_half32": (("mg_bodies32.cuh", "mg_common.cuh"), "mg_halfsweep32.cu",
                 ("__global__ void __launch_bounds__(hsw::threads<N>()) k_half32(",
                  "void launch_half_sweep32(")),
    "k_smooth_colour64": (("mg_bodies64.cuh", "mg_common.cuh"), "mg_fp64.cu",
                          ("__global__ void __launch_bounds__(256) k_smooth_colour64(",
                           "int tpb_for(long long items)", "void launch_smooth64(")),
    "k_smooth_colour32_n": (("mg_bodies32.cuh", "mg_common.cuh"), "mg_mixed.cu",
                            ("__global__ void __launch_bounds__(256) k_smooth_colour32_n(",
                             "__device__ __forceinline__ long long colour_cell(",
                             "static void launch_colour32_n(",
                             "  void smooth(int l, int sweeps) const {")),
    "k_smooth_slab32": (("mg_bodies32.cuh", "mg_common.cuh"), "mg_mixed.cu",
                        ("__global__ void __launch_bounds__(256) k_smooth_slab32(",
                         "  void slab_sweeps(int l, int sweeps, bool co, EventPairs* t) const {"),
                        (("mg_internal.h", "inline void slab_range("),)),
}


def kernel_source_hash(kernel: str = "k_smooth_colour64"):
    """Hash of the source that defines `kernel` and its launch: the headers its body
    comes from, plus the kernel and its launcher in its translation unit (other
    kernels in that file do not change it)."""
    headers, unit, heads, *more = _KERNEL_SOURCES[kernel]
    csrc = os.path.join(ROOT, "paper_1303_0008_gb300", "csrc")
    h = hashlib.sha256()
    for f in headers:
        h.update(open(os.path.join(csrc, f), "rb").read())
    parts = [(unit, head) for head in heads] + list(more[0] if more else ())
    for f, head in parts:
        part = _definition(open(os.path.join(csrc, f)).read(), head)
        assert part, head
        h.update(part.encode())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel: str, cells_per_launch: float, **launch):
    """DRAM bytes per launch of `kernel` at `cells_per_launch` cell updates, from the
    committed ncu record, if it was taken on the current kernel source and with the
    launch parameters given (for instance tile32=4), else None.  The record was taken
    on a grid whose arrays exceed L2, so the traffic grows in proportion to the cells
    a launch updates."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    ent = json.load(open(path)).get(kernel)
    if not ent or ent.get("source_hash") != kernel_source_hash(kernel):
        return None
    # records taken at several launch shapes: {"by_tile32": {"4": {...}, ...}}
    for k, v in launch.items():
        sub = ent.get("by_" + k)
        if sub is not None:
            ent = dict(ent, **sub.get(str(v), {"bytes_per_launch": None}), **{k: v})
    if (not ent.get("bytes_per_launch") or not ent.get("cells_per_launch") or
            any(ent.get(k) != v for k, v in launch.items())):
        return None
    return ent["bytes_per_launch"] * cells_per_launch / ent["cells_per_launch"]


def _peaks():
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(pk)) if os.path.exists(pk) else {}


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
    delta = torch.from_numpy(delta_np).cuda()
    zero = torch.zeros_like(delta)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def make(prec, time_kernels, n=N, dev=delta):
        g = mg.mg_create_grid(n, mg.options(prec=prec, time_kernels=time_kernels))
        mg.mg_set_stream(g, stream)
        mg.mg_set_density(g, 0, -1, dev)
        return g

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(step, steps, warmup):
        for _ in range(warmup):
            step([])
        barrier()
        per_step, stats = [], []
        for _ in range(steps):
            flush.zero_()                     # L2 flush: write a buffer larger than L2
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(stats)
            e1.record(stream)
            e1.synchronize()
            per_step.append(e0.elapsed_time(e1))
        barrier()
        return per_step, stats

    def solve_step(g):
        def step(out):
            mg.mg_set_field(g, 0, -1, zero)
            out.append(mg.mg_solve(g, w["branch"], w["alpha"], w["kappa"], TOL))
        return step

    # Sweep counts (and for the mixed path inner cycles and the FP32 sweep form)
    # come from the library's autotuner, run on this workload before the timed
    # region.  The finest-level smoother is then timed live by events around the
    # first launch of every smoothing call; each event removes the programmatic
    # overlap of the two launches around it.
    tuned = {}

    def tune(prec):
        g = make(prec, 2)
        mg.mg_set_field(g, 0, -1, zero)
        t0 = time.perf_counter()
        if args.no_tune:
            best = mg.mg_get_options(g)
        else:
            best, _ = mg.mg_autotune(g, w["branch"], w["alpha"], w["kappa"], TOL, None,
                                     use_cache=False)
        tuned["fp64" if prec == mg.MG_FP64 else "mixed"] = {
            "nu_pre": best.nu_pre, "nu_post": best.nu_post, "inner_cycles": best.inner_cycles,
            "half32": best.half32, "slab32": best.slab32, "tile32": best.tile32,
            "tune_s": time.perf_counter() - t0}
        return g, best

    g64, best64 = tune(mg.MG_FP64)
    gmx, bestmx = tune(mg.MG_MIXED)
    with ClockSampler(local) as clk:
        per_step, stats = timed(solve_step(g64), args.steps, args.warmup)
        per_step_m, stats_m = timed(solve_step(gmx), args.steps, args.warmup)
    mg.mg_destroy_grid(g64)
    mg.mg_destroy_grid(gmx)
    clocks = clk.summary()
    total_ms = max_over_ranks(sum(per_step))
    total_m = max_over_ranks(sum(per_step_m))
    solves_done = sum_over_ranks(args.steps)
    value = solves_done / (total_ms * 1e-3)
    value_m = solves_done / (total_m * 1e-3)

    def kernel_rate(st):
        ms = sum(s["kernel_ms"] for s in st)
        n = sum(s["kernel_launches"] for s in st)
        cells = sum(s["kernel_cells"] for s in st)
        avg_s = ms * 1e-3 / max(n, 1)
        per = cells / max(n, 1)
        return avg_s, per, n

    peaks = _peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "MEASURED_PEAKS.json hbm_gbs (STREAM-style copy), of measured"
    if not hbm_peak:
        hbm_peak, peak_src = HBM_FALLBACK_GBS, "fallback 6.8 TB/s"
    # FP32 correction smoother, HBM-bound: algorithmic bytes per launch / event time;
    # a timed unit is one colour stage, one half sweep (two colours), or one whole
    # sweep of slab launches
    avg32, cells32, n32 = kernel_rate(stats_m)
    ach32 = BYTES_PER_CELL_FP32 * cells32 / avg32 / 1e9
    slab = bestmx.slab32 if (not bestmx.half32 and N >= 256 and N % max(bestmx.slab32, 1) == 0) else 0
    k32 = "k_half32" if bestmx.half32 else "k_smooth_slab32" if slab else "k_smooth_colour32_n"
    traffic32 = (traffic_per_launch(k32, cells32, tile32=bestmx.tile32)
                 if k32 == "k_smooth_colour32_n" else traffic_per_launch(k32, cells32))
    # FP64 smoother, bound by the FP64 pipe
    avg64, cells64, n64 = kernel_rate(stats)
    ach64 = FLOP_PER_CELL_FP64 * cells64 / avg64 / 1e12
    traffic64 = traffic_per_launch("k_smooth_colour64", cells64)
    roofline = {
        "bound": "hbm",
        "kernel": (f"k_half32<{N}> (finest FP32 half sweep, two colours, mixed)" if bestmx.half32
                   else f"k_smooth_slab32<{N}> (finest FP32 sweep in slabs of {slab} planes, "
                        f"{4 * N // max(slab, 1)} launches; one timed unit is a whole sweep)" if slab
                   else f"k_smooth_colour32_n<{N}> (finest FP32 colour stage, mixed; CTA tile "
                        f"32 x {8 // bestmx.tile32} rows x {bestmx.tile32} planes)" if bestmx.tile32
                   else f"k_smooth_colour32_n<{N}> (finest FP32 colour stage, mixed)"),
        "achieved": ach32, "peak": hbm_peak, "unit": "GB/s", "frac": ach32 / hbm_peak,
        "traffic": traffic32, "peak_source": peak_src,
        "bytes_per_cell": BYTES_PER_CELL_FP32, "cells_per_launch": cells32,
        "avg_launch_us": avg32 * 1e6, "launches_timed": n32,
        "traffic_vs_algorithmic": (traffic32 / (BYTES_PER_CELL_FP32 * cells32)
                                   if traffic32 else None),
        "fp64": {"bound": "alu", "kernel": f"k_smooth_colour64 (finest FP64 colour stage)",
                 "achieved": ach64, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                 "frac": ach64 / (FP64_PEAK_GFLOPS / 1e3),
                 "peak_source": "derived FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                 "flop_per_cell": FLOP_PER_CELL_FP64, "cells_per_launch": cells64,
                 "avg_launch_us": avg64 * 1e6, "launches_timed": n64, "traffic": traffic64,
                 "hbm_frac_algorithmic": 24 * cells64 / avg64 / 1e9 / hbm_peak},
    }

    # the secondary six-solve 128^3 workload (its arrays fit in L2)
    w2 = workload_secondary()
    d2 = torch.from_numpy(w2["delta"]).cuda()
    z2 = torch.zeros_like(d2)
    sec = {}
    for name, prec in (("fp64", mg.MG_FP64), ("mixed", mg.MG_MIXED)):
        g2 = make(prec, 0, N2, d2)

        def step2(out, g2=g2):
            for s in w2["solves"]:
                mg.mg_set_field(g2, 0, -1, z2)
                out.append(mg.mg_solve(g2, s["branch"], s["alpha"], s["kappa"], TOL))
        ps, st2 = timed(step2, args.steps, args.warmup)
        mg.mg_destroy_grid(g2)
        sec[name] = sum_over_ranks(len(w2["solves"]) * args.steps) / (max_over_ranks(sum(ps)) * 1e-3)
    del d2, z2

    # end to end through the C-ABI with pinned host buffers: density in, initial
    # guess in, solve, field out, every step
    host_delta = torch.from_numpy(delta_np).pin_memory()
    host_zero = torch.zeros(delta_np.shape, dtype=torch.float64).pin_memory()
    host_out = torch.empty(delta_np.shape, dtype=torch.float64).pin_memory()
    ge = mg.mg_create_grid(N, mg.options(nu_pre=best64.nu_pre, nu_post=best64.nu_post))
    mg.mg_set_stream(ge, stream)

    phases = {"set_density": 0.0, "set_field": 0.0, "solve": 0.0, "get_field": 0.0}

    def e2e_step(acc=None):
        # each call returns after its work is done (the copies synchronise the
        # stream, the solve reads its residuals back), so host stamps split the step
        t = [time.perf_counter()]
        mg.mg_set_density(ge, 0, -1, host_delta)
        t.append(time.perf_counter())
        mg.mg_set_field(ge, 0, -1, host_zero)
        t.append(time.perf_counter())
        mg.mg_solve(ge, w["branch"], w["alpha"], w["kappa"], TOL)
        t.append(time.perf_counter())
        mg.mg_get_field(ge, 0, -1, host_out)
        t.append(time.perf_counter())
        if acc is not None:
            for name, a, b in zip(acc, t, t[1:]):
                acc[name] += (b - a) * 1e3

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    e2e_ms = []
    with ClockSampler(local) as clk_e2e:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step(phases)
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    barrier()
    mg.mg_destroy_grid(ge)
    e2e_total = max_over_ranks(sum(e2e_ms))
    cell_bytes = delta_np.size * 8
    e2e = {"value": solves_done / (e2e_total * 1e-3), "unit": "solves/s",
           "h2d_bytes_per_step": 2 * cell_bytes, "d2h_bytes_per_step": cell_bytes,
           "ms_per_step": e2e_total / args.steps, "clocks": clk_e2e.summary(),
           "phase_ms_per_step": {k: v / args.steps for k, v in phases.items()}}

    s0, m0 = stats[0], stats_m[0]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "sigma": SIGMA, "seed": SEED,
                   "alpha_kappa": w["alpha"], "solves_per_step": 1, "tol": TOL,
                   "precision": "fp64 (value); mixed under 'mixed'",
                   "tuned": tuned, "coarsest": 4,
                   "l2": "flushed before every timed step (256 MiB write); every 512^3 "
                         "array (1.07 GB FP64, 0.54 GB FP32) is larger than L2",
                   "cycles_per_solve": s0["cycles"], "res": s0["res"],
                   "floored_cells": s0["guard_hits"],
                   "floored_fraction": s0["guard_hits"] / float(N ** 3)},
        "roofline": roofline,
        "smoother": {"fp64_cell_updates_per_s": cells64 / avg64,
                     "fp32_cell_updates_per_s": cells32 / avg32},
        "mixed": {"value": value_m, "unit": "solves/s", "ms_per_step": total_m / args.steps,
                  "speedup_vs_fp64": value_m / value, "outer_per_solve": m0["outer"],
                  "inner_cycles_per_solve": m0["cycles"], "res": m0["res"],
                  "floored_cells": m0["guard_hits"]},
        "secondary": {"workload": "128^3 lognormal (sigma 1.5, seed 1302), six solves "
                                  "(r_V = 2, 8, 32 cells x both signs) per step to 1e-8",
                      "fp64_solves_per_s": sec["fp64"], "mixed_solves_per_s": sec["mixed"]},
        "e2e": e2e,
        "gpu_launches": sum(s["launches"] for s in stats),
        "gpu_launches_mixed": sum(s["launches"] for s in stats_m),
        "clocks": clocks,
        "hbm_peak_gbs": hbm_peak,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, s0["cycles"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# the CPU oracle (four-colour OpenMP build on all host cores)
# ---------------------------------------------------------------------------
SAMPLE_CYCLES = 2


def host_cores():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("CPU(s):"):
                return int(line.split(":")[1])
    except OSError:
        pass
    return os.cpu_count()


def oracle_sample(w, delta_floor):
    """One bounded sample of an oracle solve of the workload: the set-up alone
    (allocation, restriction of delta, first residual) and then the set-up plus
    SAMPLE_CYCLES V-cycles from phi = 0, on all host cores.  The solve time is
    estimated as set-up + cycles needed x time per cycle, the cycles needed being
    extrapolated from the sampled residual reduction."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    _, s0 = O.fas_solve_colour(delta_floor, w["alpha"], w["kappa"], w["branch"], tol=TOL,
                               max_cycles=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, st = O.fas_solve_colour(delta_floor, w["alpha"], w["kappa"], w["branch"], tol=TOL,
                               max_cycles=SAMPLE_CYCLES)
    t_run = time.perf_counter() - t0
    t_cycle = max(t_run - t_setup, 1e-9) / max(st["cycles"], 1)
    res0, resk = st["res0"], st["res"]
    if st["cycles"] and resk < res0:
        rate = (resk / res0) ** (1.0 / st["cycles"])
        need = max(st["cycles"], math.ceil(math.log(TOL / res0) / math.log(rate)))
    else:
        need = None
    est = t_setup + need * t_cycle if need else None
    return {"t_setup": t_setup, "t_cycle": t_cycle, "cycles_needed": need, "solve_s": est,
            "threads": st["threads"], "res0": res0, "res_sampled": resk,
            "sample_s": t_setup + t_run}


def cpu_baseline(w, gpu_cycles):
    import numpy as np
    from oracle import oracle as O
    fl, _ = O.density_floor(w["delta"], w["alpha"], w["kappa"])
    smp = oracle_sample(w, fl)
    t0 = time.perf_counter()
    _, threads = O.colour_sweeps(np.zeros_like(fl), fl, w["alpha"], w["kappa"], w["branch"],
                                 sweeps=1)
    sweep_rate = fl.size / (time.perf_counter() - t0)
    return {"value": 1.0 / smp["solve_s"] if smp["solve_s"] else None, "unit": "solves/s",
            "cores": smp["threads"], "host_cpus_lscpu": host_cores(),
            "kind": "oracle (four-colour Newton-Gauss-Seidel FAS, OpenMP on all host cores)",
            "sample": (f"set-up plus {SAMPLE_CYCLES} V-cycles of the {N}^3 solve from phi = 0 "
                       f"({smp['sample_s']:.1f} s); solve time = set-up {smp['t_setup']:.2f} s + "
                       f"{smp['cycles_needed']} cycles x {smp['t_cycle']:.2f} s, the cycle count "
                       f"extrapolated from the sampled residual drop "
                       f"{smp['res0']:.3g} -> {smp['res_sampled']:.3g} (the GPU FP64 solve took "
                       f"{gpu_cycles} cycles)"),
            "sweep_cell_updates_per_s": sweep_rate, "sweep_threads": threads}


def run_reference(args):
    """The oracle on the host cores of rank 0.  The first warm-up step takes the full
    sample of oracle_sample (set-up time and the extrapolated cycle count); the other
    warm-up steps repeat the set-up only.  Each timed step runs the set-up and one
    V-cycle from phi = 0, and is scaled to one solve by the cycles still needed at
    the time per cycle it measured."""
    rank, ws, _ = world()
    if rank != 0:
        return
    from oracle import oracle as O
    w = workload()
    fl, hits = O.density_floor(w["delta"], w["alpha"], w["kappa"])
    first = oracle_sample(w, fl)
    need, t_setup = first["cycles_needed"], first["t_setup"]
    for _ in range(args.warmup - 1):
        O.fas_solve_colour(fl, w["alpha"], w["kappa"], w["branch"], tol=TOL, max_cycles=0)
    est = []
    threads = first["threads"]
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, st = O.fas_solve_colour(fl, w["alpha"], w["kappa"], w["branch"], tol=TOL,
                                   max_cycles=1)
        t_step = time.perf_counter() - t0
        threads = st["threads"]
        est.append(t_step + (need - 1) * max(t_step - t_setup, 0.0))
    total = sum(est)
    value = len(est) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(est), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "sigma": SIGMA, "seed": SEED,
                       "alpha_kappa": w["alpha"], "tol": TOL, "floored_cells": hits},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads,
                             "host_cpus_lscpu": host_cores(),
                             "kind": "oracle (four-colour Newton-Gauss-Seidel FAS, OpenMP)",
                             "sample": (f"per step: set-up plus one V-cycle of the {N}^3 solve "
                                        f"from phi = 0, scaled to one solve by the {need} "
                                        f"cycles extrapolated from the residual drop of "
                                        f"{SAMPLE_CYCLES} cycles in the first warm-up step "
                                        f"({first['res0']:.3g} -> {first['res_sampled']:.3g})")},
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
    p.add_argument("--no-tune", action="store_true",
                   help="keep the library's default sweep counts instead of autotuning them")
    args = p.parse_args(argv)
    if args.warmup < 3:
        p.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
