#!/usr/bin/env python3
"""Benchmark of the implicit ohmic-dissipation step (Matsumoto 2011, Sec. 2) on one GB300.

Workload: uniform 256^3 periodic unit box, eta = 1e-3 (1 + 999 exp(-|x-c|^2/0.05^2)), B the
curl of a seeded k^-2 random vector potential (rms 1), dt = 100x the explicit limit at the
largest eta, consecutive CN steps each converged to ||R||/||S|| <= 1e-9.  One bench step is
one CN step (source, defect-correction cycles of residual + V-cycle + update).

Metric: cell-steps/s = cells x CN steps / device time.  `value` is the mixed-precision path
(FP32 multigrid, FGMRES-accelerated, inside FP64 iterative refinement; red-black SOR sweeps
with V(3,2) on level 0 and V(1,0) below); the plain FP64 path (the paper's Gauss-Seidel defect
correction), the same with the paper's defect correction in mixed precision, and the
float-float outer residual (OHM_MIXED_FF) and with float-float intermediate residuals checked in
float64 (OHM_MIXED_FF_CHECKED) are reported beside it.  `e2e` repeats the step
through the public API with pinned host buffers.  The oracle (FP64 CPU reference) is timed on
the host cores as `cpu_baseline`, and is the `--impl reference` arm.  `--workload batched512`
and `--workload serving` measure the batched hierarchies and the solve service.
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
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s at 256^3 to rel. residual 1e-9"
UNIT = "cell-steps/s"
L2_BYTES = 129e6


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--size", type=int, default=256, help="cells per axis (multiple of 8)")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--only", choices=["fgmres", "fgmres_ff", "fgmres_ffc", "mixed", "fp64", "fp64_fgmres"], default=None,
                   help="run just this path for a few steps and print its timing (for profiler captures)")
    p.add_argument("--nu", default="3,2", help="pre,post red-black sweeps on level 0")
    p.add_argument("--nu-coarse", default="1,0",
                   help="pre,post sweeps on the grids coarser than level 0 on the headline path (0,0 = as --nu)")
    p.add_argument("--n-coarse", type=int, default=2, help="sweeps on the coarsest grid")
    p.add_argument("--krylov", type=int, default=6, help="FGMRES restart length of the headline path")
    p.add_argument("--omega", type=float, default=1.2,
                   help="relaxation factor of the red-black sweeps on the headline path (1 = the paper's "
                        "Gauss-Seidel, kept by the FP64 and defect-correction comparisons)")
    p.add_argument("--workload", choices=["resistive_bump", "batched512", "serving"], default="resistive_bump",
                   help="resistive_bump: the headline 256^3 line; batched512: 512 independent instances "
                        "(edges 16..64) in batched hierarchies; serving: Poisson request stream through "
                        "the continuous-batching service")
    p.add_argument("--instances", type=int, default=512, help="batched512: number of instances")
    p.add_argument("--no-autotune", action="store_true", help="batched512: keep the default schedule")
    p.add_argument("--batch-krylov", type=int, default=6,
                   help="batched512 / serving: FGMRES restart length of each instance's inner solve (0: defect correction)")
    p.add_argument("--requests", type=int, default=600, help="serving: requests in the stream")
    p.add_argument("--serve-nu-coarse", default="1,1", help="serving: pre,post sweeps on the grids coarser than level 0")
    p.add_argument("--serve-max-batch", type=int, default=2,
                   help="serving: slots per batched hierarchy (a batch steps until its slowest member's step "
                        "converges; with this stream's 100x spread of dt, 2 slots serve faster than 8)")
    p.add_argument("--serve-workers", type=int, default=16, help="serving: batches in flight (host threads, streams)")
    p.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    p.add_argument("--inner-tol", type=float, default=1e-5,
                   help="residual reduction asked of each float32 inner solve (mixed precision)")
    p.add_argument("--batch-nu", default="4,4", help="batched512 without autotuning: pre,post sweeps on level 0")
    p.add_argument("--batch-omega", type=float, default=1.3, help="batched512 without autotuning: relaxation factor")
    p.add_argument("--batch-nu-coarse", default="1,1",
                   help="batched512 without autotuning: pre,post sweeps on the grids coarser than level 0")
    p.add_argument("--batch-n-coarse", type=int, default=4, help="batched512 without autotuning: coarsest sweeps")
    p.add_argument("--no-legs", action="store_true",
                   help="skip the bounded batched and serving legs of the default line")
    p.add_argument("--leg-instances", type=int, default=128, help="batched leg of the default line: instances")
    p.add_argument("--leg-requests", type=int, default=150, help="serving leg of the default line: requests")
    p.add_argument("--cpu-full-step", action="store_true",
                   help="time one complete oracle CN step of the workload on the host cores (minutes at 256^3) "
                        "beside the sampled model of cpu_baseline, print it and exit")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def fp64_peak_tflops(ohm):
    """float64 FMA rate of this GPU measured by the library's DFMA probe (2 flops per FMA): the
    "alu" roofline denominator of the float64 stencil kernels."""
    return 2.0 * ohm.ohm_fp64_fma_rate() * 1e-12

# Algorithmic work per cell of one launch (bytes that must cross HBM, flops
# that the stencil must execute), by kernel kind and precision of its multigrid arrays.
#   smooth pass:   e in, r, eta, inv in, e out  -> 13 words of the multigrid type
#                  57 flops per cell (114 per updated cell, half the cells per pass)
#   composite:     B, S, eta (float64) in, residual out in the multigrid type
#                  1728 faces x 15 flops / 512 + 9 (divergence) + 9 (combination) = 68.6 flops
#   smooth (float32) is one fused red+black sweep: e in, r, eta, e out = 10 words;
#                  flops per cell: 1.47 updates (block + recomputed ring) x 114
ALGO = {
    ("smooth", 4): {"bytes": 10 * 4, "flops": 168.0},
    ("smooth", 8): {"bytes": 13 * 8, "flops": 57.0},
    ("composite", 4): {"bytes": 7 * 8 + 3 * 4, "flops": 68.6},
    ("composite", 8): {"bytes": 7 * 8 + 3 * 8, "flops": 68.6},
}
KRYLOV = 6  # FGMRES restart length of the float32 inner solve in the headline path
LATENCY_REPS = 50  # per-solve latency percentiles are taken over at least this many CN steps


def smooth_zero_frac(nu_pre: int, nu_post: int) -> float:
    """Share of a level's float32 sweeps per V-cycle that start from e = 0 (the first
    pre-smoothing sweep: it reads r and eta and writes e, 28 instead of 40 bytes per cell)."""
    return 1.0 / (nu_pre + nu_post) if nu_pre >= 1 else 0.0


def smooth_bytes(nu_pre: int, nu_post: int) -> float:
    """Algorithmic bytes per cell of the average float32 sweep launch of a V(nu_pre, nu_post)."""
    return ALGO[("smooth", 4)]["bytes"] - 12.0 * smooth_zero_frac(nu_pre, nu_post)


def smooth_traffic(nu_pre: int, nu_post: int):
    """DRAM bytes per cell of the average float32 sweep launch, from the committed capture."""
    t, tz = kernel_traffic("smooth_f32"), kernel_traffic("smooth_f32_zero")
    if t is None or tz is None:
        return None
    f = smooth_zero_frac(nu_pre, nu_post)
    return (1.0 - f) * t + f * tz


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        sm = [num(r[1]) for r in rows]
        smax = max(num(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(num(r[3]) for r in rows)}


def dist():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as td
        if not td.is_initialized():
            td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier_max(ws, value):
    """Barrier, then the maximum of `value` over all ranks (the slowest replica's time)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as td
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    td.barrier()
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, cells, steps, elapsed_ms):
    """Whole-job cell-steps/s of ws replicas: all cells of all ranks over the slowest rank's time."""
    return ws * cells * steps / (barrier_max(ws, elapsed_ms) * 1e-3)


# ----------------------------------------------------------------------------- CPU oracle
def oracle_cycle_count(n: int):
    path = os.path.join(ROOT, "tests", "golden", "oracle_cycles.json")
    if os.path.exists(path):
        d = json.load(open(path)).get(f"resistive_bump_{n}")
        if d and d.get("converged"):
            return int(d["cycles"]), "tests/golden/oracle_cycles.json"
    return None, None


def time_oracle_sample(wl, gpu_cycles=None):
    """Times the oracle on the full workload: one source + residual (max_outer = 0) and one
    more defect-correction cycle (max_outer = 1); a CN step costs t0 + cycles x (t1 - t0)."""
    from oracle.oracle import Oracle
    n = wl.hier.base_cells[0]
    cycles, src = oracle_cycle_count(n)
    if cycles is None:
        cycles, src = gpu_cycles, "FP64 GPU run of the same schedule (parity-tested identical)"
    o = Oracle(wl.hier, wl.lam, wl.eta)
    t = time.perf_counter()
    o.cn_step(wl.B, wl.dt, -1.0, 2, 2, 16, 0)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    o.cn_step(wl.B, wl.dt, -1.0, 2, 2, 16, 1)
    t1 = time.perf_counter() - t
    per_step = t0 + cycles * max(t1 - t0, 0.0)
    cells = wl.hier.leaf_cells()
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": cells / per_step, "unit": UNIT, "cores": threads, "kind": "oracle", "extrapolated": True,
            "sample": (f"one {n}^3 step's source+residual ({t0:.1f} s) and one defect-correction cycle "
                       f"({t1 - t0:.1f} s) on the full input; step = source + {cycles} cycles ({src})"),
            "seconds_per_step": per_step}


FULL_STEP_RECORD = os.path.join(ROOT, "profiles", "oracle_full_step_resistive_bump_{n}.json")


def oracle_full_step_record(n: int):
    """The committed measurement of one complete oracle step at n^3 (written by --cpu-full-step on
    a GPU machine's host), set beside the sampled model: both its measured and its modelled seconds."""
    path = FULL_STEP_RECORD.format(n=n)
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    return {"full_step_s": d["full_step_s"], "model_s": d["model_s"], "model_error": d["model_s"] / d["full_step_s"] - 1.0,
            "cores": d["cores"], "cycles": d["cycles"], "source": os.path.relpath(path, ROOT)}


def run_cpu_full_step(args):
    """One complete oracle CN step (V(2,2), 16 coarsest sweeps, defect correction to the
    workload's tolerance) timed on the host cores, next to the sampled model of time_oracle_sample
    on the same input in the same process."""
    from paper_1009_0798_gb300 import workloads as W
    from oracle import build as obuild
    from oracle.oracle import Oracle
    obuild.build()
    wl = W.resistive_bump_256(n=args.size)
    model = time_oracle_sample(wl)
    o = Oracle(wl.hier, wl.lam, wl.eta)
    t = time.perf_counter()
    _, info = o.cn_step(wl.B, wl.dt, wl.tol, 2, 2, 16, 400)
    full = time.perf_counter() - t
    print(json.dumps({"workload": f"resistive_bump_{args.size}^3", "full_step_s": full,
                      "model_s": model["seconds_per_step"], "cycles": info["cycles"], "converged": info["converged"],
                      "cores": model["cores"], "model_sample": model["sample"]}), flush=True)


def run_reference(args):
    ws, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    from paper_1009_0798_gb300 import workloads as W
    import __graft_entry__ as ge
    from oracle import build as obuild
    obuild.build()
    wl = W.resistive_bump_256(n=args.size)
    samples = []
    for k in range(args.warmup + args.steps):
        s = time_oracle_sample(wl)
        if k >= args.warmup:
            samples.append(s)
    v = statistics.median(s["value"] for s in samples)
    per = statistics.median(s["seconds_per_step"] for s in samples)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"resistive_bump_{args.size}^3", "cells": wl.hier.leaf_cells(), "tol": wl.tol,
                       "precision": "fp64 CPU oracle", "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": samples[0]["cores"], "kind": "oracle",
                             "extrapolated": True, "sample": samples[0]["sample"],
                             "model_check": oracle_full_step_record(args.size)},
            "timing": ("each step is a sample (one source+residual and one cycle on the full input) scaled to a "
                       "whole step; ms_per_step is that modelled step, not the sample's own time"),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    del ge
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
# The source of the sweep and of the point update it uses: from the update's constants to the
# block-pair residual section of ohm_kernels.cu.  A traffic figure stays valid while this text
# is unchanged (edits elsewhere in the file do not touch the sweep).
SWEEP_SRC_START = "// Constants of the point update (Eqs. 19-23)"
SWEEP_SRC_END = "// ------------------------------------------------------------------ residual on brick pairs"


def sweep_source_sha() -> str:
    src = open(os.path.join(ROOT, "paper_1009_0798_gb300", "csrc", "ohm_kernels.cu")).read()
    i = src.index(SWEEP_SRC_START)
    j = src.index(SWEEP_SRC_END, i)
    return hashlib.sha256(src[i:j].encode()).hexdigest()[:16]


def kernel_traffic(kind: str):
    """DRAM bytes per cell of a kernel from a committed ncu capture, if it was taken on the
    current source of the sweep (hash match), else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(kind)
    if not e or e.get("sweep_source_sha") != sweep_source_sha():
        return None
    return float(e["dram_bytes_per_cell"])


def run_steps(ohm, g, B, B0, eta, wl, nsteps, stream, evs=None):
    import torch
    infos = []
    B.copy_(B0)
    for k in range(nsteps):
        if evs is not None:
            evs[k].record(stream)
        st = ohm.ohm_cn_step(g, B, None, wl.dt, wl.tol)
        infos.append(st)
        if not st["converged"]:
            raise RuntimeError(f"step {k} did not converge: {st}")
    if evs is not None:
        evs[nsteps].record(stream)
    torch.cuda.synchronize()
    return infos


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__ as ge
    from paper_1009_0798_gb300 import ohm
    from paper_1009_0798_gb300 import workloads as W

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    ge.build()
    wl = W.resistive_bump_256(n=args.size)
    cells = wl.hier.leaf_cells()
    stream = torch.cuda.current_stream()
    B0 = torch.from_numpy(np.ascontiguousarray(wl.B)).cuda()
    eta = torch.from_numpy(np.ascontiguousarray(wl.eta)).cuda()
    B = torch.empty_like(B0)
    hbm_peak, peak_src = peaks()
    nu = tuple(int(v) for v in args.nu.split(","))
    nuc = tuple(int(v) for v in args.nu_coarse.split(","))
    KRYLOV = args.krylov

    def make(precision, krylov=0, omega=1.0, nu_coarse=(0, 0)):
        g = ohm.ohm_create_hierarchy(wl.hier.base_cells, wl.hier.dx0, wl.hier.blocks, lam=wl.lam,
                                     precision=precision, nu_pre=nu[0], nu_post=nu[1], n_coarse=args.n_coarse,
                                     max_outer=400, stream=stream, krylov=krylov,
                                     inner_tol=args.inner_tol if precision != ohm.OHM_FP64 else 0.0, omega=omega,
                                     nu_coarse=nu_coarse)
        ohm.ohm_set_eta(g, eta)
        return g

    def timed(g, precision, profile=True):
        tsize = 4 if precision != ohm.OHM_FP64 else 8
        # warm-up; the first two also pick the dominant kernel (composite vs smooth)
        totals = {}
        for k in range(args.warmup):
            kind = [ohm.OHM_K_COMPOSITE, ohm.OHM_K_SMOOTH][k % 2] if k < 2 else None
            if kind is not None:
                ohm.ohm_prof_enable(g, kind, min_blocks=wl.hier.nblocks, max_launches=8192)
            run_steps(ohm, g, B, B0, eta, wl, 1, stream)
            if kind is not None:
                totals[kind] = ohm.ohm_prof_read(g)["ms"]
                ohm.ohm_prof_enable(g, -1)
        dom = max(totals, key=totals.get) if totals else ohm.OHM_K_SMOOTH
        if profile:
            ohm.ohm_prof_enable(g, dom, min_blocks=wl.hier.nblocks, max_launches=1 << 16)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        n0 = ohm.ohm_launch_count(g)
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            infos = run_steps(ohm, g, B, B0, eta, wl, args.steps, stream, evs)
        launches = ohm.ohm_launch_count(g) - n0
        per = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
        total_ms = evs[0].elapsed_time(evs[args.steps])
        prof = ohm.ohm_prof_read(g) if profile else None
        ohm.ohm_prof_enable(g, -1)
        name = "composite" if dom == ohm.OHM_K_COMPOSITE else "smooth"
        return {"total_ms": total_ms, "per_step_ms": per, "infos": infos, "launches": launches,
                "clocks": clk.summary(), "dom": name, "prof": prof, "tsize": tsize}

    def summary(r):
        return {"value": ws * cells * args.steps / (barrier_max(ws, r["total_ms"]) * 1e-3),
                "ms_per_step": r["total_ms"] / args.steps, "cycles_per_step": [s["cycles"] for s in r["infos"]]}

    if args.only:
        prec = {"fp64": ohm.OHM_FP64, "fp64_fgmres": ohm.OHM_FP64, "fgmres_ff": ohm.OHM_MIXED_FF,
                "fgmres_ffc": ohm.OHM_MIXED_FF_CHECKED}.get(args.only, ohm.OHM_MIXED)
        fg = "fgmres" in args.only
        g1 = make(prec, KRYLOV if fg else 0, args.omega if fg else 1.0, nuc if fg else (0, 0))
        for _ in range(args.warmup):
            run_steps(ohm, g1, B, B0, eta, wl, 1, stream)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        infos = run_steps(ohm, g1, B, B0, eta, wl, args.steps, stream, evs)
        ms = evs[0].elapsed_time(evs[args.steps])
        if rank == 0:
            print(json.dumps({"only": args.only, "size": args.size, "steps": args.steps, "nu": nu,
                              "n_coarse": args.n_coarse, "krylov": KRYLOV if fg else 0,
                              "inner_tol": args.inner_tol, "omega": args.omega if fg else 1.0,
                              "nu_coarse": nuc if fg else (0, 0),
                              "ms_per_step": ms / args.steps, "cycles_per_step": [s["cycles"] for s in infos],
                              "final_rel_l2": [s["rel_l2"] for s in infos]}),
                  flush=True)
        return

    # headline: float32 multigrid, FGMRES-accelerated, inside float64 iterative refinement
    gm = make(ohm.OHM_MIXED, KRYLOV, args.omega, nuc)
    mixed = timed(gm, ohm.OHM_MIXED)
    # per-solve latency over at least 50 steps: the timed steps plus further ones after the
    # timed region (not part of value)
    lat_ms = list(mixed["per_step_ms"])
    extra = max(0, LATENCY_REPS - args.steps)
    if extra:
        evx = [torch.cuda.Event(enable_timing=True) for _ in range(extra + 1)]
        run_steps(ohm, gm, B, B0, eta, wl, extra, stream, evx)
        lat_ms += [evx[k].elapsed_time(evx[k + 1]) for k in range(extra)]
    t_max = barrier_max(ws, mixed["total_ms"])
    value = job_throughput(ws, cells, args.steps, mixed["total_ms"])
    # the same without Krylov acceleration (inner defect correction), and plain FP64 (the
    # paper's scheme: float64 V-cycles in float64 defect correction)
    others = {}
    if not args.no_fp64:
        # plain FP64 (float64 V-cycles in float64 defect correction) with the headline's sweep
        # counts and relaxation, the same with the headline's FGMRES in float64 (the fastest
        # float64 solver here), and with the paper's schedule (Gauss-Seidel, the same sweeps on
        # every grid)
        for name, prec, kr, om, nc in (("mixed_float_float_residual", ohm.OHM_MIXED_FF, KRYLOV, args.omega, nuc),
                                       ("mixed_float_float_checked", ohm.OHM_MIXED_FF_CHECKED, KRYLOV, args.omega, nuc),
                                       ("mixed_defect_correction", ohm.OHM_MIXED, 0, 1.0, (0, 0)),
                                       ("fp64_plain", ohm.OHM_FP64, 0, args.omega, nuc),
                                       ("fp64_fgmres", ohm.OHM_FP64, KRYLOV, args.omega, nuc),
                                       ("fp64_paper_schedule", ohm.OHM_FP64, 0, 1.0, (0, 0))):
            g2 = make(prec, kr, om, nc)
            r2 = timed(g2, prec, profile=False)
            others[name] = summary(r2)
            if prec == ohm.OHM_MIXED_FF:
                others[name]["precision"] = ("OHM_MIXED_FF: as the headline, but the outer residual in float-float "
                                             "(float32 pairs, ~48 bits) with float32-accumulated norms")
            if prec == ohm.OHM_MIXED_FF_CHECKED:
                others[name]["precision"] = ("OHM_MIXED_FF_CHECKED: as the headline, but the intermediate outer "
                                             "residuals in float-float; the source, the first and every "
                                             "step-ending residual in float64")
                others[name]["final_rel_l2_max"] = max(st["rel_l2"] for st in r2["infos"])
            if prec == ohm.OHM_FP64:
                outer = f"float64 FGMRES({kr}) right-preconditioned by the V-cycle" if kr else "float64 defect correction"
                others[name]["multigrid"] = (f"float64 V({nu[0]},{nu[1]}) on level 0, "
                                             f"V({nc[0] or nu[0]},{nc[1] if nc != (0, 0) else nu[1]}) below, "
                                             f"omega {om}, {args.n_coarse} coarsest sweeps, {outer}")
            g2.close()
            del g2
    fp64 = others.get("fp64_plain")
    fp64_fg = others.get("fp64_fgmres")
    fp64_paper = others.get("fp64_paper_schedule")

    # end to end through the public API with host buffers: every step uploads its inputs (B, eta)
    # from pinned host memory and downloads its result.  The steps are independent solves of the
    # workload's first step; their copies run on a second stream, double-buffered, so the upload
    # of step k+1 and the download of step k-1 overlap the compute of step k.
    e2e = None
    if not args.no_e2e:
        Bh = torch.from_numpy(np.ascontiguousarray(wl.B)).pin_memory()
        Eh = torch.from_numpy(np.ascontiguousarray(wl.eta)).pin_memory()
        outs = [torch.empty_like(Bh).pin_memory() for _ in range(2)]
        Bd = [torch.empty_like(B0) for _ in range(2)]
        Ed = [torch.empty_like(eta) for _ in range(2)]
        cs = torch.cuda.Stream()

        def upload(k):
            with torch.cuda.stream(cs):
                Bd[k % 2].copy_(Bh, non_blocking=True)
                Ed[k % 2].copy_(Eh, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(cs)
            return ev

        def pipeline(n):
            # ohm_cn_step returns when its step is done, so the next upload is enqueued first:
            # its buffers were last read by step k-1 (finished) and its download (earlier on cs)
            up = upload(0)
            for k in range(n):
                nxt = upload(k + 1) if k + 1 < n else None
                stream.wait_event(up)
                st = ohm.ohm_cn_step(gm, Bd[k % 2], Ed[k % 2], wl.dt, wl.tol)
                if not st["converged"]:
                    raise RuntimeError(f"e2e step {k} did not converge: {st}")
                done = torch.cuda.Event()
                done.record(stream)
                with torch.cuda.stream(cs):
                    cs.wait_event(done)
                    outs[k % 2].copy_(Bd[k % 2], non_blocking=True)
                up = nxt

        pipeline(2)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cs)
        pipeline(args.steps)
        e1.record(cs)
        torch.cuda.synchronize()
        et = barrier_max(ws, e0.elapsed_time(e1))
        e2e = {"value": ws * cells * args.steps / (et * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": Bh.numel() * 8 + Eh.numel() * 8, "d2h_bytes_per_step": outs[0].numel() * 8,
               "timing": "CUDA events around all steps; independent steps from the host inputs, uploads and "
                         "downloads on a copy stream overlapping the neighbouring steps' compute"}

    # bounded batched and serving legs (each its own timed region, clock sample and metric)
    legs = {}
    if not args.no_legs:
        legs = run_legs(args)
    if rank != 0:
        return
    # roofline of the dominant kernel, measured with events inside the timed region
    prof = mixed["prof"]
    algo = dict(ALGO[(mixed["dom"], mixed["tsize"])])
    if (mixed["dom"], mixed["tsize"]) == ("smooth", 4):
        algo["bytes"] = smooth_bytes(*nu)
    per_launch_cells = prof["cells"] / max(prof["launches"], 1)
    sec = prof["ms"] * 1e-3
    if mixed["dom"] == "composite":
        achieved = algo["flops"] * prof["cells"] / sec * 1e-12
        fp64_peak = fp64_peak_tflops(ohm)
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "peak_source": "measured in this run: DFMA probe (x2 flops)"}
    else:
        achieved = algo["bytes"] * prof["cells"] / sec * 1e-9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"}
    tb = (smooth_traffic(*nu) if (mixed["dom"], mixed["tsize"]) == ("smooth", 4)
          else kernel_traffic(mixed["dom"] + ("_f32" if mixed["tsize"] == 4 else "_f64")))
    roof.update({"kernel": mixed["dom"], "launches": prof["launches"], "ms_per_launch": prof["ms"] / max(prof["launches"], 1),
                 "algorithmic_bytes_per_launch": algo["bytes"] * per_launch_cells,
                 "traffic": tb * per_launch_cells if tb is not None else None})
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        try:
            from oracle import build as obuild
            obuild.build()
            cyc = fp64_paper["cycles_per_step"][0] if fp64_paper else mixed["infos"][0]["cycles"]
            cpu = time_oracle_sample(wl, gpu_cycles=cyc)
            cpu.pop("seconds_per_step", None)
            chk = oracle_full_step_record(args.size)
            if chk:
                cpu["model_check"] = chk
        except Exception as ex:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {ex}"}
    lat = sorted(lat_ms)
    p99 = lat[min(len(lat) - 1, math.ceil(0.99 * len(lat)) - 1)]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 multigrid + f64 residual/update/norms", "data": "synthetic",
            "config": {"workload": f"resistive_bump_{args.size}^3", "cells": cells, "tol": wl.tol,
                       "dt_over_explicit_limit": 100, "cn_steps_per_run": args.steps, "precision": "mixed",
                       "multigrid": f"V({nu[0]},{nu[1]}) on level 0 and V({nuc[0]},{nuc[1]}) below, red-black SOR sweeps "
                                    f"(omega {args.omega}), {args.n_coarse} coarsest sweeps; float32 inner solve "
                                    f"FGMRES({KRYLOV}) right-preconditioned by the V-cycle; float64 iterative refinement",
                       "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (402 MB per float64 field vs 129 MB L2), no flush"},
            "latency_ms": {"p50": statistics.median(lat), "p99": p99, "solves": len(lat)},
            "cycles_per_step": [s["cycles"] for s in mixed["infos"]],
            "final_rel_l2": [s["rel_l2"] for s in mixed["infos"]],
            "fp64_plain": fp64, "fp64_fgmres": fp64_fg, "fp64_paper_schedule": fp64_paper,
            "speedup_vs_fp64_plain": (value / fp64["value"]) if fp64 else None,
            "speedup_vs_fp64_fgmres": (value / fp64_fg["value"]) if fp64_fg else None,
            "fp64_fma_tflops": fp64_peak_tflops(ohm),
            "mixed_defect_correction": others.get("mixed_defect_correction"),
            "mixed_float_float_residual": others.get("mixed_float_float_residual"),
            "mixed_float_float_checked": others.get("mixed_float_float_checked"),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": mixed["clocks"],
            "gpu_launches": mixed["launches"], **legs}
    print(json.dumps(line), flush=True)


def run_legs(args):
    """The batched and serving workloads at bounded sizes inside the default run: `batched_leg`
    (args.leg_instances instances of the 512-instance recipe, the fixed batch schedule, no
    autotuning) and `serving_leg` (the first args.leg_requests requests of the Poisson stream).
    Each reports its own value, solves/s, latency percentiles and clock sample."""
    la = argparse.Namespace(**vars(args))
    la.instances, la.no_autotune, la.no_fp64, la.no_e2e, la.no_cpu_baseline = args.leg_instances, True, True, True, True
    la.steps, la.warmup = 3, 1
    b = run_batched(la, emit=False)
    ls = argparse.Namespace(**vars(args))
    ls.requests, ls.no_cpu_baseline = args.leg_requests, True
    v = run_serving(ls, emit=False)
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "solves_per_s", "latency_ms", "clocks", "gpu_launches")
    out = {}
    if b:
        out["batched_leg"] = {**{k: b.get(k) for k in keep}, "workload": b["config"]["workload"],
                              "classes": b["config"]["classes"], "multigrid": b["config"]["multigrid"],
                              "mean_cycles_per_instance": b.get("mean_cycles_per_instance")}
    if v:
        out["serving_leg"] = {**{k: v.get(k) for k in keep}, "workload": v["config"]["workload"],
                              "requests": v["config"]["requests"], "mix": v["config"]["mix"],
                              "converged": v.get("converged"), "alone_vs_mix_identical": v.get("alone_vs_mix_identical")}
    return out


# ----------------------------------------------------------------------------- batches
def run_batched(args, emit=True):
    """512 independent periodic instances (edges 16..64), one CN step each to 1e-9: one
    batched hierarchy per edge length (every launch covers all its instances, CUDA-graph
    inner iterations, autotuned schedule), the five classes stepped concurrently from five
    host threads on five streams.  A bench step solves every instance once from its initial
    field."""
    import concurrent.futures as cf

    import numpy as np
    import torch

    import __graft_entry__ as ge
    from paper_1009_0798_gb300 import ohm
    from paper_1009_0798_gb300 import workloads as W

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    ge.build()
    tol = 1e-9
    inst = W.batched_instances(args.instances, seed=4)
    nu = tuple(int(v) for v in args.batch_nu.split(","))
    bnuc = tuple(int(v) for v in args.batch_nu_coarse.split(","))
    groups = {}
    for i in inst:
        groups.setdefault(i.n, []).append(i)
    cells = sum(i.n ** 3 for i in inst)
    C = []
    for n in sorted(groups):
        lst = groups[n]
        s = torch.cuda.Stream()
        h = lst[0].hier
        c = {"n": n, "K": len(lst), "s": s, "dts": [i.dt for i in lst], "hier": h}
        with torch.cuda.stream(s):
            c["B0"] = torch.from_numpy(np.concatenate([i.B for i in lst]).reshape(-1)).cuda()
            c["eta"] = torch.from_numpy(np.concatenate([i.eta for i in lst]).reshape(-1)).cuda()
            c["B"] = torch.empty_like(c["B0"])
            c["g"] = ohm.ohm_create_hierarchy(h.base_cells, h.dx0, h.blocks, lam=0.5, precision=ohm.OHM_MIXED,
                                              nu_pre=nu[0], nu_post=nu[1], n_coarse=args.batch_n_coarse, max_outer=400,
                                              stream=s, n_instances=len(lst), use_graphs=True,
                                              krylov=args.batch_krylov, omega=args.batch_omega, nu_coarse=bnuc)
            ohm.ohm_set_eta(c["g"], c["eta"])
        C.append(c)
    torch.cuda.synchronize()
    tuned = {}
    if not args.no_autotune:
        for c in C:
            with torch.cuda.stream(c["s"]):
                tuned[c["n"]] = ohm.ohm_autotune(c["g"], c["B0"], c["dts"], tol)
        torch.cuda.synchronize()

    def step(c):
        with torch.cuda.stream(c["s"]):
            c["B"].copy_(c["B0"])
            status, st = ohm.ohm_cn_step_batch(c["g"], c["B"], c["dts"], tol)
        if status != ohm.OHM_OK:
            raise RuntimeError(f"class {c['n']}: not converged")
        return st

    pool = cf.ThreadPoolExecutor(len(C))
    main_s = torch.cuda.current_stream()

    def one_round(timed=False):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main_s)
        for c in C:
            c["s"].wait_event(e0)
        res = list(pool.map(step, C))
        for c in C:
            ev = torch.cuda.Event()
            ev.record(c["s"])
            main_s.wait_event(ev)
        e1.record(main_s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), res

    for _ in range(args.warmup):
        one_round()
    n0 = sum(ohm.ohm_launch_count(c["g"]) for c in C)
    per, cyc = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms, res = one_round(True)
            per.append(ms)
            cyc.append(sum(x["cycles"] for st in res for x in st) / len(inst))
    launches = sum(ohm.ohm_launch_count(c["g"]) for c in C) - n0
    total = sum(per)
    t_max = barrier_max(ws, total)
    value = ws * cells * args.steps / (t_max * 1e-3)

    # the smoother of the largest class, timed with events in one more (untimed) round
    big = max(C, key=lambda c: c["n"])
    nfine = big["hier"].nblocks * big["K"]
    ohm.ohm_prof_enable(big["g"], ohm.OHM_K_SMOOTH, min_blocks=nfine, max_launches=4096)
    step(big)
    torch.cuda.synchronize()
    prof = ohm.ohm_prof_read(big["g"])
    ohm.ohm_prof_enable(big["g"], -1)
    hbm_peak, peak_src = peaks()
    sec = prof["ms"] * 1e-3
    tn = tuned.get(big["n"], {})
    sb = smooth_bytes(tn.get("nu_pre", nu[0]), tn.get("nu_post", nu[1]))
    ach = sb * prof["cells"] / max(sec, 1e-12) * 1e-9
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)", "kernel": f"smooth ({big['n']}^3 class)",
            "launches": prof["launches"], "ms_per_launch": prof["ms"] / max(prof["launches"], 1),
            "algorithmic_bytes_per_launch": sb * prof["cells"] / max(prof["launches"], 1),
            "traffic": None}

    # comparisons: every instance alone through the single-problem API (FGMRES(6), the
    # headline path), one after another; and the batched plain-FP64 scheme
    comp = {}
    if not args.no_fp64 and rank == 0:
        t = time.perf_counter()
        cyc1 = 0
        for n in sorted(groups):
            lst = groups[n]
            h = lst[0].hier
            g = ohm.ohm_create_hierarchy(h.base_cells, h.dx0, h.blocks, lam=0.5, precision=ohm.OHM_MIXED, max_outer=400,
                                         krylov=KRYLOV)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            B = torch.empty(h.nblocks * 1536, dtype=torch.float64, device="cuda")
            eta = torch.empty(h.nblocks * 512, dtype=torch.float64, device="cuda")
            ms = 0.0
            for i in lst:
                B.copy_(torch.from_numpy(i.B.reshape(-1)))
                eta.copy_(torch.from_numpy(i.eta.reshape(-1)))
                e0.record()
                st = ohm.ohm_cn_step(g, B, eta, i.dt, tol)
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                cyc1 += st["cycles"]
            comp.setdefault("unbatched_ms", 0.0)
            comp["unbatched_ms"] += ms
            g.close()
        comp = {"one_at_a_time_fgmres": {"value": cells / (comp["unbatched_ms"] * 1e-3),
                                         "ms_per_step": comp["unbatched_ms"],
                                         "mean_cycles": cyc1 / len(inst),
                                         "note": "each instance alone through ohm_cn_step (eta upload excluded)"}}
        ms64 = 0.0
        for n in sorted(groups):
            c = next(x for x in C if x["n"] == n)
            h = c["hier"]
            g = ohm.ohm_create_hierarchy(h.base_cells, h.dx0, h.blocks, lam=0.5, precision=ohm.OHM_FP64,
                                         max_outer=400, n_instances=c["K"])
            ohm.ohm_set_eta(g, c["eta"])
            B = c["B0"].clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ohm.ohm_cn_step_batch(g, B, c["dts"], tol)
            e1.record()
            torch.cuda.synchronize()
            ms64 += e0.elapsed_time(e1)
            g.close()
        comp["fp64_plain_batched"] = {"value": cells / (ms64 * 1e-3), "ms_per_step": ms64,
                                      "note": "classes one after another"}

    # end to end: host fields in, results out, every step
    e2e = None
    if not args.no_e2e:
        hosts = [(torch.from_numpy(np.concatenate([i.B for i in groups[c["n"]]]).reshape(-1)).pin_memory(),
                  torch.from_numpy(np.concatenate([i.eta for i in groups[c["n"]]]).reshape(-1)).pin_memory()) for c in C]
        outs = [torch.empty_like(hb).pin_memory() for hb, _ in hosts]

        def step_e2e(k):
            c, (hb, he), out = C[k], hosts[k], outs[k]
            with torch.cuda.stream(c["s"]):
                c["B"].copy_(hb, non_blocking=True)
                c["eta"].copy_(he, non_blocking=True)
                ohm.ohm_set_eta(c["g"], c["eta"])
                ohm.ohm_cn_step_batch(c["g"], c["B"], c["dts"], tol)
                out.copy_(c["B"], non_blocking=True)
            c["s"].synchronize()

        step_e2e_all = lambda: list(pool.map(step_e2e, range(len(C))))  # noqa: E731
        step_e2e_all()
        t = time.perf_counter()
        for _ in range(args.steps):
            step_e2e_all()
        et = barrier_max(ws, (time.perf_counter() - t) * 1e3)
        e2e = {"value": ws * cells * args.steps / (et * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": sum(hb.numel() * 8 + he.numel() * 8 for hb, he in hosts),
               "d2h_bytes_per_step": sum(o.numel() * 8 for o in outs),
               "timing": "host wall clock around all classes' threads (copies, eta set, step, copy back)"}
    cpu = None
    if ws == 1 and not args.no_cpu_baseline and rank == 0:
        try:
            from oracle import build as obuild
            from oracle.oracle import Oracle
            obuild.build()
            i = next(x for x in inst if x.n == 32)
            o = Oracle(i.hier, 0.5, i.eta)
            t = time.perf_counter()
            o.cn_step(i.B, i.dt, tol, 2, 2, 16, 400)
            sec_o = time.perf_counter() - t
            cpu = {"value": i.n ** 3 / sec_o, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
                   "kind": "oracle", "sample": f"one 32^3 instance of the batch, one CN step to 1e-9 ({sec_o:.1f} s)"}
        except Exception as ex:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {ex}"}
    if rank != 0:
        return
    lat = sorted(per)
    p99 = lat[min(len(lat) - 1, math.ceil(0.99 * len(lat)) - 1)]
    line = {"metric": f"cell-steps/s, {len(inst)} independent instances to rel. residual 1e-9", "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 multigrid + f64 residual/update/norms", "data": "synthetic",
            "config": {"workload": f"batched_{len(inst)}", "cells": cells,
                       "classes": {str(c["n"]): c["K"] for c in C}, "tol": tol,
                       "multigrid": "per-instance float64 iterative refinement, float32 inner solve: " +
                                    (f"per-instance FGMRES({args.batch_krylov}) right-preconditioned by the V-cycle"
                                     if args.batch_krylov else "defect-correction V-cycles"),
                       "autotuned": {str(k): v for k, v in tuned.items()}, "graphs": True,
                       "parallelism": f"replicas x{ws}; 5 size classes on 5 streams",
                       "l2": "working set 3 GB (> 129 MB L2), no flush"},
            "solves_per_s": ws * len(inst) * args.steps / (t_max * 1e-3),
            "latency_ms": {"p50": statistics.median(lat), "p99": p99},
            "mean_cycles_per_instance": cyc, **comp,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "gpu_launches": launches}
    if not args.no_autotune:
        line["config"]["schedule_before_tuning"] = (f"V({nu[0]},{nu[1]}), V{bnuc} below, omega {args.batch_omega}, "
                                                    f"{args.batch_n_coarse} coarsest sweeps")
    else:
        line["config"]["schedule"] = (f"V({nu[0]},{nu[1]}) on level 0, V{bnuc} below, omega {args.batch_omega}, "
                                      f"{args.batch_n_coarse} coarsest sweeps")
    for c in C:
        c["g"].close()
    pool.shutdown()
    if emit:
        print(json.dumps(line), flush=True)
    return line


# ----------------------------------------------------------------------------- serving
SERVE_EDGES = tuple(range(32, 129, 8))  # every multiple of 8 in 32..128


def serving_requests(count, rate, seed=5):
    """Seeded Poisson request stream: arrival times at `rate` per second; 70% uniform periodic
    boxes with edge from SERVE_EDGES, 30% two-level AMR (base 32^3, blocks meeting the sphere
    r < 0.2 about the centre refined); each request has its own eta (a pooled smooth 2-decade
    field times its own factor 10^U(-1,1)), its own B (pooled k^-2 field times U(0.5, 2)),
    dt = 10^U(1,3) times the explicit limit at its finest level, 1-5 steps."""
    import numpy as np

    from paper_1009_0798_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    c = np.array([0.5, 0.5, 0.5])

    def sphere(lo, hi):
        nearest = np.clip(c, lo, hi)
        return float(np.sum((nearest - c) ** 2)) < 0.2 ** 2

    pool = {}

    def fields(key, n_variant):
        if (key, n_variant) not in pool:
            if key == "amr":
                h = W.refined(32, 32, 32, 1.0 / 32, [sphere])
                dense_b = W.random_potential_field((64, 64, 64), 1.0 / 64, 900 + n_variant, 1.0)
                dense_e = W.smooth_lognormal_eta(64, 950 + n_variant)
                # level 0 from the mean of 2^3 fine cells, level 1 from the fine field
                def lv0(f):
                    return f.reshape(f.shape[0], 32, 2, 32, 2, 32, 2).mean(axis=(2, 4, 6))
                B = np.concatenate([W.dense_to_blocks(h, lv0(dense_b), 0), W.dense_to_blocks(h, dense_b, 1)])
                E = np.concatenate([W.dense_to_blocks(h, lv0(dense_e), 0), W.dense_to_blocks(h, dense_e, 1)])
            else:
                n = key
                h = W.uniform(n, n, n, 1.0 / n)
                B = W.dense_to_blocks(h, W.random_potential_field((n, n, n), 1.0 / n, 700 + n + n_variant, 1.0))
                E = W.dense_to_blocks(h, W.smooth_lognormal_eta(n, 800 + n + n_variant))
            pool[(key, n_variant)] = (h, B, E)
        return pool[(key, n_variant)]

    reqs = []
    for i in range(count):
        key = "amr" if rng.uniform() < 0.3 else int(rng.choice(SERVE_EDGES))
        h, B, E = fields(key, int(rng.integers(0, 2)))
        fe = 10.0 ** rng.uniform(-1.0, 1.0)
        fb = rng.uniform(0.5, 2.0)
        dxf = h.dx(h.nlevels - 1)
        dt = 10.0 ** rng.uniform(1.0, 3.0) * dxf * dxf / (6.0 * float(E.max()) * fe)
        reqs.append({"t": float(t[i]), "key": key, "hier": h, "B": B, "eta": E, "fb": fb, "fe": fe, "dt": dt,
                     "steps": int(rng.integers(1, 6))})
    return reqs


def serving_cpu_baseline(reqs, inputs):
    """The oracle on the host cores for one request of the stream's smallest uniform class (one
    step to 1e-9): a bounded sample, in served cell-steps/s."""
    try:
        from oracle import build as obuild
        from oracle.oracle import Oracle
        obuild.build()
        k = min((q for q, r in enumerate(reqs) if r["key"] != "amr"), key=lambda q: reqs[q]["hier"].leaf_cells())
        r = reqs[k]
        o = Oracle(r["hier"], 0.5, inputs[k][1])
        t = time.perf_counter()
        o.cn_step(inputs[k][0], r["dt"], 1e-9, 2, 2, 16, 400)
        sec = time.perf_counter() - t
        return {"value": r["hier"].leaf_cells() / sec, "unit": UNIT,
                "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
                "sample": f"request {k} of the stream ({r['key']}^3, one step to 1e-9, {sec:.1f} s)"}
    except Exception as ex:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {ex}"}


def run_serving(args, emit=True):
    """Poisson stream of CN-solve requests through the continuous-batching service: requests
    are submitted at their arrival times (host clock) with host arrays; latency = completion
    minus submission on the service clock.  Throughput = solved cell-steps over the span from
    the first submission to the last completion."""
    import threading

    import numpy as np
    import torch

    import __graft_entry__ as ge
    from paper_1009_0798_gb300 import server

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    ge.build()
    torch.cuda.init()
    reqs = serving_requests(args.requests, args.rate)
    budget = 60 << 30
    # V(4,4) with 4 coarsest sweeps, omega 1.3 and V(1,1) on the coarser grids: the schedule the
    # autotuner picks for most classes of the batched workload
    cfg = dict(hbm_budget_bytes=budget, max_batch=args.serve_max_batch, n_workers=args.serve_workers, precision=1,
               tol=1e-9, use_graphs=True,
               nu_pre=4, nu_post=4, n_coarse=4, max_outer=400, krylov=args.batch_krylov, omega=1.3,
               nu_coarse=tuple(int(v) for v in args.serve_nu_coarse.split(",")))
    # warm-up service: one request per class (kernels loaded, batches of each class built once)
    with server.Server(**cfg) as s:
        seen = {}
        for r in reqs:
            seen.setdefault(r["key"], r)
        ids = [s.submit(r["hier"], r["B"] * r["fb"], r["eta"] * r["fe"], r["dt"], 1) for r in seen.values()]
        for i in ids:
            s.wait(i)
    inputs = [(r["B"] * r["fb"], r["eta"] * r["fe"]) for r in reqs]
    results = [None] * len(reqs)
    with server.Server(**cfg) as s, ClockSampler(local) as clk:
        ids = [None] * len(reqs)
        ready = threading.Event()

        def collector():
            ready.wait()
            for k in range(len(reqs)):
                while ids[k] is None:
                    time.sleep(0.0005)
                results[k] = s.wait(ids[k])

        th = threading.Thread(target=collector)
        th.start()
        t0 = time.perf_counter()
        ready.set()
        for k, r in enumerate(reqs):
            delay = r["t"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids[k] = s.submit(r["hier"], inputs[k][0], inputs[k][1], r["dt"], r["steps"])
        th.join()
        stats = s.stats()
    lat = sorted((res[1]["t_done"] - res[1]["t_submit"]) * 1e3 for res in results)
    span = max(res[1]["t_done"] for res in results) - min(res[1]["t_submit"] for res in results)
    cell_steps = sum(r["hier"].leaf_cells() * r["steps"] for r in reqs)
    ok = sum(1 for res in results if res[1]["status"] == 0)
    # alone versus in the mix: a few requests again, each alone on a fresh service
    same = []
    for k in range(0, len(reqs), max(1, len(reqs) // 4))[:4]:
        r = reqs[k]
        with server.Server(**cfg) as s1:
            out, res = s1.wait(s1.submit(r["hier"], inputs[k][0], inputs[k][1], r["dt"], r["steps"]))
        same.append(bool(np.array_equal(out, results[k][0])))
    p = lambda q: lat[min(len(lat) - 1, max(0, math.ceil(q * len(lat)) - 1))]  # noqa: E731
    value = cell_steps / span
    line = {"metric": "served cell-steps/s, Poisson request stream to rel. residual 1e-9", "value": value,
            "unit": UNIT, "n_gpus": ws, "steps": len(reqs), "warmup": len(seen), "ms_per_step": span * 1e3 / len(reqs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 multigrid + f64 residual/update/norms", "data": "synthetic",
            "config": {"workload": f"serving_poisson_{args.rate:g}_per_s", "requests": len(reqs),
                       "mix": "70% uniform 32^3-128^3 (edges " + ",".join(map(str, SERVE_EDGES)) + "), 30% 2-level AMR",
                       "hbm_budget_gb": budget / 2 ** 30, "max_batch": cfg["max_batch"], "n_workers": cfg["n_workers"],
                       "graphs": True, "tol": 1e-9, "parallelism": f"replicas x{ws}",
                       "multigrid": f"V({cfg['nu_pre']},{cfg['nu_post']}) on level 0, V{cfg['nu_coarse']} below, omega "
                                    f"{cfg['omega']}, {cfg['n_coarse']} coarsest sweeps, FGMRES({cfg['krylov']}) inner solves"},
            "latency_ms": {"p50": p(0.5), "p99": p(0.99), "max": lat[-1]},
            "solves_per_s": len(reqs) / span, "offered_rate_per_s": args.rate,
            "span_s": span, "converged": ok, "alone_vs_mix_identical": same,
            "service": stats,
            "e2e": {"value": value, "unit": UNIT,
                    "h2d_bytes_per_step": int(np.mean([a.nbytes + b.nbytes for a, b in inputs])),
                    "d2h_bytes_per_step": int(np.mean([a.nbytes for a, _ in inputs])),
                    "timing": "host clock, submit to result in host memory"},
            "clocks": clk.summary(), "gpu_launches": stats.get("kernel_launches"),
            "roofline": None, "roofline_note": "the service runs the kernels of the batched and headline lines",
            "cpu_baseline": serving_cpu_baseline(reqs, inputs) if not args.no_cpu_baseline else None}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def main():
    args = args_parse()
    if args.cpu_full_step:
        run_cpu_full_step(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched512":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
