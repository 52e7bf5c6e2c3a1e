#!/usr/bin/env python
"""Benchmark of one forced isothermal MHD time step on a B300.

Workload (N=1 line): 512^3 periodic box, FP32 fields and arithmetic,
helical forcing (sigma = 1, shell 2.5 <= |k| <= 3.5, k_f ~ 3.13, f0 = 0.02),
nu = eta = 6.4e-5 (Re_M ~ 250 for u_rms ~ 0.05), CFL time step (0.4), the
paper's weak-seed-field initial condition (Sec. 4) generated on the device.
A step = device time-step reduction + forcing draw + three fused RHS/RK3-2N
substeps, all of it inside the timed region.  Inputs are larger than L2
(11.7 GB of state), so no L2 flush is needed between steps.  The same line
carries the FP64 step on the same workload, the batched ensemble (16 x 64^3
+ 8 x 128^3) against one-at-a-time stepping, and the continuous-batching
serving loop's p50/p99 latency.

Prints ONE JSON line.  --impl reference times the FP64 CPU oracle on the
host cores instead (a deliberately slow baseline, not a target)."""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s & %HBM roofline, FP32 vs FP64; batched p50/p99 job latency"
UNIT = "cell-updates/s"
BYTES_PER_CELL = {"f32": 70 * 4, "f64": 70 * 8}  # algorithmic: 70 values per cell-update
KF = 3.134           # mean |k| of the 98-vector shell 2.5 <= |k| <= 3.5
URMS0 = 0.05         # rms velocity estimate of the f0 = 0.02 forced flow
SEED_AMP = 1e-5      # seed-field amplitude (Sec. 4)


def re_m(n):
    """Magnetic Reynolds number of the n^3 single-run workload: ~250 at 512^3
    (the at-scale configuration), ~100 otherwise (the 256^3 configuration)."""
    return 250.0 if n >= 512 else 100.0


def workload(n):
    nu = URMS0 / (re_m(n) * KF)
    return dict(f0=0.02, sigma=1.0, kmin=2.5, kmax=3.5, nu=nu, eta=nu, cfl=0.4, seed=1)


# kept for the other workloads (C2 at 256^3, spectra, CPU timings)
WORKLOAD = workload(256)


def workload_name(n, dtype):
    w = workload(n)
    return (f"{n}^3 forced isothermal MHD step ({dtype.upper()}): helical sigma=1, shell [2.5,3.5] "
            f"(k_f~3.13), f0=0.02, nu=eta={w['nu']:.2g} (Re_M~{re_m(n):.0f}), CFL 0.4, seed field 1e-5 "
            f"(Sec. 4) generated on the device")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy of 1 Gi bf16)"
    except Exception:
        return 6400.0, "fallback (6.4 TB/s, earlier B300 measurement)"


def kernel_source_hash():
    """Hash of the sources that define the fused substep kernel (the traffic
    figure of the committed ncu capture is void once any of them changes)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2012_08758_b300", "csrc")
    for name in ("kernels_tma.cu", "kernels_x2.cu", "tma_util.cuh", "x2_variants.h", "physics.cuh",
                 "step_device.cuh", "mhd_internal.h"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(n, dtype):
    """DRAM bytes per substep launch from the committed ncu summary, or None
    when the kernels changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "substep_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    key = f"{n}_{dtype}"
    ent = d.get("workloads", {}).get(key)
    return None if ent is None else ent.get("bytes_per_launch")


def ncu_flops(dtype):
    """Floating-point operations per cell-update (three substeps, an FMA
    counted as 2) executed by the substep kernel, from the committed ncu
    instruction counts, or None when the kernels changed since."""
    path = os.path.join(ROOT, "profiles", "substep_flops.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    ent = d.get("dtypes", {}).get(dtype)
    return None if ent is None else ent.get("flops_per_cell_update")


def alu_peaks():
    """Measured FMA throughput of this GPU (flop/s): FP32 scalar, FP32
    packed pairs and FP64."""
    from paper_2012_08758_b300 import binding as B
    return {"f32": B.mhd_alu_peak(B.MHD_F32)[0], "f32x2": B.mhd_alu_peak(B.MHD_F32X2)[0],
            "f64": B.mhd_alu_peak(B.MHD_F64)[0]}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = str(gpu_index)
        self.samples = []
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([c.strip() for c in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.1)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _oracle_steps(n, cores, seconds, max_steps=200):
    """Whole FP64 oracle steps of the n^3 version of the workload on `cores`
    host threads (host-tuned build): (steps, seconds, threads used)."""
    from oracle import oracle as O
    from paper_2012_08758_b300 import inputs

    O.use_native()
    used = O.set_threads(cores)
    p = O.Params(nx=n, ny=n, nz=n, **workload(n))
    q = inputs.seed_field_state(n, seed=0)
    O.run(p, q, 1)  # warm-up
    steps, t0 = 0, time.perf_counter()
    while True:
        O.run(p, q, 1, step0=1 + steps)
        steps += 1
        el = time.perf_counter() - t0
        if el > seconds or steps >= max_steps:
            break
    return steps, el, used


def cpu_baseline(seconds=12.0, n=64, one_core_seconds=8.0):
    """The FP64 oracle, as it stands (gcc -O3 -march=native, ISO C11, OpenMP
    over z-planes), on the host cores: cell-updates/s on whole steps of an n^3
    sample of the same workload (its cost per point does not depend on the
    grid), on all cores and on one core."""
    allc = os.cpu_count() or 1
    steps, el, used = _oracle_steps(n, allc, seconds)
    s1, e1, _ = _oracle_steps(n, 1, one_core_seconds)
    from oracle import oracle as O
    O.set_threads(allc)
    return {"value": n ** 3 * steps / el, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{steps} whole steps of the {n}^3 version of the workload (FP64 oracle, gcc -O3 "
                      f"-march=native, OpenMP over z-planes), {el:.1f} s",
            "one_core": {"value": n ** 3 * s1 / e1, "cores": 1,
                         "sample": f"{s1} whole {n}^3 steps on one thread, {e1:.1f} s"}}


def dist_setup():
    from paper_2012_08758_b300.replicas import env
    return env()


def step_config(n, dtype, world, nz=None):
    """config of the step line (shared by both arms)."""
    nz = nz or n
    px = (n + 7 + 7) // 8 * 8
    nbytes = 21 * px * (n + 6) * (nz + 6) * (4 if dtype == "f32" else 8)
    name = workload_name(n, dtype) if nz == n else workload_name(n, dtype).replace(f"{n}^3", f"{n}^2 x {nz}", 1)
    return {"workload": name, "grid": n, "nz": nz, "replicas": world,
            "parallelism": f"replicas x{world} (independent runs, no collective)",
            "l2": "inputs larger than L2 (21 padded arrays, %.2f GB)" % (nbytes / 1e9)}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (there is no
    upstream code).  Each step is a bounded sample of the workload -- one
    whole oracle step of its 64^3 version (the cost per point does not depend
    on the grid) -- W untimed and K timed, so value, ms_per_step and the
    wall time are all this run's own."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2012_08758_b300 import inputs

    ns = 64
    O.use_native()
    cores = O.set_threads(os.cpu_count() or 1)
    p = O.Params(nx=ns, ny=ns, nz=ns, **workload(args.n))
    q = inputs.seed_field_state(ns, seed=0)
    O.run(p, q, args.warmup)
    t0 = time.perf_counter()
    O.run(p, q, args.steps, step0=args.warmup)
    el = time.perf_counter() - t0
    value = ns ** 3 * args.steps / el
    sample = (f"each step: one whole step of the {ns}^3 version of the workload (FP64 oracle, gcc -O3 "
              f"-march=native, OpenMP over z-planes, {cores} threads); {args.warmup} untimed + "
              f"{args.steps} timed steps, {el:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": step_config(args.n, args.dtype, world),
            "sample": {"grid": ns, "cells_per_step": ns ** 3, "note": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.replicas import replica_seed
    from paper_2012_08758_b300.run import Run

    n, dtype = args.n, args.dtype
    nz = args.nz or n  # --nz: an n^2 x nz box (smaller captures of the same x-y structure)
    cells = n * n * nz
    wl = workload(n)
    if nz != n:  # keep the grid spacing isotropic: box 2 pi x 2 pi x 2 pi nz / n
        wl = dict(wl, lz=2 * math.pi * nz / n)
    run = Run(nx=n, ny=n, nz=nz, device=dev, dtype=B.MHD_F32 if dtype == "f32" else B.MHD_F64,
              kernel=args.kernel, tile=args.tile, **dict(wl, seed=wl["seed"] + rank))
    seed_key = replica_seed(0, rank)
    run.set_seed_field(seed_key, SEED_AMP)  # the paper's initial condition, on the device
    # host copy of the initial state (pinned), for the end-to-end leg
    hdt = torch.float32 if dtype == "f32" else torch.float64
    host_in = torch.empty((7, nz, n, n), dtype=hdt).pin_memory().numpy()
    B.mhd_get_state(run.ctx, host_in)
    run.step(args.warmup)
    run.sync()

    from paper_2012_08758_b300 import replicas as RP

    def barrier():
        RP.barrier(dev)

    # --- device-timed region: K steps, events on the context's stream ---
    barrier()
    with ClockSampler(local) as clk:
        stage_ms, total_ms = B.mhd_step_timed(run.ctx, args.steps)
    barrier()
    t_max = RP.max_over_ranks(total_ms / 1e3, dev)
    run.sync()  # raises if the run blew up
    value = RP.job_throughput(world, cells * args.steps, t_max)

    # --- roofline of the dominant kernel (fused substep, 3 launches/step) ---
    sub_ms = sum(stage_ms[1:4])
    bpc = BYTES_PER_CELL[dtype]
    achieved = bpc * cells * args.steps / (sub_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    traffic = ncu_traffic(n, dtype) if nz == n else None
    step_gbs = bpc * cells * args.steps / (total_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_substep (fused RHS + RK3-2N), 3 launches per step",
            "algorithmic_bytes_per_cell_update": bpc, "peak_source": peak_src,
            "traffic_over_algorithmic": None if traffic is None else traffic / (bpc / 3 * cells),
            "whole_step": {"achieved": step_gbs, "frac": step_gbs / peak,
                           "note": "the same algorithmic bytes over the whole step (prologue included)"},
            "stage_ms_per_step": {"prologue": stage_ms[0] / args.steps,
                                  "substep1": stage_ms[1] / args.steps,
                                  "substep2": stage_ms[2] / args.steps,
                                  "substep3": stage_ms[3] / args.steps}}

    # --- end to end through the public API with host buffers ---
    host_out = torch.empty((7, nz, n, n), dtype=hdt).pin_memory().numpy()
    e2e_steps = args.steps
    barrier()
    t0 = time.perf_counter()
    B.mhd_set_state(run.ctx, host_in, 0.0, 0)
    for _ in range(e2e_steps):
        B.mhd_step(run.ctx, 1)
        B.mhd_reduce(run.ctx, B.MHD_BRMS)  # one double back per step
    B.mhd_get_state(run.ctx, host_out)
    barrier()
    e2e_t = RP.max_over_ranks(time.perf_counter() - t0, dev)
    state_bytes = host_in.nbytes
    e2e = {"value": world * cells * e2e_steps / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": state_bytes / e2e_steps,
           "d2h_bytes_per_step": (state_bytes + 8 * e2e_steps) / e2e_steps,
           "note": "per job: state upload from pinned host memory, K x (mhd_step(1) + mhd_reduce(B_rms)), "
                   "state download"}
    run.close()
    del host_in, host_out

    # --- FP64 beside FP32 on the same workload (few steps: ALU-bound) ---
    fp64 = None
    if dtype == "f32" and not args.skip_fp64:
        run64 = Run(nx=n, ny=n, nz=nz, device=dev, dtype=B.MHD_F64, **dict(wl, seed=wl["seed"] + rank))
        run64.set_seed_field(seed_key, SEED_AMP)
        run64.step(1)
        run64.sync()
        k64 = args.fp64_steps
        st64, tot64 = B.mhd_step_timed(run64.ctx, k64)
        d64 = run64.diagnostics()
        run64.close()
        # per-quantity FP32 error against FP64 after the same 1 + k64 steps
        # from the same initial state (the at-scale configuration's check)
        run32 = Run(nx=n, ny=n, nz=nz, device=dev, dtype=B.MHD_F32, **dict(wl, seed=wl["seed"] + rank))
        run32.set_seed_field(seed_key, SEED_AMP)
        run32.step(1 + k64)
        d32 = run32.diagnostics()
        run32.close()
        err32 = {k: abs(d32[k] - d64[k]) / max(abs(d64[k]), 1e-300)
                 for k in ("urms", "brms", "umax", "bmax", "ekin", "emag", "mass", "vmax")}
        sub64 = sum(st64[1:4])
        peaks = alu_peaks()
        fl64 = ncu_flops("f64")
        alu = {"bound": "alu", "peak": peaks["f64"] / 1e12, "unit": "TFLOP/s",
               "peak_source": "measured FP64 FMA chains on this GPU (mhd_alu_peak)",
               "flops_per_cell_update": fl64, "achieved": None, "frac": None}
        if fl64:
            alu["achieved"] = fl64 * cells * k64 / (sub64 / 1e3) / 1e12
            alu["frac"] = alu["achieved"] / alu["peak"]
        fp64 = {"value": cells * k64 / (tot64 / 1e3), "unit": UNIT, "steps": k64, "grid": n,
                "ms_per_step": tot64 / k64,
                "hbm_frac": BYTES_PER_CELL["f64"] * cells * k64 / (sub64 / 1e3) / 1e9 / peak,
                "roofline": alu,
                "fp32_rel_err": {"steps": 1 + k64, **err32},
                "fma_peaks_tflops": {k: v / 1e12 for k, v in peaks.items()}}
        fl32 = ncu_flops("f32")
        if fl32:
            roof["alu"] = {"achieved": fl32 * cells * args.steps / (sub_ms / 1e3) / 1e12,
                           "peak": peaks["f32"] / 1e12, "unit": "TFLOP/s",
                           "flops_per_cell_update": fl32,
                           "peak_source": "measured FP32 FMA chains on this GPU (mhd_alu_peak)"}
            roof["alu"]["frac"] = roof["alu"]["achieved"] / roof["alu"]["peak"]

    # --- batched ensemble and serving loop (C4, C5), rank 0 of a 1-GPU job ---
    batch = serve = None
    if world == 1 and not args.skip_batch:
        batch = measure_batch(steps=args.batch_steps, warmup=3, tune=False)
    if world == 1 and not args.skip_serve:
        serve = measure_serve(requests=args.requests, rate=args.serve_rate, scale=args.serve_scale,
                              chunk=args.serve_chunk, checks=args.serve_checks)

    cb = cpu_baseline() if (rank == 0 and world == 1 and not args.skip_cpu) else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": step_config(n, dtype, world, nz),
                "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "fp64": fp64,
                "batch": batch, "serving": serve,
                "gpu_launches": 4 * args.steps, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


BATCH_SIZES = [64] * 16 + [128] * 8


def measure_batch(steps=20, warmup=3, tune=True):
    """C4: 16 x 64^3 + 8 x 128^3 runs, nu = eta log-spaced for Re_M 5-250,
    alternating helicity, FP32 with FP64 reductions; one batch (one launch
    per kernel stage over the combined tile table, k steps replayed from a
    CUDA graph) against the same runs stepped one at a time.  Device time
    with CUDA events on the runs' stream."""
    import torch

    from paper_2012_08758_b300 import autotune
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.run import Batch, Run

    sizes = BATCH_SIZES
    rems = np.exp(np.linspace(np.log(5.0), np.log(250.0), len(sizes)))
    best = autotune.tune([(n, n, n) for n in sizes], B.MHD_F32, steps=3) if tune else \
        {"kernel": 0, "tile": 0, "note": "default variant (no autotuning in this line)"}
    cells = sum(n ** 3 for n in sizes)

    def make():
        runs = []
        for i, (n, rem) in enumerate(zip(sizes, rems)):
            nu = URMS0 / (rem * KF)
            r = Run(n=n, nu=nu, eta=nu, f0=0.02, sigma=float(i % 2), seed=100 + i, kernel=best["kernel"],
                    tile=best["tile"])
            r.set_seed_field(10_000 + i, SEED_AMP)
            runs.append(r)
        return runs

    runs = make()
    b = Batch(runs)
    b.step(warmup)
    torch.cuda.synchronize()
    stream = runs[0].stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    for r in runs:
        r.sync()
    b.close()
    for r in runs:
        r.close()
    runs = make()
    for r in runs:
        r.step(warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    for r in runs:
        r.step(steps)
    e1.record(stream)
    e1.synchronize()
    t_serial = e0.elapsed_time(e1) / 1e3
    for r in runs:
        r.close()
    return {"workload": "batch: 16x64^3 + 8x128^3, Re_M 5-250 log-spaced, sigma 0/1 alternating, FP32",
            "unit": UNIT, "steps": steps, "warmup": warmup,
            "batched": cells * steps / t_batch, "one_at_a_time": cells * steps / t_serial,
            "speedup": t_serial / t_batch, "variant": best, "cells": cells,
            "launches": "4 per step (prologue + 3 substeps) over all 24 runs, replayed from a CUDA graph"}


def measure_serve(requests=200, rate=4.0, scale=0.1, chunk=25, checks=6):
    """C5: Poisson stream of seeded requests (grid uniform over {64, 96, 128,
    192, 256}, Re_M log-uniform 10-250, sigma in {0, 1}); the step budgets
    are the config's 500-5000 times `scale`.  Continuous batching under a
    150 GB HBM budget; p50/p99 latency and aggregate throughput, against
    serial FP64 stepping of the same work (per-size FP64 rates measured here)
    and growth rates against FP64 runs of the smallest requests."""
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.growth import brms_series, fit_last
    from paper_2012_08758_b300.run import Run
    from paper_2012_08758_b300.serving import Server, requests_from_inputs, run_params, start, summarize

    lo, hi = max(int(500 * scale), 20), max(int(5000 * scale), 40)
    reqs = requests_from_inputs(n=requests, seed=2025, rate=rate, steps=(lo, hi))
    srv = Server(budget_bytes=150e9, chunk=chunk)
    t0 = time.perf_counter()
    res = srv.serve(reqs, realtime=True)
    wall = time.perf_counter() - t0
    summ = summarize(res, wall, srv.stepped_cells)
    # serial FP64: measured rate per grid size on short runs
    rates = {}
    for n in sorted({r.n for r in reqs}):
        rr = Run(n=n, dtype=B.MHD_F64, f0=0.02, seed=1)
        start(rr, reqs[0].__class__(0, 0, n, 100.0, 1.0, 10, 1))
        rr.step(1)
        st, tot = B.mhd_step_timed(rr.ctx, 3)
        rates[n] = n ** 3 * 3 / (tot / 1e3)
        rr.close()
    work = sum(r.n ** 3 * r.steps for r in reqs)
    t_serial64 = sum(r.n ** 3 * r.steps / rates[r.n] for r in reqs)
    # growth-rate accuracy: the served FP32 result equals the FP32 run alone
    # (tested bit for bit), so FP32 and FP64 runs of the same request with the
    # same sampling are compared, for the smallest requests
    cks = []
    for r in sorted(reqs, key=lambda q: q.n ** 3 * q.steps)[:checks]:
        lam = {}
        for dt in (B.MHD_F32, B.MHD_F64):
            rr = Run(**run_params(r, dtype=dt))
            start(rr, r)
            ts, bs = brms_series(rr, r.steps, max(1, r.steps // 40))
            rr.close()
            lam[dt] = fit_last(ts, bs, 0.5)
        cks.append({"id": r.id, "n": r.n, "steps": r.steps, "lambda_f32": lam[B.MHD_F32],
                    "lambda_f64": lam[B.MHD_F64],
                    "rel_diff": abs(lam[B.MHD_F32] - lam[B.MHD_F64]) / max(abs(lam[B.MHD_F64]), 1e-300)})
    return {"workload": f"serve: {requests} Poisson requests (rate {rate}/s), step budgets {lo}-{hi} "
                        f"(the config's 500-5000 scaled by {scale}), FP32 continuous batching, 150 GB budget",
            "metric": "p50/p99 job latency and aggregate cell-updates/s", "budget_scale": scale, **summ,
            "serial_fp64_cell_updates_per_s": work / t_serial64,
            "speedup_vs_serial_fp64": summ["cell_updates_per_s"] / (work / t_serial64),
            "fp64_rates": rates, "growth_rate_checks": cks,
            "max_growth_rate_rel_diff": max((c["rel_diff"] for c in cks), default=None)}


def run_batch(args):
    line = measure_batch(steps=args.steps, warmup=args.warmup, tune=not args.no_tune)
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    line = measure_serve(requests=args.requests, rate=args.serve_rate, scale=args.serve_scale,
                         chunk=args.serve_chunk, checks=args.serve_checks)
    print(json.dumps(line), flush=True)
    return 0


def run_paper_protocol(args):
    """The paper's timing protocol (App. A): all seven fields uniform in
    [0, 1), fixed dt = 1.19209e-7, forcing off, 10 warm-up steps, then
    per-step device times of 100 steps; p50 / p90 and ns per step per
    point."""
    import torch

    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300 import inputs
    from paper_2012_08758_b300.run import Run

    n = args.n
    dt = B.MHD_F32 if args.dtype == "f32" else B.MHD_F64
    run = Run(n=n, dtype=dt, kernel=args.kernel, tile=args.tile,
              **dict(WORKLOAD, f0=0.0, dt_fixed=1.19209e-7))
    run.set_state(inputs.uniform_state(n, seed=0, dtype=np.float32 if dt == B.MHD_F32 else np.float64))
    run.step(10)
    run.sync()
    steps = max(args.steps, 100)
    ms = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(steps):
            ms.append(B.mhd_step_timed(run.ctx, 1)[1])
    run.sync()
    run.close()
    ms.sort()
    p50, p90 = ms[len(ms) // 2], ms[int(0.9 * (len(ms) - 1))]
    line = {"workload": f"{n}^3, all fields U[0,1), dt = 1.19209e-7, forcing off ({args.dtype.upper()}), "
                        f"10 warm-up + {steps} timed steps",
            "p50_ms": p50, "p90_ms": p90, "ns_per_step_per_point_p50": p50 * 1e6 / n ** 3,
            "cell_updates_per_s_p50": n ** 3 / (p50 / 1e3), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_spectrum(args):
    """Magnetic energy spectrum (Sec. 5) of the n^3 workload state after a
    few steps: device time of one mhd_spectrum call (curl, cuFFT
    real-to-complex transform, shell sums, copy of the shells), p50 of 10."""
    import torch

    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300 import inputs
    from paper_2012_08758_b300.run import Run

    n = args.n
    dt = B.MHD_F32 if args.dtype == "f32" else B.MHD_F64
    run = Run(n=n, dtype=dt, **WORKLOAD)
    run.set_state(inputs.seed_field_state(n, seed=0))
    run.step(args.warmup)
    E = run.spectrum()
    emag = run.diagnostics()["emag"]
    ms = []
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(run.stream)
        run.spectrum()
        e1.record(run.stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    run.close()
    ms.sort()
    line = {"workload": f"magnetic spectrum E_B(k) of the {n}^3 workload state ({args.dtype.upper()}), "
                        f"{len(E)} shells",
            "p50_ms": ms[len(ms) // 2], "cells_per_s": n ** 3 / (ms[len(ms) // 2] / 1e3),
            "parseval_rel": abs(E.sum() - emag) / emag, "shells": len(E)}
    print(json.dumps(line), flush=True)
    return 0


def paper_tables():
    """Growth rates and Re_M printed in the paper's Tables 1 and 2 (stored
    with their citation in tests/golden)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "growth_rates_tables_1_2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, n, eta, lam, rem = line.split()
            rows.append(dict(sigma=float(s), n=int(n), eta=float(eta), lam=float(lam), rem=float(rem)))
    return rows


def run_tables(args):
    """Kinematic growth rates at the setup of the paper's Tables 1-2 (rows of
    the chosen grids, --tables-seeds forcing realisations each), stepped as one
    FP32 batch to t = --tables-tmax (paper_2012_08758_b300.tables); the JSON
    record goes to stdout and, with --tables-out, to that file."""
    from paper_2012_08758_b300 import tables

    grids = [int(g) for g in args.tables_grids.split(",")]
    etas = [float(e) for e in args.tables_eta.split(",")] if args.tables_eta else None
    rows = [dict(r, realisation=s) for r in paper_tables() if r["n"] in grids and (etas is None or r["eta"] in etas)
            for s in range(args.tables_seeds)]
    res = tables.run_rows(rows, f0=args.tables_f0, tmax=args.tables_tmax, chunk=args.tables_chunk,
                          upwind=args.tables_upwind, spectra=args.tables_spectra, series=args.tables_series)
    line = {"workload": f"growth rates at the setup of Tables 1-2, grids {grids}, "
                        f"{args.tables_seeds} realisation(s) per row, t <= {args.tables_tmax}",
            "command": "python bench.py " + " ".join(sys.argv[1:]), **res}
    if args.tables_out:
        with open(args.tables_out, "w") as f:
            json.dump(line, f, indent=1)
    print(json.dumps(line), flush=True)
    return 0


def run_c2(args):
    """C2: the 256^3 FP32 workload for 2000 steps (device-timed throughput
    and achieved HBM bandwidth of the fused substeps), and the growth rate
    of ln B_rms over the first 300 steps in FP32 against the same 300 steps
    in FP64 on the GPU (the FP64 path is the one pinned to the oracle; the
    oracle itself would need hours for 256^3 x 300)."""
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300 import inputs
    from paper_2012_08758_b300.growth import brms_series, fit_last
    from paper_2012_08758_b300.run import Run

    n = args.n
    q0 = inputs.seed_field_state(n, seed=0)
    run = Run(n=n, dtype=B.MHD_F32, **WORKLOAD)
    run.set_state(q0)
    run.step(args.warmup)
    run.sync()
    stage_ms, total_ms = B.mhd_step_timed(run.ctx, 2000)
    run.sync()
    run.close()
    out = {}
    for dt in (B.MHD_F32, B.MHD_F64):
        r = Run(n=n, dtype=dt, **WORKLOAD)
        r.set_state(q0)
        ts, bs = brms_series(r, 300, 10)
        r.close()
        out[dt] = (ts, bs, fit_last(ts, bs, 0.5))
    la, lb = out[B.MHD_F32][2], out[B.MHD_F64][2]
    line = {"workload": f"C2: {n}^3 FP32, " + workload_name(n, "f32") + ", 2000 steps",
            "cell_updates_per_s": n ** 3 * 2000 / (total_ms / 1e3), "ms_per_step": total_ms / 2000,
            "substep_gbs": BYTES_PER_CELL["f32"] * n ** 3 * 2000 / (sum(stage_ms[1:4]) / 1e3) / 1e9,
            "lambda_f32_first_300": la, "lambda_f64_first_300": lb, "lambda_rel": abs(la - lb) / abs(lb),
            "brms_rel_max": float(np.max(np.abs(out[B.MHD_F32][1] - out[B.MHD_F64][1]) / out[B.MHD_F64][1]))}
    print(json.dumps(line), flush=True)
    return 0


def run_slabs(args):
    """The decomposed run on one GPU: device time per step of the n^3
    workload cut into 1, 2 and 4 z-slabs, with and without overlapping the
    halo exchange with the inner planes, against the undecomposed run (the
    cost of the decomposition's outer/inner split and copies on one GPU)."""
    import torch

    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.run import Run
    from paper_2012_08758_b300.slabs import Slabs

    n = args.n
    wl = workload(n)
    dt = B.MHD_F32 if args.dtype == "f32" else B.MHD_F64
    out = {}
    run = Run(n=n, dtype=dt, **wl)
    run.set_seed_field(1, SEED_AMP)
    run.step(args.warmup)
    run.sync()
    st, tot = B.mhd_step_timed(run.ctx, args.steps)
    out["undecomposed"] = tot / args.steps
    q = run.get_state(dtype=np.float32 if dt == B.MHD_F32 else np.float64)[0]
    run.close()
    stream = torch.cuda.Stream()
    for ns in (1, 2, 4):
        for ov in (0, 1):
            sl = Slabs(ns, n=n, dtype=dt, overlap=bool(ov), stream=stream, **wl)
            sl.set_state(q)
            sl.step(args.warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sl.step(args.steps)
            e1.record(stream)
            e1.synchronize()
            out[f"{ns}_slabs_overlap{ov}"] = e0.elapsed_time(e1) / args.steps
            sl.close()
    line = {"workload": f"{n}^3 {args.dtype.upper()} step decomposed into z-slabs on one GPU", "ms_per_step": out,
            "steps": args.steps}
    print(json.dumps(line), flush=True)
    return 0


def run_cpu(args):
    """The FP64 oracle timed on the host: one core and all cores, whole steps
    at 64^3 and 128^3 (per-cell cost, which extrapolates to 512^3 by the
    point count)."""
    from oracle import oracle as O
    from paper_2012_08758_b300 import inputs

    allc = os.cpu_count() or 1
    res = []
    for n, cores in ((64, 1), (64, allc), (128, allc)):
        used = O.set_threads(cores)
        p = O.Params(nx=n, ny=n, nz=n, **WORKLOAD)
        q = inputs.seed_field_state(n, seed=0)
        t0 = time.perf_counter()
        O.run(p, q, 1)
        el = time.perf_counter() - t0
        res.append({"n": n, "cores": used, "s_per_step": el, "cell_updates_per_s": n ** 3 / el,
                    "ns_per_point_step": el * 1e9 / n ** 3})
    O.set_threads(allc)
    print(json.dumps({"workload": "FP64 oracle on the host cores, one whole step", "runs": res}), flush=True)
    return 0


def run_fp32vs64(args):
    """C3: the same initial state advanced in FP32 and in FP64 on the GPU;
    per-quantity FP32 error against FP64 (fields, rms values, energies,
    growth rate of ln B_rms over the second half)."""
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300 import inputs
    from paper_2012_08758_b300.growth import brms_series, fit_last
    from paper_2012_08758_b300.run import Run

    n = args.n
    wl = dict(WORKLOAD, nu=1.25e-4, eta=1.25e-4)  # Re_M ~ 250 at u_rms ~ 0.05 (512^3 config)
    q0 = inputs.seed_field_state(n, seed=0, amp=1e-5)
    out = {}
    for dt in (B.MHD_F32, B.MHD_F64):
        r = Run(n=n, dtype=dt, **wl)
        r.set_state(q0)
        t0 = time.perf_counter()
        ts, bs = brms_series(r, args.steps, max(1, args.steps // 20))
        el = time.perf_counter() - t0
        st, t, _ = r.get_state(dtype=np.float32 if dt == B.MHD_F32 else np.float64)
        out[dt] = dict(state=st.astype(np.float64), diag=r.diagnostics(), ts=ts, bs=bs, wall=el)
        r.close()
    a, b = out[B.MHD_F32], out[B.MHD_F64]
    umax = np.abs(b["state"][1:4]).max()
    amax = np.abs(b["state"][4:7]).max()
    scales = [max(np.abs(b["state"][0]).max(), umax), umax, umax, umax, amax, amax, amax]
    field_err = {name: float(np.abs(a["state"][i] - b["state"][i]).max() / scales[i])
                 for i, name in enumerate(("lnrho", "ux", "uy", "uz", "Ax", "Ay", "Az"))}
    diag_err = {k: abs(a["diag"][k] - b["diag"][k]) / max(abs(b["diag"][k]), 1e-300)
                for k in ("urms", "brms", "ekin", "emag", "umax", "bmax", "mass")}
    la, lb = fit_last(a["ts"], a["bs"], 0.5), fit_last(b["ts"], b["bs"], 0.5)
    line = {"workload": f"{n}^3 helical forcing, Re_M ~ 250 (nu = eta = 1.25e-4), {args.steps} steps, FP32 vs FP64",
            "field_rel_linf": field_err, "diag_rel": diag_err, "lambda_f32": la, "lambda_f64": lb,
            "lambda_rel": abs(la - lb) / max(abs(lb), 1e-300), "t_end": b["ts"][-1],
            "wall_s": {"f32": a["wall"], "f64": b["wall"]}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--nz", type=int, default=0, help="z planes of the step workload (default: n)")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--workload", choices=["step", "batch", "serve", "fp32vs64", "paper", "spectrum", "tables",
                                           "c2", "cpu", "slabs"],
                    default="step",
                    help="step: the benchmark line; the others measure the batch (16x64^3+8x128^3), "
                         "serving and FP32-vs-FP64 configurations and the paper's timing protocol")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=4.0,
                    help="request arrivals per second (4/s is about 0.9x the batched capacity: a request "
                         "averages 1.5e9 cell-updates at the scaled budgets, the batch steps 6.5e9 per second)")
    ap.add_argument("--serve-scale", type=float, default=0.1, help="scale of the 500-5000 step budgets")
    ap.add_argument("--serve-chunk", type=int, default=25)
    ap.add_argument("--serve-checks", type=int, default=6)
    ap.add_argument("--tables-grids", default="64", help="grids of the Tables 1-2 rows to run")
    ap.add_argument("--tables-tmax", type=float, default=400.0)
    ap.add_argument("--tables-chunk", type=int, default=200)
    ap.add_argument("--tables-f0", type=float, default=0.029)
    ap.add_argument("--tables-out", default="", help="also write the tables record (JSON) to this file")
    ap.add_argument("--tables-eta", default="", help="comma-separated eta values to keep (default: all rows)")
    ap.add_argument("--tables-seeds", type=int, default=1, help="forcing realisations per table row")
    ap.add_argument("--tables-series", action="store_true", help="include the (t, B_rms, u_rms) samples")
    ap.add_argument("--tables-upwind", type=int, default=1, help="upwinding of the continuity equation (0/1)")
    ap.add_argument("--tables-spectra", action="store_true",
                    help="also sample E_B(k) and fit the growth rates of channels k = 1, 5, 9 (Sec. 5)")
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 plane ring, 2 TMA")
    ap.add_argument("--tile", type=int, default=0, help="tile variant id (0: default)")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU-baseline leg")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the FP64 side measurement")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 leg")
    ap.add_argument("--skip-batch", action="store_true", help="omit the batched-ensemble leg")
    ap.add_argument("--skip-serve", action="store_true", help="omit the serving leg")
    ap.add_argument("--batch-steps", type=int, default=20, help="timed steps of the batched-ensemble leg")
    ap.add_argument("--no-tune", action="store_true", help="batch workload: default variant, no autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "fp32vs64":
        return run_fp32vs64(args)
    if args.workload == "paper":
        return run_paper_protocol(args)
    if args.workload == "spectrum":
        return run_spectrum(args)
    if args.workload == "tables":
        return run_tables(args)
    if args.workload == "c2":
        return run_c2(args)
    if args.workload == "cpu":
        return run_cpu(args)
    if args.workload == "slabs":
        return run_slabs(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
