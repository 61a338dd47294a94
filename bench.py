#!/usr/bin/env python
"""Benchmark: unknowns/s solved to 1e-10 relative residual on one GB300.

Workload (default): the 4095 x 4095 cell-centred diffusion problem with
64 x 64-cell blocks of k = 10^U, U ~ uniform[-4, 4] (seed 1), uniform[-1, 1]
right-hand side, plain FP64 BoxMG V(2,1) cycles.  A step is the whole hot
path on device-resident inputs: setup (assembly, interpolation, Galerkin
coarse operators, coarsest Cholesky) and the solve from x = 0 to
||b - A x|| / ||b|| <= 1e-10.  value = fine unknowns x steps / device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own copy (independent problems,
weak scaling, no collective on the data path).  ``--impl reference`` times
the CPU oracle on a bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_02481_gb300 import inputs  # noqa: E402

METRIC = "unknowns/s solved to 1e-10 rel. residual (FP64 vs FP32+refine); HBM % of peak"
UNIT = "unknowns/s"
TOL = 1e-10
N_SIDE = 4095
WORKLOAD = {"workload": "diffusion 4095x4095, 64x64-cell blocks k=10^U(-4,4), seed 1, V(2,1), tol 1e-10",
            "nx": N_SIDE, "ny": N_SIDE, "block": 64, "contrast_log10": [-4, 4], "seed": 1,
            "cycle": "V(2,1)", "smoother": "red-black GS (fine), 4-colour GS (coarse)", "tol": TOL}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the
    timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(window=511, budget_note=""):
    """The oracle, as it stands, on a bounded window of the same field."""
    from oracle import boxmg_oracle as O
    pr = inputs.block_problem(N_SIDE, seed=1, block=64, lo=-4, hi=4)
    k = np.ascontiguousarray(pr["k"][:window, :window])
    b = np.ascontiguousarray(pr["b"][:window, :window])
    t0 = time.perf_counter()
    h = O.setup(k)
    r = O.solve(h, b, tol=TOL, max_cycles=1000)
    dt = time.perf_counter() - t0
    return {"value": window * window / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle setup+solve to 1e-10 of the top-left {window}x{window} window of the "
                      f"same block field ({window // 64 + 1}x{window // 64 + 1} blocks), "
                      f"{r.cycles} cycles, {dt:.1f} s, numpy single thread{budget_note}"}


def run_reference(args, rank, world):
    if world > 1 and rank != 0:
        return
    window = 255
    from oracle import boxmg_oracle as O
    pr = inputs.block_problem(N_SIDE, seed=1, block=64, lo=-4, hi=4)
    k = np.ascontiguousarray(pr["k"][:window, :window])
    b = np.ascontiguousarray(pr["b"][:window, :window])
    times = []
    cycles = 0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        h = O.setup(k)
        r = O.solve(h, b, tol=TOL, max_cycles=1000)
        dt = time.perf_counter() - t0
        cycles = r.cycles
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = window * window * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, sample_window=window),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"oracle setup+solve of the top-left {window}x{window} window of the "
                                       f"same block field per step, {cycles} cycles, numpy single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1803_02481_gb300 as bm
    from paper_1803_02481_gb300 import build as bld
    bld.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    pr = inputs.block_problem(N_SIDE, seed=1, block=64, lo=-4, hi=4)
    n_fine = N_SIDE * N_SIDE
    k = torch.from_numpy(pr["k"]).to(dev)
    b = torch.from_numpy(pr["b"]).to(dev)
    x = torch.zeros_like(b)
    opts = bm.default_options(precision=bm.BMG_FP64 if args.precision == "fp64" else bm.BMG_FP32_REFINE)
    if args.threshold is not None:
        opts.coarse_threshold = args.threshold

    def step():
        x.zero_()
        h = bm.setup(k, opts, stream=stream)
        _, info = h.solve(b, x, tol=TOL, stream=stream)
        h.destroy()
        return info

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    prof_kind = bm.BMG_PROF_FINE_SMOOTH
    bm.profile_set(prof_kind)
    launches0 = bm.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = bm.kernel_launches() - launches0
    nprof, prof_ms = bm.profile_read()
    bm.profile_set(bm.BMG_PROF_NONE)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n_fine * args.steps * world / (ms / 1e3)
    info = infos[-1]

    # FP32 + refinement on the same workload (one extra timed pass)
    extra = {}
    if args.precision == "fp64" and not args.quick:
        opts32 = bm.default_options(precision=bm.BMG_FP32_REFINE)

        def step32():
            x.zero_()
            h = bm.setup(k, opts32, stream=stream)
            _, inf = h.solve(b, x, tol=TOL, stream=stream)
            h.destroy()
            return inf
        step32()
        torch.cuda.synchronize()
        ev0.record(stream)
        reps = max(1, args.steps // 2)
        for _ in range(reps):
            i32 = step32()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms32 = ev0.elapsed_time(ev1) / reps
        extra["fp32_refine"] = {"value": n_fine / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32,
                                "refinement_steps": i32.cycles, "rel_resid": i32.rel_resid,
                                "speedup_vs_fp64": (ms / args.steps) / ms32}

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.quick:
        kh = torch.from_numpy(pr["k"]).pin_memory()
        bh = torch.from_numpy(pr["b"]).pin_memory()
        xh = torch.zeros_like(bh).pin_memory()
        kn, bn, xn = kh.numpy(), bh.numpy(), xh.numpy()
        reps = max(1, args.steps // 2)
        bm.solve_host(kn, bn, xn, opts, TOL, stream=stream)
        tot = 0.0
        for _ in range(reps):
            xn[...] = 0.0
            torch.cuda.synchronize()
            ev0.record(stream)
            bm.solve_host(kn, bn, xn, opts, TOL, stream=stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            tot += ev0.elapsed_time(ev1)
        e2e = {"value": n_fine * world / (tot / reps / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * n_fine, "d2h_bytes_per_step": 8 * n_fine,
               "ms_per_step": tot / reps}

    peaks, peak_kind = load_peaks()
    # fine-level smoothing: one bracket = one full red-black sweep (2 colour
    # launches); algorithmic bytes per fine unknown: 1/C, W, S, b, x read,
    # x written = 48 B (FP64)
    per_unit = 48.0 if args.precision == "fp64" else 24.0
    sweep_ms = prof_ms / max(1, nprof)
    achieved = per_unit * n_fine / (sweep_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "kernel": "fine-level red-black Gauss-Seidel sweep (k_relax_colour x2)",
                "per_launch_ms": sweep_ms, "launches_timed": nprof, "peak_source": peak_kind,
                "algorithmic_bytes_per_unknown": per_unit}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": dict(WORKLOAD, precision=args.precision, l2="inputs and hierarchy larger than L2",
                           parallelism=f"replicas{world}"),
            "cycles": info.cycles, "rel_resid": info.rel_resid, "threshold": info.threshold,
            "setup_ms": info.setup_ms, "gpu_launches": int(launches), "roofline": roofline, "e2e": e2e,
            "clocks": clk.summary(), **extra}
    if rank == 0 and not args.quick and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--threshold", type=int, default=None)
    ap.add_argument("--quick", action="store_true", help="skip the e2e, fp32 and CPU legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
