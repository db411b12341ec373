#!/usr/bin/env python3
"""Benchmark of one MPRK2 slow step on one GB300 (C ABI of libmprk.so).

A bench step is one slow step of the whole hot path (2m fused stage launches
plus the step completion) on the 2048x1024-cell, m = 8, FP64 workload
(S/B/F = 480/64/480 rows, Fourier-mode perturbations). The metric is
cell-stage updates per second: cell right-hand-side evaluations per slow step,
nx (2 nS + 2 m (nB + nF)) (Sec. 4 of the paper), times steps, over the time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Prints one JSON line. With N > 1 (torchrun) each rank runs its own replica of
the workload (the path does not shard) and the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2202_11890_gb300 import workloads as W  # noqa: E402

METRIC = "cell-stage updates/s"
# stage launches dominate; algorithmic work per cell-stage
FP64_FLOPS_PER_CELL_STAGE = 418.0
FP32_FLOPS_PER_CELL_STAGE = 418.0
HBM_BYTES_PER_CELL_STAGE_FP64 = 80.0
HBM_BYTES_PER_CELL_STAGE_FP32 = 64.0
# FP64 unit count x clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07


def workload(name: str) -> W.Workload:
    return {"large_2048": W.large_2048, "plain_64": W.plain_64, "mixed_4096": W.mixed_4096}[name]()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2202_11890_gb300 import build as B
    from paper_2202_11890_gb300 import mprk as M
    from paper_2202_11890_gb300 import timing as T

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    wl = workload(args.workload)
    if args.precision:
        wl.precision = args.precision
    g = wl.grid
    q0 = wl.initial_state()
    cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m)
    cfg.precision = M.MPRK_FP32FLUX if wl.precision == "fp32flux" else M.MPRK_FP64
    inst = M.Instance(cfg, q0)
    info = inst.info()
    cs = info["cell_stages_per_step"]
    stream = info["stream"]
    launches_per_step = 2 * wl.m + 1

    # warm-up
    inst.step(args.warmup)
    inst.sync()

    # timed region: K slow steps, CUDA events on the instance stream, plus the
    # stage kernel's own launches bracketed by events inside the graph-free
    # stage timer (T.stage_kernel_times) run afterwards on the same state
    sampler = ClockSampler(torch.cuda.current_device())
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with sampler:
        t_ms = T.time_steps(inst.h, stream, args.steps)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t = torch.tensor([t_ms], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_ms = float(t.item())
    value = cs * args.steps * ws / (t_ms * 1e-3)

    # dominant kernel: average duration of one stage launch (events on the
    # instance stream around each launch of one un-captured slow step)
    stage_ms, stage_cells = T.stage_kernel_times(inst.h, stream, reps=3)
    fp64 = cfg.precision == M.MPRK_FP64
    flops = FP64_FLOPS_PER_CELL_STAGE if fp64 else FP32_FLOPS_PER_CELL_STAGE
    peak = FP64_PEAK_GFLOPS if fp64 else FP32_PEAK_GFLOPS
    # achieved over all stage launches of a step: algorithmic work / kernel time
    ach_gflops = stage_cells * flops / (stage_ms * 1e-3) / 1e9
    peaks, src = measured_peaks()
    hbm_bytes = HBM_BYTES_PER_CELL_STAGE_FP64 if fp64 else HBM_BYTES_PER_CELL_STAGE_FP32
    ach_gbs = stage_cells * hbm_bytes / (stage_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: pinned host state in,
    # one slow step, state out, every step
    pin_in = torch.from_numpy(q0).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        M.mprk_set_state(inst.h, pin_in)
        M.mprk_step(inst.h, 1)
        M.mprk_get_state(inst.h, pin_out)
    e2e_s = time.perf_counter() - t0
    nbytes = q0.nbytes
    e2e_value = cs * e2e_steps * ws / e2e_s
    inst.close()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "cell-stages/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if fp64 else "f32 flux / f64 accumulate", "data": "synthetic",
            "config": {"workload": wl.name, "nx": g.nx, "nz": g.nz, "rows_S_B_F": [g.nS, g.nB, g.nF],
                       "m": wl.m, "cell_stages_per_step": cs, "parallelism": f"replicas x{ws}",
                       "l2": "working set > L2 (about 4 states of 67 MB); no flush"},
            "roofline": {"bound": "alu", "achieved": ach_gflops, "peak": peak,
                         "unit": "GFLOP/s", "frac": ach_gflops / peak, "traffic": None,
                         "peak_source": "FP64 unit count x max clock (152 SMs x 2 DFMA/clk)"
                         if fp64 else "FP32 unit count x max clock",
                         "hbm_achieved_gbs": ach_gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                         "hbm_frac": ach_gbs / peaks["hbm_gbs"], "hbm_peak_source": src},
            "e2e": {"value": e2e_value, "unit": "cell-stages/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "steps": e2e_steps},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": sampler.summary(),
        }
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


def oracle_sample(wl: W.Workload, cols: int):
    """The workload's rows, rate and perturbation on a strip of `cols` columns
    (the oracle's cost per cell-stage does not depend on nx)."""
    g = wl.grid
    sg = W.Grid(cols, g.nS, g.nB, g.nF, dx=g.dx, dz1=g.dz1, dz2=g.dz2)
    sw = W.Workload(wl.name + f"_strip{cols}", sg, wl.m, 1, wl.precision, wl.perturbation, wl.seed)
    return sw


def cpu_baseline(wl: W.Workload, cols: int = 512, budget_s: float = 10.0, max_steps: int = 8):
    """The oracle as it stands, all host cores, on slow steps of a strip of
    the workload (same rows, m and perturbation), repeated until about
    budget_s seconds of CPU work."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    sw = oracle_sample(wl, cols)
    g = sw.grid
    q = sw.initial_state()
    P = O.make_problem(g.nx, g.nS, g.nB, g.nF, sw.m, 0.0, g.dx, dz1=g.dz1, dz2=g.dz2)
    P.dt = O.stable_dt(P, q, 0.4)
    t0 = time.perf_counter()
    total, steps = 0, 0
    while steps < max_steps and (time.perf_counter() - t0) < budget_s:
        q, cnt = O.mprk_step(P, q, 1)
        total += cnt
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": total / dt, "unit": "cell-stages/s", "cores": O.get_threads(), "kind": "oracle",
            "sample": f"{steps} slow steps of the {wl.name} rows on a {cols}-column strip "
                      f"({total} cell-stages, {dt:.1f} s)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    wl = workload(args.workload)
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    cols = args.ref_cols
    sw = oracle_sample(wl, cols)
    g = sw.grid
    q = sw.initial_state()
    P = O.make_problem(g.nx, g.nS, g.nB, g.nF, sw.m, 0.0, g.dx, dz1=g.dz1, dz2=g.dz2)
    P.dt = O.stable_dt(P, q, 0.4)
    for _ in range(args.warmup):
        q, cnt = O.mprk_step(P, q, 1)
    t0 = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        q, cnt = O.mprk_step(P, q, 1)
        total += cnt
    el = time.perf_counter() - t0
    value = total / el
    out = {
        "metric": METRIC, "value": value, "unit": "cell-stages/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": wl.name, "sample": f"{cols}-column strip of the same rows and m"},
        "cpu_baseline": {"value": value, "unit": "cell-stages/s", "cores": O.get_threads(),
                         "kind": "oracle",
                         "sample": f"each step: one oracle slow step on a {cols}-column strip "
                                   f"of {wl.name}"},
        "e2e": {"value": value, "unit": "cell-stages/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_2048", choices=["large_2048", "plain_64", "mixed_4096"])
    ap.add_argument("--precision", default="", choices=["", "fp64", "fp32flux"])
    ap.add_argument("--ref-cols", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
