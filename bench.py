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
# Algorithmic floating-point operations per cell-stage of the stage kernel,
# counted from its formulas (+ - * / sqrt each 1, a*b+c 2): 130 per face
# (LF flux 92, viscous flux 26, reconstruction 8, F* assembly 4) times 2.156
# faces per cell of a 32x8 tile, plus ring primitives 14.6, slopes 28.8,
# divergence and source 24, stage combination 8. The FP32-flux form adds
# the reference/deviation sums: 12 per face.
FLOPS_PER_CELL_STAGE = {True: 355.7, False: 381.6}
# Nominal unit counts of the GB300 for context: 152 SMs x 2 DFMA/clk x
# 2 flop x 2.07 GHz, and 128 FP32 lanes per SM. The FP64 roofline's peak is
# measured on the box by the library's register-only FMA probe
# (mprk_probe_fp64), like the HBM peak is a measured copy.
FP64_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.07
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07
_FP64_PROBE = None


def fp64_peak():
    """(peak GFLOP/s, source, probe) of the FP64 units: the unit count taken
    from the device (its SM count and peak SM clock) at 2 DFMA per SM clock,
    with the register-only FMA probe's measured rate beside it (run once per
    process). The unit-count figure is the larger, so fractions against it
    are the conservative ones."""
    global _FP64_PROBE
    if _FP64_PROBE is None:
        from paper_2202_11890_gb300 import mprk as M
        _FP64_PROBE = M.mprk_probe_fp64()
    p = _FP64_PROBE
    peak = p["sms"] * 2 * 2 * p["max_mhz"] / 1e3
    src = (f"unit count of the device: {p['sms']} SMs x 2 DFMA/clk x 2 flop x {p['max_mhz']:.0f} MHz peak clock "
           f"(cudaDevAttrMultiProcessorCount, cudaDevAttrClockRate) = {peak:.1f} GFLOP/s; the register-only FMA "
           f"probe (mprk_probe_fp64) measured {p['gflops']:.1f} GFLOP/s ({p['dfma_per_clk_per_sm']:.2f} DFMA/clk/SM "
           f"at {p['sm_mhz']:.0f} MHz), {p['gflops'] / peak:.2f} of it")
    return peak, src, p

# DRAM traffic of the stage kernel (dram__bytes_read.sum + dram__bytes_write.sum)
# summed over the 2m stage launches of one slow step of the bench workload,
# from one ncu capture; the profile summaries under profiles/ give the command.
# A figure holds only for the code it was taken on (sha256 over the files in
# order, comments and whitespace removed); after any change to that code
# bench.py reports traffic as null.
CSRC = os.path.join(ROOT, "paper_2202_11890_gb300", "csrc")
TRAFFIC = {
    "stage_kernel": {
        "files": ("stage_tile.cuh", "fp64_recip.cuh", "mprk_internal.h", "mprk_kernels.cu"),
        "sha256": "1cc93c59d4076bfba1a35f3537abd9cf162908f0f45fe50a6fd7e47b9f7c8894",
        "bytes_per_step": 1170924544,
    },
    "stage_kernel_mixed": {
        "files": ("stage_tile_mixed.cuh", "mprk_internal.h", "mprk_kernels.cu"),
        "sha256": "70f97e7c7a75239400053bc9d8f307e748da86b7a75da26c9e9f119fa6b11ae3",
        "bytes_per_step": 5149178880,
    },
}


def source_hash(files) -> str:
    """sha256 over the files' code in order, with comments and whitespace
    removed: editing a comment keeps a capture valid, changing code does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f)) as fh:
            code = re.sub(r"/\*.*?\*/", " ", fh.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()


def measured_traffic(kernel: str, launches: int):
    """DRAM bytes per stage launch (mean over one slow step), or None when the
    kernel's sources changed since the capture."""
    t = TRAFFIC[kernel]
    if t["bytes_per_step"] is None or t["sha256"] != source_hash(t["files"]):
        return None
    return t["bytes_per_step"] / launches


def algorithmic_bytes(g: W.Grid, m: int, fp64: bool):
    """HBM bytes one slow step must move, each array element read or written
    once per launch that needs it (stencil halos are L2 hits). Returns
    (bytes of the stage launches, bytes of the step completion)."""
    nx, nS, nB, nF = g.nx, g.nS, g.nB, g.nF
    if fp64:
        d, r, q, a = 32, 32, 32, 32  # stage state read, R_a, q (double), accumulator
    else:
        d, r, q, a = 16, 16, 32, 32  # float shadow, float R_a, double q and accumulator
    tot = 0
    for st in range(2 * m):
        odd = st % 2 == 1
        last = st == 2 * m - 1
        # buffer rows: read the stage state (and R_a on odd stages), write R_a
        # on even stages, read and write the accumulator (write only at stage
        # 1), and at the last stage read q (the mixed mode reads it apart from
        # its float shadow)
        B = d + r + (a if st == 0 else 2 * a) + (q if (last and not fp64) else 0)
        # slow rows: stage 1 reads the state and writes R_a; stage 2 reads both
        # and writes q_{n+1} to the accumulator
        S = (d + r) if st == 0 else ((d + r + a + (0 if fp64 else q)) if st == 1 else 0)
        if fp64:
            F = (d + r + q) if odd else (d + r)       # odd: read q, R_a; write q_next
        else:
            # odd: read d, R_a, q; write q, d (the last stage of an even m
            # leaves the shadow to the step completion)
            F = (d + r + q + q + (0 if (last and m % 2 == 0) else d)) if odd else (d + r)
        tot += nx * (nS * S + nB * B + nF * F)
    if fp64:
        fin = nx * (nS + nB) * 64 + (nx * nF * 64 if m % 2 else 0)
    else:
        fin = nx * (nS + nB) * 80 + nx * nF * (80 if m % 2 else 48)
    return tot, fin


def workload(name: str) -> W.Workload:
    return {"large_2048": W.large_2048, "plain_64": W.plain_64, "mixed_4096": W.mixed_4096}[name]()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device: str) -> float:
    """The largest x over the ranks of the default process group (x itself
    without one): the job's time is its slowest replica's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, ranks: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time."""
    return units_per_rank * ranks / seconds


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


def fp32_accuracy(M, cfg, q0, steps: int) -> dict:
    """The FP32-flux mode against the FP64 path after `steps` slow steps from
    the same state and dt, and the relative change of each fluid's mass over
    the run in both. The FP64 path matches the oracle to 1e-12 per slow step
    (tests/test_gpu_parity.py); the FP32-flux step matches the oracle to
    1e-5 at this size (tests/test_gpu_full_size.py)."""
    import ctypes as C
    c64 = M.mprk_config()
    C.memmove(C.byref(c64), C.byref(cfg), C.sizeof(cfg))
    c64.precision = M.MPRK_FP64
    with M.Instance(cfg, q0) as a:
        c64.dt = a.info()["dt"]
        with M.Instance(c64, q0) as b:
            d0a, d0b = a.diagnostics(), b.diagnostics()
            a.step(steps)
            b.step(steps)
            d1a, d1b = a.diagnostics(), b.diagnostics()
            qa, qb = a.state(), b.state()
    scale = np.abs(qb).max(axis=(1, 2))
    err = np.abs(qa - qb).max(axis=(1, 2)) / np.where(scale > 0, scale, 1.0)
    drift = lambda d0, d1: [float((d1[0] - d0[0]) / d0[0]), float((d1[4] - d0[4]) / d0[4])]
    return {"steps": steps, "against": "FP64 path from the same state and dt",
            "max_rel_err": float(err.max()), "rel_err_rho_rhou_rhow_rhoE": [float(x) for x in err],
            "mass_drift_fluid1_fluid2": {"fp32flux": drift(d0a, d1a), "fp64": drift(d0b, d1b)}}


def roofline_of(fp64: bool, stage_cells: int, stage_ms: float, stage_bytes: float, traffic):
    """Both fractions of the stage kernel: the binding one first (FP64 units
    in the FP64 mode, HBM in the FP32-flux mode), the other beside it."""
    peaks, src = measured_peaks()
    ach_gflops = stage_cells * FLOPS_PER_CELL_STAGE[fp64] / (stage_ms * 1e-3) / 1e9
    ach_gbs = stage_bytes / (stage_ms * 1e-3) / 1e9
    if fp64:
        peak, psrc, probe = fp64_peak()
        return {"bound": "alu", "achieved": ach_gflops, "peak": peak, "unit": "GFLOP/s",
                "frac": ach_gflops / peak, "traffic": traffic, "peak_source": psrc,
                "probe_gflops": probe["gflops"], "frac_of_probe": ach_gflops / probe["gflops"],
                "hbm_achieved_gbs": ach_gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                "hbm_frac": ach_gbs / peaks["hbm_gbs"], "hbm_peak_source": src}
    return {"bound": "hbm", "achieved": ach_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach_gbs / peaks["hbm_gbs"], "traffic": traffic, "peak_source": src,
            "alu_achieved_gflops": ach_gflops, "alu_peak_gflops": FP32_PEAK_GFLOPS,
            "alu_frac": ach_gflops / FP32_PEAK_GFLOPS, "alu_peak_source": "FP32 unit count x max clock (nominal)"}


def measure_single(M, T, wl: W.Workload, steps: int, warmup: int, ws: int = 1, e2e: bool = True,
                   traffic_key: bool = True):
    """One instance of workload wl: K slow steps timed by CUDA events on the
    instance stream (max over ranks), the stage kernel's own time inside the
    step graph, the roofline, clocks and (e2e) the same metric through the C
    ABI with host buffers. Returns (record, instance config, q0, dt)."""
    import torch
    g = wl.grid
    q0 = wl.initial_state()
    cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m)
    cfg.precision = M.MPRK_FP32FLUX if wl.precision == "fp32flux" else M.MPRK_FP64
    fp64 = cfg.precision == M.MPRK_FP64
    inst = M.Instance(cfg, q0)
    info = inst.info()
    cs = info["cell_stages_per_step"]
    stream = info["stream"]
    inst.step(warmup)
    inst.sync()
    sampler = ClockSampler(torch.cuda.current_device())
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with sampler:
        t_ms = T.time_steps(inst.h, stream, steps)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_ms = max_over_ranks(t_ms, "cuda")
    value = replica_value(cs * steps, ws, t_ms * 1e-3)
    # dominant kernel: the stage launches' share of a slow step (event nodes
    # inside a graph of the step, median of 3 steps) times the step time
    ev_ms, stage_cells, share = T.stage_kernel_times(inst.h, stream, reps=3)
    stage_ms = T.kernel_ms_per_step(t_ms / steps, share)
    stage_bytes, fin_bytes = algorithmic_bytes(g, wl.m, fp64)
    kname = "stage_kernel" if fp64 else "stage_kernel_mixed"
    traffic = measured_traffic(kname, 2 * wl.m) if traffic_key else None
    rec = {"value": value, "unit": "cell-stages/s", "steps": steps, "warmup": warmup,
           "ms_per_step": t_ms / steps,
           "dtype": "f64" if fp64 else "f32 flux / f64 accumulate",
           "config": {"workload": wl.name, "nx": g.nx, "nz": g.nz, "rows_S_B_F": [g.nS, g.nB, g.nF],
                      "m": wl.m, "cell_stages_per_step": cs, "dt": info["dt"]},
           "roofline": roofline_of(fp64, stage_cells, stage_ms, stage_bytes, traffic),
           "kernel": {"name": kname, "ms_per_step": stage_ms, "cell_stages_per_step": stage_cells,
                      "launches_per_step": 2 * wl.m, "share_of_step": share, "event_node_ms_per_step": ev_ms,
                      "timed": "share of the stage launches in a graph of one slow step with an event node "
                               "after every launch, times the plain step graph's ms_per_step",
                      "algorithmic_bytes_per_step": stage_bytes,
                      "algorithmic_bytes_per_launch": stage_bytes / (2 * wl.m),
                      "completion_bytes_per_step": fin_bytes},
           "gpu_launches": (2 * wl.m + 1) * steps,
           "clocks": sampler.summary()}
    if e2e:
        # every step uploads its input state from pinned host memory,
        # advances one slow step and downloads the result (mprk_step_io
        # overlaps step j's copies with the neighbouring steps' compute)
        pin_in = torch.from_numpy(q0).pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        e2e_steps = max(3, min(steps, 20))
        M.mprk_step_io(inst.h, [pin_in], [pin_out])  # allocates the staging buffers
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        M.mprk_step_io(inst.h, [pin_in] * e2e_steps, [pin_out] * e2e_steps)
        e2e_s = max_over_ranks(time.perf_counter() - t0, "cuda")
        rec["e2e"] = {"value": replica_value(cs * e2e_steps, ws, e2e_s), "unit": "cell-stages/s",
                      "h2d_bytes_per_step": q0.nbytes, "d2h_bytes_per_step": q0.nbytes, "steps": e2e_steps}
    dt = info["dt"]
    inst.close()
    return rec, cfg, q0, dt


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
    traffic_key = args.workload in ("large_2048", "mixed_4096") and not args.precision
    tiles = tune_tiles(M, wl) if wl.precision == "fp64" and not args.no_tune else None
    rec, cfg, q0, dt = measure_single(M, T, wl, args.steps, args.warmup, ws, True, traffic_key)
    if tiles is not None:
        rec["kernel"]["tile_shapes"] = tiles
    fp64 = cfg.precision == M.MPRK_FP64
    if rank == 0:
        out = {"metric": METRIC, "value": rec["value"], "unit": "cell-stages/s", "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": rec["dtype"], "data": "synthetic",
               "config": {**rec["config"], "parallelism": f"replicas x{ws}",
                          "l2": "working set > L2 (about 4 states of 67 MB); no flush"},
               "roofline": rec["roofline"], "kernel": rec["kernel"], "e2e": rec["e2e"],
               "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"]}
        if not fp64 and not args.no_accuracy:
            out["accuracy"] = mixed_accuracy(M, cfg, q0, wl, dt, args)
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline(wl)
        if ws == 1 and args.workload == "large_2048" and not args.precision and not args.no_sub:
            out["workloads"] = sub_records(args)
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


def tune_tiles(M, wl) -> dict:
    """The library's tile-shape autotuner (mprk_tile_tune) on an instance of
    the workload, before the measured instance is created (it captures its
    step with the tuned shapes; results do not depend on them). Returns the
    shape chosen for each of the workload's stage launches."""
    g = wl.grid
    cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m)
    M.mprk_tune_clear()
    with M.Instance(cfg, wl.initial_state()) as inst:
        M.mprk_tile_tune([inst.h], reps=3)
    out = {}
    for name, rows in (("first_substep_all_rows", g.nz), ("later_substeps_B_F_rows", g.nB + g.nF)):
        sh = M.mprk_tile_lookup(float(g.nx * rows))
        out[name] = {"cells": g.nx * rows, "tile": f"32x{sh['tile_rows']}" if sh else None,
                     "threads_per_cell": sh["threads_per_cell"] if sh else None}
    return out


def mixed_accuracy(M, cfg, q0, wl, dt, args) -> dict:
    """The FP32-flux result's error: against the FP64 path over the whole
    run, and against the oracle at full size over the slow steps of the
    oracle's timed sample (the CPU-baseline leg)."""
    acc = {"fp64_path": fp32_accuracy(M, cfg, q0, wl.steps),
           "tests": ["tests/test_gpu_full_size.py::test_mixed_4096_20_steps_against_oracle (<= 1e-5 after 20 "
                     "slow steps at full size)",
                     "tests/test_gpu_full_size.py::test_mixed_strip_whole_run_against_oracle (<= 1e-5 after the "
                     "500 slow steps on a 64-column strip of the same rows, m and dx)"]}
    if not args.no_cpu_baseline:
        acc["oracle"] = oracle_full_size(M, cfg, q0, wl, dt, args.oracle_steps)
    return acc


def oracle_full_size(M, cfg, q0, wl, dt, steps: int) -> dict:
    """CPU-baseline leg of the FP32-flux workload: the oracle as it stands,
    all host cores, `steps` slow steps of the full-size workload from its
    initial state with the GPU's dt (timed), and the GPU's FP32-flux state
    after the same steps compared with it per component."""
    from oracle import oracle as O
    g = wl.grid
    with M.Instance(cfg, q0) as inst:
        inst.step(steps)
        q_gpu = inst.state()
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    P = O.make_problem(g.nx, g.nS, g.nB, g.nF, wl.m, dt, g.dx, dz1=g.dz1, dz2=g.dz2)
    t0 = time.perf_counter()
    q_or, cnt = O.mprk_step(P, q0, steps)
    el = time.perf_counter() - t0
    cnt *= steps  # the oracle counts one step's RHS evaluations
    scale = np.abs(q_or).max(axis=(1, 2))
    err = np.abs(q_gpu - q_or).max(axis=(1, 2)) / np.where(scale > 0, scale, 1.0)
    return {"steps": steps, "against": "the FP64 CPU oracle from the same state and dt (full size)",
            "max_rel_err": float(err.max()), "rel_err_rho_rhou_rhow_rhoE": [float(x) for x in err],
            "tolerance": 1e-5,
            "cpu_baseline": {"value": cnt / el, "unit": "cell-stages/s", "cores": O.get_threads(),
                             "kind": "oracle",
                             "sample": f"{steps} full-size slow steps of {wl.name} ({cnt} cell-stages, {el:.1f} s)"}}


def measure_batched(M, T, precision: str, steps: int, warmup: int, count: int = 256, tune: bool = False):
    """256 uneven instances (sides log-uniform in [64, 512], m in {2, 4, 8},
    buffer 4-16 rows; FP64 or FP32 flux): one graph launch per slow step
    (mprk_step_batch; in the form the tuning table picks: the persistent
    kernel, or for FP32 flux the per-stage launches) against the same
    instances stepped one after another with mprk_step on the same stream,
    and the two paths' results from the same start compared bitwise on 8
    instances. FP32 flux adds one 4096 x 2048 instance stepped both ways."""
    import torch
    wls = W.batched_256(count=count)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    insts, q0s = [], []
    for wl in wls:
        g = wl.grid
        cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m)
        if precision == "fp32flux":
            cfg.precision = M.MPRK_FP32FLUX
        q0 = wl.initial_state()
        q0s.append(q0)
        insts.append(M.Instance(cfg, q0, stream=sp))
    hs = [i.h for i in insts]
    cs = sum(i.info()["cell_stages_per_step"] for i in insts)
    cells = sum(wl.grid.nx * wl.grid.nz for wl in wls)

    def plain(n):
        for _ in range(n):
            for h in hs:
                M.mprk_step(h, 1)

    def batched(n):
        M.mprk_step_batch(hs, n)

    # warm-up both paths (graphs, plan), then the launch the tuning table
    # gives (defaults when it has no entry; tune=True fills it first)
    plain(warmup)
    batched(warmup)
    torch.cuda.synchronize()
    tuned = None
    if tune:
        t_default = T.time_region(sp, lambda: batched(steps))
        tuned = M.mprk_batch_tune(hs, reps=3)
        tuned["default_launch_cell_stages_per_s"] = cs * steps / (t_default * 1e-3)
        batched(warmup)
        torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    with sampler:
        t_batch = T.time_region(sp, lambda: batched(steps))
        t_plain = T.time_region(sp, lambda: plain(steps))
    # equal accuracy: same start, same steps, both paths, bitwise
    same = True
    for i, q0 in zip(insts[:8], q0s[:8]):
        i.set_state(q0)
    M.mprk_step_batch(hs[:8], 2)
    out_b = [i.state() for i in insts[:8]]
    for i, q0 in zip(insts[:8], q0s[:8]):
        i.set_state(q0)
        i.step(2)
    maxrel = 0.0
    for i, ob in zip(insts[:8], out_b):
        op = i.state()
        same = same and bool(np.array_equal(op, ob))
        scale = np.abs(ob).max(axis=(1, 2))
        maxrel = max(maxrel, float((np.abs(op - ob).max(axis=(1, 2)) / scale).max()))
    value = cs * steps / (t_batch * 1e-3)
    plain_value = cs * steps / (t_plain * 1e-3)
    # both fractions of the whole batched launch (stage tiles and
    # completions), from the algorithmic flops and bytes of every instance
    fp64 = precision != "fp32flux"
    peaks, src = measured_peaks()
    nbytes = sum(sum(algorithmic_bytes(wl.grid, wl.m, fp64)) for wl in wls)
    gbs = nbytes * steps / (t_batch * 1e-3) / 1e9
    gflops = cs * FLOPS_PER_CELL_STAGE[fp64] * steps / (t_batch * 1e-3) / 1e9
    if fp64:
        peak, psrc, probe = fp64_peak()
        roof = {"bound": "alu", "achieved": gflops, "peak": peak, "unit": "GFLOP/s", "frac": gflops / peak,
                "traffic": None, "peak_source": psrc, "frac_of_probe": gflops / probe["gflops"], "hbm_achieved_gbs": gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                "hbm_frac": gbs / peaks["hbm_gbs"], "hbm_peak_source": src, "algorithmic_bytes_per_step": nbytes}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                "algorithmic_bytes_per_step": nbytes, "alu_achieved_gflops": gflops,
                "alu_peak_gflops": FP32_PEAK_GFLOPS, "alu_frac": gflops / FP32_PEAK_GFLOPS,
                "alu_peak_source": "FP32 unit count x max clock (nominal)"}
    for i in insts:
        i.close()
    launch = M.mprk_tune_lookup(0 if fp64 else 1, cells / len(wls))
    if launch["tiles_per_item"] == 0:
        # per-stage form: each instance group launches its stages and its
        # completions (at most as many stages as the largest m gives)
        groups = min(launch["ctas_per_sm"] or 2, len(wls))
        kernels = groups * (2 * max(wl.m for wl in wls) + 1)
    else:
        kernels = 1
    rec = {"value": value, "unit": "cell-stages/s", "steps": steps, "warmup": warmup,
           "ms_per_step": t_batch / steps,
           "dtype": "f32 flux / f64 accumulate" if precision == "fp32flux" else "f64",
           "config": {"workload": f"batched_{len(wls)}_uneven_{precision}", "instances": len(wls), "cells": cells,
                      "cell_stages_per_step": cs},
           "batched_vs_plain": {"batched": value, "plain_sequential": plain_value, "speedup": value / plain_value,
                                "bitwise_equal": same, "max_rel_diff": maxrel,
                                "plain_ms_per_step": t_plain / steps,
                                "plain": "each instance's own captured step graph (mprk_step), one after another"},
           "launch": launch,
           "roofline": roof, "gpu_launches": steps * kernels,
           "gpu_launches_note": "kernels per slow step x steps (upper bound for the per-stage form)",
           "clocks": sampler.summary()}
    if tuned is not None:
        rec["tuned_launch"] = tuned
    if not fp64:
        rec["one_large_instance"] = one_large_batched(M, T, steps, warmup)
    return rec


def one_large_batched(M, T, steps: int, warmup: int) -> dict:
    """One 4096 x 2048 FP32-flux instance (the mixed workload's grid, m = 8):
    slow steps through mprk_step_batch (a batch of one) against mprk_step,
    and the two results from the same start after one step compared."""
    import torch
    wl = W.mixed_4096()
    g = wl.grid
    cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m)
    cfg.precision = M.MPRK_FP32FLUX
    q0 = wl.initial_state()
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    with M.Instance(cfg, q0, stream=sp) as inst:
        cs = inst.info()["cell_stages_per_step"]
        M.mprk_step_batch([inst.h], warmup)
        inst.step(warmup)
        t_b = T.time_region(sp, lambda: M.mprk_step_batch([inst.h], steps))
        t_s = T.time_region(sp, lambda: inst.step(steps))
        inst.set_state(q0)
        M.mprk_step_batch([inst.h], 1)
        qb = inst.state()
        inst.set_state(q0)
        inst.step(1)
        qs = inst.state()
    scale = np.abs(qs).max(axis=(1, 2))
    rel = float((np.abs(qb - qs).max(axis=(1, 2)) / scale).max())
    return {"workload": "mixed_4096x2048_m8_fp32flux", "steps": steps,
            "batched": cs * steps / (t_b * 1e-3), "single_instance": cs * steps / (t_s * 1e-3),
            "batched_over_single": t_s / t_b, "bitwise_equal": bool(np.array_equal(qb, qs)),
            "max_rel_diff_one_step": rel, "launch": M.mprk_tune_lookup(1, g.nx * g.nz)}


def run_batched(args):
    """The batched workload on its own line (--workload batched_256)."""
    import torch
    from paper_2202_11890_gb300 import build as B
    from paper_2202_11890_gb300 import mprk as M
    from paper_2202_11890_gb300 import timing as T

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    M.mprk_tune_clear()
    rec = measure_batched(M, T, args.precision or "fp64", args.steps, args.warmup, args.batch_count, tune=True)
    out = {"metric": METRIC, "value": rec["value"], "unit": "cell-stages/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
           "config": {**rec["config"], "parallelism": "replicas x1"}}
    out.update({k: v for k, v in rec.items() if k not in out})
    print(json.dumps(out))


def measure_served(M, rate: float, n_warm: int, n_meas: int, budget_gb: float, slots: int,
                   sequential: bool = True, solo_cells: int = 0):
    """Poisson arrivals (mean `rate` requests/s) of FP32-flux solves with
    sides log-uniform in [32, 1024], m in {2, 4, 8}, buffer 4-16 rows and slow
    steps log-uniform in [10, 1000], admitted under an HBM budget. Reports
    the aggregate cell-stage rate and p50/p99 latency (finish - submit on the
    server's clock) of the requests after the warm-up ones; with sequential,
    the same measured requests solved one after another through mprk_create,
    mprk_step and mprk_get_state, each result checked against the served
    one."""
    import torch
    arrivals, wls = W.served_stream(n_warm + n_meas, rate_hz=rate)
    reqs = []
    for wl in wls:
        g = wl.grid
        cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m)
        cfg.precision = M.MPRK_FP32FLUX
        reqs.append((cfg, wl.initial_state(), wl.steps, wl.cell_stages_per_step() * wl.steps,
                     sum(algorithmic_bytes(g, wl.m, False)) * wl.steps))
    srv = M.mprk_server_create(hbm_budget_bytes=int(budget_gb * 1e9), max_slots=slots, solo_cells=solo_cells)
    sampler = ClockSampler(torch.cuda.current_device())
    tickets = {}
    done = {}
    results = {}
    t0 = time.perf_counter()
    nxt = 0
    # the server's count of cell-stages done, sampled when the first and the
    # last measured request are submitted: the work rate over the arrival
    # window of the measured requests, without the drain after it
    window = {}
    with sampler:
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and arrivals[nxt] <= now:
                cfg, q, n, _, _ = reqs[nxt]
                if nxt in (n_warm, len(reqs) - 1):
                    window[nxt] = (time.perf_counter(), M.mprk_server_stats(srv)[1])
                tickets[M.mprk_submit(srv, cfg, q, n)] = nxt
                nxt += 1
            for t, j in list(tickets.items()):
                st, err, stats = M.mprk_poll(srv, t)
                if st == M.MPRK_REQ_DONE:
                    res = np.empty(reqs[j][1].shape)
                    M.mprk_poll(srv, t, res)  # read and release
                    done[j] = (err, stats)
                    if sequential and j >= n_warm:
                        results[j] = res
                    del tickets[t]
            time.sleep(0.0005)
    wall = time.perf_counter() - t0
    sstats = M.mprk_server_stats(srv)
    sprof = M.mprk_server_profile(srv)
    M.mprk_server_destroy(srv)
    meas = [done[j] for j in range(n_warm, len(reqs))]
    lat = np.array([s["t_finish"] - s["t_submit"] for _, s in meas])
    errors = sum(1 for e, _ in meas if e)
    t_first = min(s["t_submit"] for _, s in meas)
    t_last = max(s["t_finish"] for _, s in meas)
    work = sum(reqs[j][3] for j in range(n_warm, len(reqs)))
    value = work / (t_last - t_first)
    offered = sum(r[3] for r in reqs[n_warm:]) / (arrivals[-1] - arrivals[n_warm])
    (w0, c0), (w1, c1) = window[n_warm], window[len(reqs) - 1]
    window_rate = (c1 - c0) / max(w1 - w0, 1e-9)
    peaks, src = measured_peaks()
    gbs = sum(reqs[j][4] for j in range(n_warm, len(reqs))) / (t_last - t_first) / 1e9
    rec = {"value": value, "unit": "cell-stages/s", "requests": n_meas, "warmup_requests": n_warm,
           "dtype": "f32 flux / f64 accumulate",
           "config": {"workload": "served_poisson_fp32flux", "rate_hz": rate, "requests": n_meas,
                      "budget_gb": budget_gb, "max_slots": slots,
                      "solo_cells": solo_cells if solo_cells else
                      f"default: {M.MPRK_SOLO_CELLS_DEFAULT} for FP64 requests, FP32-flux requests all batched"},
           "served": {"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                      "mean_latency_s": float(lat.mean()), "errors": errors,
                      "offered_cell_stages_per_s": offered, "achieved_over_offered": value / offered,
                      "arrival_window": {
                          "cell_stages_per_s": window_rate, "over_offered": window_rate / offered,
                          "seconds": w1 - w0,
                          "how": "cell-stages of the server's batched steps (all resident requests; "
                                 "counted as each step is enqueued, at most two steps ahead of the GPU) "
                                 "between the first and the last measured submission, over that time; "
                                 "value above divides the measured requests' work by first submit to "
                                 "last finish, which includes the drain of the longest requests"},
                      "batched_steps": int(sstats[2]), "wall_s": wall,
                      "loop": {**sprof, "gpu_busy_over_step_span": sprof["gpu_busy_s"] / max(sprof["step_span_s"], 1e-9)}},
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                        "note": "algorithmic bytes of the measured requests over their first submit to last finish"},
           "gpu_launches": int(sstats[2]), "clocks": sampler.summary()}
    if sequential:
        # the same measured requests without the server: each alone, one
        # after another, through the plain C ABI calls
        maxrel = 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(n_warm, len(reqs)):
            cfg, q, n, _, _ = reqs[j]
            with M.Instance(cfg, q) as inst:
                inst.step(n)
                out = inst.state()
            r = results[j]
            scale = np.abs(out).max(axis=(1, 2))
            maxrel = max(maxrel, float((np.abs(out - r).max(axis=(1, 2)) / scale).max()))
        seq_s = time.perf_counter() - t0
        rec["sequential"] = {"value": work / seq_s, "wall_s": seq_s,
                             "served_over_sequential": value / (work / seq_s),
                             "max_rel_diff_vs_served": maxrel, "tolerance": 1e-5,
                             "how": "each measured request alone: mprk_create (upload, graph capture), "
                                    "mprk_step(n), mprk_get_state, mprk_destroy, one after another"}
    return rec


def run_served(args):
    """The served workload on its own line (--workload served)."""
    import torch
    from paper_2202_11890_gb300 import build as B
    from paper_2202_11890_gb300 import mprk as M

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    rec = measure_served(M, args.rate, args.served_warmup, args.served_requests, args.budget_gb, args.slots,
                         sequential=args.served_sequential, solo_cells=args.served_solo_cells)
    out = {"metric": METRIC, "value": rec["value"], "unit": "cell-stages/s", "n_gpus": ws,
           "steps": args.served_requests, "warmup": args.served_warmup, "ms_per_step": None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"],
           "data": "synthetic", "config": {**rec["config"], "parallelism": "replicas x1"}}
    out.update({k: v for k, v in rec.items() if k not in out})
    print(json.dumps(out))


def sub_records(args) -> dict:
    """The metric's other parts on the same line as the headline: the
    FP32-flux workload (HBM roofline, accuracy), the 256-instance batch in
    both precisions (batched vs plain), and the served Poisson stream
    (p50/p99 latency, served vs sequential). Each carries its own step
    counts and clocks."""
    from paper_2202_11890_gb300 import mprk as M
    from paper_2202_11890_gb300 import timing as T
    out = {}
    wl = W.mixed_4096()
    rec, cfg, q0, dt = measure_single(M, T, wl, args.sub_steps, args.warmup, 1, True, True)
    rec["accuracy"] = mixed_accuracy(M, cfg, q0, wl, dt, args)
    out["mixed_4096"] = rec
    for prec in ("fp64", "fp32flux"):
        # the launch choices (tiles per item, CTAs per SM, FP64 tile shape)
        # tuned on the instances first, the default launch timed beside
        out[f"batched_256_{prec}"] = measure_batched(M, T, prec, args.sub_steps, args.warmup,
                                                     tune=not args.no_tune)
    out["served"] = measure_served(M, args.rate, args.sub_served_warmup, args.sub_served_requests, args.budget_gb,
                                   args.slots, sequential=True)
    # the same stream's distribution at a lower arrival rate, below the
    # GPU's saturation, for the latency of an unsaturated server
    out["served_below_saturation"] = measure_served(M, args.sub_served_rate_low, args.sub_served_warmup,
                                                    args.sub_served_requests, args.budget_gb, args.slots,
                                                    sequential=False)
    return out


def run_speedup(args):
    """MPRK2 against its single-rate base RK2 on the GPU (Sec. 4, Eq. speedup;
    the shape of Table 2): 100 rows, 6 buffer rows, N_S/N in {4, 14, ..., 84}
    per 100, m in {2, 4, 8}, FP64, nx columns. The single-rate run takes m
    RK2 steps of dt/m over the whole grid per slow step. Reports the measured
    wall-clock ratio next to the theoretical spd."""
    import torch
    from paper_2202_11890_gb300 import build as B
    from paper_2202_11890_gb300 import mprk as M
    from paper_2202_11890_gb300 import timing as T

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    nx = args.speedup_nx
    rows = []
    for ns in range(4, 85, 10):
        nB, nF = 6, 100 - ns - 6
        g = W.Grid(nx, ns, nB, nF, dx=10.0 / nx, dz1=10.0 / 100, dz2=10.0 / 100)
        q0 = W.gaussian_bumps(g, SEED_SPEEDUP)
        for m in (2, 4, 8):
            times = {}
            for scheme in (M.MPRK_SCHEME_MPRK2, M.MPRK_SCHEME_SR_RK2):
                cfg = M.mprk_config_default(nx, ns, nB, nF, m, dx=g.dx, dz1=g.dz1, dz2=g.dz2)
                cfg.scheme = scheme
                cfg.dt = 1e-3
                with M.Instance(cfg, q0) as inst:
                    inst.step(args.warmup)
                    inst.sync()
                    times[scheme] = T.time_steps(inst.h, inst.info()["stream"], args.steps) / args.steps
            spd = 1.0 / (1.0 + (1.0 / m - 1.0) * ns / 100.0)
            rows.append({"NS_over_N": ns / 100, "m": m, "ms_mprk2": times[M.MPRK_SCHEME_MPRK2],
                         "ms_rk2": times[M.MPRK_SCHEME_SR_RK2],
                         "wcr": times[M.MPRK_SCHEME_SR_RK2] / times[M.MPRK_SCHEME_MPRK2], "spd": spd})
    out = {"metric": "wall-clock ratio RK2/MPRK2 (Table 2 shape)", "value": rows[-1]["wcr"], "unit": "ratio",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "speedup_sweep", "nx": nx, "rows": 100, "buffer_rows": 6},
           "table": rows}
    print(json.dumps(out))


SEED_SPEEDUP = W.SEED0 + 9

# Algorithmic floating-point operations per cell-stage of the 3-D stage
# (yface3 + stage3), counted from their formulas like the 2-D figure:
# 176 per face (Lax–Friedrichs flux of five components 110, viscous flux
# with the full stress tensor 41, reconstruction 20, F* assembly 5) times
# 3.16 faces per cell (x 33/32, z 9/8, y 1), plus ring primitives of both
# kernels and the y derivatives 91, slopes and tangential derivatives 70,
# divergence and source 32, stage combination 10.
FLOPS_PER_CELL_STAGE_3D = 759.0


def algorithmic_bytes3(g, m: int) -> tuple[int, int]:
    """HBM bytes one 3-D slow step must move, like algorithmic_bytes with
    five doubles per state (40 B), plus the y-face buffer written once and
    read once per cell-stage (80 B)."""
    cols = g.nx * g.ny
    s = 40
    tot = 0
    for st in range(2 * m):
        odd = st % 2 == 1
        B = s + s + (s if st == 0 else 2 * s)
        S = (s + s) if st == 0 else ((s + s + s) if st == 1 else 0)
        F = (s + s + s) if odd else (s + s)
        rows = g.nS * (1 if st < 2 else 0) + g.nB + g.nF
        tot += cols * (g.nS * S + g.nB * B + g.nF * F) + cols * rows * 80
    fin = cols * (g.nS + g.nB) * 80 + (cols * g.nF * 80 if m % 2 else 0)
    return tot, fin


def run_cube(args):
    """The 3-D model on one GPU: `cube_512` (512 x 64 x 200 cells, m = 4,
    FP64). Reports the FP64-ALU roofline of the stage launches, e2e through
    the C ABI with host buffers, and the 3-D oracle on a strip of columns."""
    import torch
    from paper_2202_11890_gb300 import build as B
    from paper_2202_11890_gb300 import mprk as M
    from paper_2202_11890_gb300 import timing as T

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    wl = W.cube_512()
    g = wl.grid
    q0 = wl.initial_state()
    cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m, dx=g.dx, dz1=g.dz1, dz2=g.dz2)
    cfg.ny, cfg.dy = g.ny, g.dy
    steps = args.steps if args.steps != 200 else wl.steps
    with M.Instance(cfg, q0) as inst:
        info = inst.info()
        cs = info["cell_stages_per_step"]
        inst.step(args.warmup)
        inst.sync()
        sampler = ClockSampler(torch.cuda.current_device())
        torch.cuda.synchronize()
        with sampler:
            t_ms = T.time_steps(inst.h, info["stream"], steps)
        torch.cuda.synchronize()
        _, stage_cells, share = T.stage_kernel_times(inst.h, info["stream"], reps=3)
        stage_ms = T.kernel_ms_per_step(t_ms / steps, share)
        pin_in = torch.from_numpy(q0).pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        e2e_steps = 3
        M.mprk_step_io(inst.h, [pin_in], [pin_out])  # allocates the staging buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.mprk_step_io(inst.h, [pin_in] * e2e_steps, [pin_out] * e2e_steps)
        e2e_s = time.perf_counter() - t0
    value = cs * steps / (t_ms * 1e-3)
    ach = stage_cells * FLOPS_PER_CELL_STAGE_3D / (stage_ms * 1e-3) / 1e9
    stage_bytes, fin_bytes = algorithmic_bytes3(g, wl.m)
    peaks, src = measured_peaks()
    out = {"metric": METRIC, "value": value, "unit": "cell-stages/s", "n_gpus": ws, "steps": steps,
           "warmup": args.warmup, "ms_per_step": t_ms / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "nx": g.nx, "ny": g.ny, "rows_S_B_F": [g.nS, g.nB, g.nF], "m": wl.m,
                      "cell_stages_per_step": cs, "parallelism": f"replicas x{ws}",
                      "l2": "working set > L2 (a state is 262 MB); no flush"},
           "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak()[0], "unit": "GFLOP/s",
                        "frac": ach / fp64_peak()[0], "traffic": None, "peak_source": fp64_peak()[1],
                        "frac_of_probe": ach / fp64_peak()[2]["gflops"],
                        "hbm_achieved_gbs": stage_bytes / (stage_ms * 1e-3) / 1e9,
                        "hbm_peak_gbs": peaks["hbm_gbs"],
                        "hbm_frac": stage_bytes / (stage_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                        "hbm_peak_source": src},
           "kernel": {"name": "yface3_kernel + stage3_kernel", "ms_per_step": stage_ms,
                      "cell_stages_per_step": stage_cells, "launches_per_step": 4 * wl.m,
                      "algorithmic_bytes_per_step": stage_bytes, "completion_bytes_per_step": fin_bytes},
           "e2e": {"value": cs * e2e_steps / e2e_s, "unit": "cell-stages/s", "h2d_bytes_per_step": q0.nbytes,
                   "d2h_bytes_per_step": q0.nbytes, "steps": e2e_steps},
           "gpu_launches": (4 * wl.m + 1) * steps, "clocks": sampler.summary()}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline3(wl)
    print(json.dumps(out))


def cpu_baseline3(wl, cols=(16, 8), budget_s: float = 10.0, max_steps: int = 200):
    """The 3-D oracle, all host cores, on slow steps of a 16 x 8 column strip
    of the workload's rows."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    g = wl.grid
    sg = W.Grid3(cols[0], cols[1], g.nS, g.nB, g.nF, dx=g.dx, dy=g.dy, dz1=g.dz1, dz2=g.dz2)
    q = W.gaussian_bumps3(sg, wl.seed)
    P = O.make_problem3(sg.nx, sg.ny, sg.nS, sg.nB, sg.nF, wl.m, 0.0, sg.dx, dy=sg.dy, dz1=sg.dz1, dz2=sg.dz2)
    P.dt = O.stable_dt3(P, q, 0.4)
    per_step = sg.nx * sg.ny * (2 * sg.nS + 2 * wl.m * (sg.nB + sg.nF))
    n, t0 = 0, time.perf_counter()
    while n < max_steps and time.perf_counter() - t0 < budget_s:
        q = O.mprk_step3(P, q)
        n += 1
    el = time.perf_counter() - t0
    return {"value": per_step * n / el, "unit": "cell-stages/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} slow steps of the {wl.name} rows on a {cols[0]}x{cols[1]}-column strip "
                      f"({per_step * n} cell-stages, {el:.1f} s)"}


def run_convection(args):
    """Table 6's thermal convection (Sec. 5.2, second set-up) on the GPU:
    walls on all boundaries, 100 x (100 + 200) cells, MPRK2 with m = 4.
    Throughput of the dt = 0.025 run to t = 2.5 (100 slow steps) in FP64 and
    in the FP32-flux mode, and the temporal-convergence study: L2 errors of
    rho, momentum and rho E at t = 2.5 for dt = 0.025 {1, 1/2, 1/4, 1/8}
    against a single-rate RK2 run on the GPU with dt = 0.003125/64 (the
    paper's reference is RK45 with dt = 0.00125; the oracle check of the same
    study is tests/test_gpu_xwall.py)."""
    import torch
    from paper_2202_11890_gb300 import build as B
    from paper_2202_11890_gb300 import mprk as M
    from paper_2202_11890_gb300 import timing as T

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    wl = W.convection_100()
    g = wl.grid
    q0 = wl.initial_state()
    t_end = 2.5

    def config(dt, m=wl.m, scheme=M.MPRK_SCHEME_MPRK2, precision=M.MPRK_FP64):
        cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, m, dx=g.dx, dz1=g.dz1, dz2=g.dz2)
        cfg.dt, cfg.scheme, cfg.precision, cfg.x_walls = dt, scheme, precision, M.MPRK_X_WALLS
        return cfg

    # throughput of the dt = 0.025 run, FP64 and FP32 flux
    rates = {}
    for name, prec in (("fp64", M.MPRK_FP64), ("fp32flux", M.MPRK_FP32FLUX)):
        with M.Instance(config(0.025, precision=prec), q0) as inst:
            cs = inst.info()["cell_stages_per_step"]
            inst.step(args.warmup)
            inst.sync()
            sampler = ClockSampler(torch.cuda.current_device())
            with sampler:
                t_ms = T.time_steps(inst.h, inst.info()["stream"], wl.steps)
            rates[name] = {"value": cs * wl.steps / (t_ms * 1e-3), "ms_per_step": t_ms / wl.steps,
                           "clocks": sampler.summary()}

    # reference: single-rate RK2 with a tiny step (fast-band Courant ~0.01)
    ref_dt = 0.003125 / 64
    with M.Instance(config(ref_dt, m=1, scheme=M.MPRK_SCHEME_SR_RK2), q0) as inst:
        inst.step(int(round(t_end / ref_dt)))
        ref = inst.state()
    cell = g.dx * np.concatenate([np.full(g.n1, g.dz1), np.full(g.nF, g.dz2)])[:, None]

    def l2(a):
        return float(np.sqrt((a * a * cell).sum()))

    dts, errs = [0.025, 0.0125, 0.00625, 0.003125], []
    for dt in dts:
        with M.Instance(config(dt), q0) as inst:
            inst.step(int(round(t_end / dt)))
            d = inst.state() - ref
        errs.append([l2(d[0]), l2(np.stack([d[1], d[2]])), l2(d[3])])
    e = np.array(errs)
    orders = np.log2(e[:-1] / e[1:]).tolist()
    out = {"metric": METRIC, "value": rates["fp64"]["value"], "unit": "cell-stages/s", "n_gpus": 1,
           "steps": wl.steps, "warmup": args.warmup, "ms_per_step": rates["fp64"]["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": wl.name, "nx": g.nx, "rows_S_B_F": [g.nS, g.nB, g.nF], "m": wl.m,
                      "dt": 0.025, "x_walls": True, "dz1": g.dz1, "dz2": g.dz2},
           "fp32flux": rates["fp32flux"], "clocks": rates["fp64"]["clocks"],
           "convergence": {"t": t_end, "dt": dts, "l2_rho_momentum_energy": errs, "orders": orders,
                           "reference": f"SR-RK2 on the GPU, dt = {ref_dt}",
                           "paper_orders": [[2.04, 2.04, 2.04], [2.00, 2.00, 2.00], [2.00, 2.00, 2.00]]},
           "gpu_launches": (2 * wl.m + 1) * wl.steps}
    print(json.dumps(out))


def run_base(args):
    """MPRK with the classical RK4 base (Sec. 3 remark) on the GPU. Throughput
    of the 2048x1024, m = 8, FP64 workload with the RK4 base (4m stages per
    slow step), and the accuracy experiment the remark calls for: on the
    thermal convection set-up (walls on all sides, m = 4, to t = 2.5), the L2
    errors of rho, momentum and rho E for the RK2, RK3 and RK4 bases at dt =
    0.025 {1, 1/2, 1/4, 1/8} against single-rate RK4 with dt = 0.003125/16,
    and their observed orders (the coupling keeps every base at second order
    or below)."""
    import torch
    from paper_2202_11890_gb300 import build as B
    from paper_2202_11890_gb300 import mprk as M
    from paper_2202_11890_gb300 import timing as T

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    bases = {"rk2": M.MPRK_BASE_RK2, "rk3": M.MPRK_BASE_RK3, "rk4": M.MPRK_BASE_RK4}
    stages = {"rk2": 2, "rk3": 3, "rk4": 4}

    # throughput: the large FP64 workload with the RK4 base
    wl = W.large_2048()
    g = wl.grid
    q0 = wl.initial_state()
    cfg = M.mprk_config_default(g.nx, g.nS, g.nB, g.nF, wl.m)
    cfg.base = M.MPRK_BASE_RK4
    steps = min(args.steps, 60)
    with M.Instance(cfg, q0) as inst:
        cs = inst.info()["cell_stages_per_step"]
        stream = inst.info()["stream"]
        inst.step(args.warmup)
        inst.sync()
        sampler = ClockSampler(torch.cuda.current_device())
        torch.cuda.synchronize()
        with sampler:
            t_ms = T.time_steps(inst.h, stream, steps)
        torch.cuda.synchronize()
        _, stage_cells, share = T.stage_kernel_times(inst.h, stream, reps=3)
        stage_ms = T.kernel_ms_per_step(t_ms / steps, share)
    value = cs * steps / (t_ms * 1e-3)
    ach = stage_cells * FLOPS_PER_CELL_STAGE[True] / (stage_ms * 1e-3) / 1e9

    # accuracy: the thermal convection with each base
    cw = W.convection_100()
    cg = cw.grid
    cq = cw.initial_state()
    t_end = 2.5

    def config(dt, base, m=cw.m, scheme=M.MPRK_SCHEME_MPRK2):
        c = M.mprk_config_default(cg.nx, cg.nS, cg.nB, cg.nF, m, dx=cg.dx, dz1=cg.dz1, dz2=cg.dz2)
        c.dt, c.scheme, c.x_walls, c.base = dt, scheme, M.MPRK_X_WALLS, bases[base]
        return c

    ref_dt = 0.003125 / 16
    with M.Instance(config(ref_dt, "rk4", m=1, scheme=M.MPRK_SCHEME_SR_RK2), cq) as inst:
        inst.step(int(round(t_end / ref_dt)))
        ref = inst.state()
    cell = cg.dx * np.concatenate([np.full(cg.n1, cg.dz1), np.full(cg.nF, cg.dz2)])[:, None]

    def l2(a):
        return float(np.sqrt((a * a * cell).sum()))

    dts = [0.025, 0.0125, 0.00625, 0.003125]
    study = {}
    for base in bases:
        errs = []
        for dt in dts:
            with M.Instance(config(dt, base), cq) as inst:
                inst.step(int(round(t_end / dt)))
                d = inst.state() - ref
            errs.append([l2(d[0]), l2(np.stack([d[1], d[2]])), l2(d[3])])
        e = np.array(errs)
        study[base] = {"l2_rho_momentum_energy": errs, "orders": np.log2(e[:-1] / e[1:]).tolist()}

    out = {"metric": METRIC, "value": value, "unit": "cell-stages/s", "n_gpus": 1, "steps": steps,
           "warmup": args.warmup, "ms_per_step": t_ms / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name.replace("_m8", "_m8_rk4base"), "nx": g.nx,
                      "rows_S_B_F": [g.nS, g.nB, g.nF], "m": wl.m, "base": "rk4",
                      "cell_stages_per_step": cs, "l2": "working set > L2; no flush"},
           "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak()[0], "unit": "GFLOP/s",
                        "frac": ach / fp64_peak()[0], "traffic": None, "peak_source": fp64_peak()[1],
                        "frac_of_probe": ach / fp64_peak()[2]["gflops"],
                        "flops": "the Heun stage's count; the RK4 stage values and weights add < 2 %"},
           "kernel": {"name": "stage_kernel<GEN>", "ms_per_step": stage_ms,
                      "cell_stages_per_step": stage_cells, "launches_per_step": 4 * wl.m},
           "clocks": sampler.summary(),
           "accuracy": {"setup": cw.name, "t": t_end, "dt": dts, "m": cw.m,
                        "reference": f"single-rate RK4 on the GPU, dt = {ref_dt}", "bases": study},
           "gpu_launches": (4 * wl.m + 1) * steps}
    print(json.dumps(out))


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
    out = {"value": total / dt, "unit": "cell-stages/s", "cores": O.get_threads(), "kind": "oracle",
           "sample": f"{steps} slow steps of the {wl.name} rows on a {cols}-column strip "
                     f"({total} cell-stages, {dt:.1f} s)"}
    # the same oracle on one thread, on a narrower strip
    O.set_threads(1)
    s1 = oracle_sample(wl, 64)
    g1 = s1.grid
    q1 = s1.initial_state()
    P1 = O.make_problem(g1.nx, g1.nS, g1.nB, g1.nF, s1.m, P.dt, g1.dx, dz1=g1.dz1, dz2=g1.dz2)
    t0 = time.perf_counter()
    total1, steps1 = 0, 0
    while steps1 < max_steps and (time.perf_counter() - t0) < budget_s / 2:
        q1, cnt = O.mprk_step(P1, q1, 1)
        total1 += cnt
        steps1 += 1
    dt1 = time.perf_counter() - t0
    O.set_threads(cores)
    out["single_thread"] = {"value": total1 / dt1, "unit": "cell-stages/s", "cores": 1,
                            "sample": f"{steps1} slow steps on a 64-column strip ({total1} cell-stages, "
                                      f"{dt1:.1f} s)"}
    return out


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
    ap.add_argument("--workload", default="large_2048",
                    choices=["large_2048", "plain_64", "mixed_4096", "batched_256", "served", "speedup",
                             "convection", "cube", "base_rk4"])
    ap.add_argument("--speedup-nx", type=int, default=2048)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--served-warmup", type=int, default=200)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--slots", type=int, default=4096)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--precision", default="", choices=["", "fp64", "fp32flux"])
    ap.add_argument("--ref-cols", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="headline line only, without the other workloads")
    ap.add_argument("--no-tune", action="store_true", help="default launch choices, no autotuning")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP32-flux accuracy runs (for profiling commands)")
    ap.add_argument("--sub-steps", type=int, default=20, help="slow steps timed per sub-record")
    ap.add_argument("--sub-served-requests", type=int, default=500)
    ap.add_argument("--sub-served-warmup", type=int, default=100)
    ap.add_argument("--sub-served-rate-low", type=float, default=120.0)
    ap.add_argument("--served-sequential", action="store_true")
    ap.add_argument("--served-solo-cells", type=int, default=0,
                    help="server's solo_cells: 0 the library default, -1 every instance batched")
    ap.add_argument("--oracle-steps", type=int, default=2,
                    help="full-size oracle slow steps of the FP32-flux CPU-baseline leg")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, _ = dist_env()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload not in ("large_2048", "plain_64", "mixed_4096") and rank != 0:
        return  # the other workloads are single-GPU studies: rank 0 runs them alone
    elif args.workload == "batched_256":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "convection":
        run_convection(args)
    elif args.workload == "cube":
        run_cube(args)
    elif args.workload == "base_rk4":
        run_base(args)
    elif args.workload == "speedup":
        run_speedup(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
