"""Benchmark: MLUPS and time per Biot step of the coupled LBM on one GB300.

Workload (one step = one physical time step of Alg. 5: explicit force, N_E = 3
multigrid V-cycles of the pseudo-time MRT elasticity LBM with K = 4 smoothing
sweeps per level, then the SRT pressure step): Terzaghi consolidation on
4097x4097 nodes (4096x4096 cells), FP32 populations with FP64 residual norms,
coarsest level and coupling accumulators, 10 multigrid levels.  Synthetic
input (the problem is fully defined by its parameters); all state stays
resident in HBM and is larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own independent instance (instances do not
exchange data, so the run is weak-scaled replicas); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & time per Biot step at stated error vs FP64 oracle"
WORKLOAD = "terzaghi_4097x4097_fp32"
PROFILE = os.path.join(ROOT, "profiles", "sweep_fp32_terzaghi_4097.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2409_11382_gb300", "csrc", "sweep_mom.cuh")


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_sha():
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def profiled_traffic_per_cell():
    """DRAM bytes per cell of one finest-level sweep from the committed ncu summary,
    or None if the kernel source changed since the counters were taken."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    m = re.search(r"traffic_bytes_per_cell:\s*([0-9.]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_sha():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = []
        for line in open(self.out.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample_step():
    """The oracle (single-threaded FP64 C) on one physical step of the same workload,
    restricted to a 512-cell-wide strip: the problem does not depend on x, so every
    cell does the same work as in the full grid.  Returns (seconds, cells)."""
    from oracle import oracle as O
    from paper_2409_11382_gb300 import workloads as W
    params, _, _ = W.terzaghi_4097(precision=W.FP64)
    strip = dict(params, nx=512, lx=512 / 4096)
    o = O.Oracle(strip, W.top_load_sides(512, W.uniform_load(512)))
    o.step(0)  # elastic solve at t = 0 (untimed set-up)
    t0 = time.perf_counter()
    o.step(1)  # one Biot step: flow step + elastic solve
    dt = time.perf_counter() - t0
    o.close()
    return dt, 512 * params["ny"]


def cpu_baseline_entry():
    secs, cells = oracle_sample_step()
    return {"value": cells / secs / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"1 physical step of the same problem on a 512x4096-cell strip "
                      f"(x-independent solution, same per-cell work), {secs:.1f} s, FP64, 1 thread"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample_step()
    t = []
    cells = 0
    for _ in range(args.steps):
        secs, cells = oracle_sample_step()
        t.append(secs)
    total = sum(t)
    value = cells * args.steps / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps * (4096 * 4096) / cells,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + "_strip512_oracle", "cells": "512x4096",
                                        "levels": 10, "ne_fixed": 3, "K": 4},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": "each step: 1 physical step on a 512x4096-cell strip of the workload"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "ms_per_step extrapolated linearly from the strip to 4096x4096 cells",
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    from paper_2409_11382_gb300 import biot, workloads as W
    from paper_2409_11382_gb300 import build as B

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    params, sides, _ = W.terzaghi_4097(n=args.n)
    nx, ny = params["nx"], params["ny"]
    cells = nx * ny
    stream = torch.cuda.current_stream()
    solver = biot.Solver(params, sides, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        solver.step(1)
    torch.cuda.synchronize()
    launches0 = solver.stats()["kernel_launches"]

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    solver.step(args.steps)  # K time steps, each one CUDA-graph launch; one read-back at the end
    stop.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = start.elapsed_time(stop)
    clock_info = clocks.stop() if clocks else None
    launches = solver.stats()["kernel_launches"] - launches0
    st = solver.stats()

    # instrumented pass over the same number of steps (direct launches, CUDA
    # events around every finest-level smoothing sweep on the solver's stream)
    solver.sweep_timing(True)
    solver.step(args.steps)
    sweep_ms, sweep_n = solver.sweep_timing_get()
    solver.sweep_timing(False)

    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())

    # ---- end to end through the public API with host buffers ------------------------
    e2e_steps = max(1, min(args.steps, 5))
    load = W.uniform_load(nx)
    eta_prof = np.zeros((2, 2 * nx + 1))
    eta_prof[1] = -load
    pin_eta = torch.empty((2, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    pin_p = torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    pin_prof = torch.empty((2, 2 * nx + 1), dtype=torch.float64, pin_memory=True).numpy()
    pin_prof[:] = eta_prof
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_side_profile(W.TOP, pin_prof, np.zeros(2 * nx + 1))
        solver.step(1)
        solver.read_u(pin_eta)
        solver.read_p(pin_p)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = pin_prof.nbytes + 8 * (2 * nx + 1)
    d2h = pin_eta.nbytes + pin_p.nbytes
    finite = bool(np.isfinite(pin_eta).all() and np.isfinite(pin_p).all())
    solver.close()

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    value = world * cells * args.steps / (ms / 1e3) / 1e6
    peak, peak_kind = measured_peaks()
    # finest-level smoothing sweep, FP32: 8 moments + 2 low parts in and out, F~ in;
    # the prolongated correction (8 coarse moments per 4 cells) once per 2K sweeps
    bytes_per_cell = (10 + 10 + 2) * 4.0 + 8.0 / (2 * params["K"])
    avg_sweep_ms = sweep_ms / max(sweep_n, 1)
    achieved = bytes_per_cell * cells / (avg_sweep_ms / 1e3) / 1e9
    traffic_pc = profiled_traffic_per_cell()
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.n == 4096 else f"terzaghi_{args.n + 1}x{args.n + 1}_fp32",
                   "cells": f"{nx}x{ny}", "levels": params["levels"],
                   "ne_fixed": params["ne_fixed"], "K": params["K"], "gamma": params["gamma"],
                   "precision": "fp32 populations; fp64 residual norms, coarsest level, coupling",
                   "l2": "state (3.4 GB) larger than L2; no flush needed",
                   "parallelism": f"replicas{world}"},
        "roofline": {"kernel": "k_sweep_mom<float,float> finest level, smoothing", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                     "bytes_per_cell": bytes_per_cell, "launches": sweep_n, "avg_launch_ms": avg_sweep_ms,
                     "traffic": None if traffic_pc is None else traffic_pc * cells},
        "cpu_baseline": cpu_baseline_entry() if (rank == 0 and not args.no_cpu_baseline) else None,
        "e2e": {"value": cells * e2e_steps / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps, "finite": finite},
        "gpu_launches": launches,
        "clocks": clock_info,
        "solver": {"last_ne": st["last_ne"], "last_res": st["last_res"], "diverged": st["diverged"],
                   "device_bytes": st["device_bytes"]},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=4096, help="cells per side (4096 = the benchmark workload)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
