"""Benchmark: MLUPS and time per Biot step of the coupled LBM on one GB300.

Workload (one step = one physical time step of Alg. 5: explicit force, N_E = 3
multigrid V-cycles of the pseudo-time MRT elasticity LBM with K = 4 smoothing
sweeps per level, then the SRT pressure step): Terzaghi consolidation on
4097x4097 nodes (4096x4096 cells), FP32 populations with FP64 residual norms,
coarsest level and coupling accumulators, 10 multigrid levels.  Synthetic
input (the problem is fully defined by its parameters); all state stays
resident in HBM and is larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --precision fp64     # the plain FP64 path on the same problem

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
PROFILE64 = os.path.join(ROOT, "profiles", "sweep_fp64_terzaghi_4097.md")
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


def profiled_per_cell(key, path=PROFILE):
    """A per-cell figure of one finest-level sweep (``key: value``) from a
    committed ncu summary, or None if the kernel source changed since the
    counters were taken."""
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(key + r":\s*([0-9.]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_sha():
        return None
    return float(m.group(1))


def profiled_traffic_per_cell(path=PROFILE):
    return profiled_per_cell("traffic_bytes_per_cell", path)


DEV_PRECISIONS = {"fp32dev16": 3, "fp32devbf16": 4}  # BIOT_FP32_DEV16, BIOT_FP32_DEVBF16 of include/biot.h


def step_model(params, n, fp64, dev=False):
    """Sweeps and algorithmic bytes of one physical step with fixed V-cycle counts
    (N_E V-cycles of 2K smoothing sweeps and one residual + restriction sweep per
    level, 2K sweeps on the coarsest level, then the fused flow step).  Per cell
    and sweep:
      finest smoothing: 5 moments in and out, F~ in, with FP32 storage the 2 low
        parts in and out, plus the prolongated correction (5 coarse moments per 4
        cells) once per 2K sweeps;
      finest residual + restriction: the same inputs, 5 coarse moments per 4 cells out;
      coarse smoothing: 5 moments and 5 of r in, 5 moments out (+ prolongation);
      coarse residual + restriction: 10 in, 5 coarse out per 4 cells;
      coarsest level: as coarse smoothing (FP64 on the FP32 path, FP32 with
        the option BIOT_OPT_COARSEST_STORAGE);
      flow step: 9 f in and out, m_s, D(t - dt) (FP64) and the previous history
        difference in, D(t) (FP64), the new difference and F~ out.
    With the 16-bit deviation store (dev) the finest level's m_11, m_s, m_d move
    as 2-byte values; the last finest sweep of a solve also writes them in FP32
    (3 planes, once per solve).
    Returns (cell-sweeps per step, bytes per step)."""
    L, K, ne = params["levels"], params["K"], params["ne_fixed"]
    K_level = list(params.get("K_level", ())) + [0] * 16

    def sweeps(l):  # per-level smoothing sweeps (level l from the coarsest)
        k = K_level[L - 1 - l]
        return k if k > 0 else K
    esz = 8 if fp64 else 4
    c64 = coarsest_fp64(params)
    cell_sweeps = 0.0
    nbytes = 0.0
    for l in range(L - 1, -1, -1):  # finest first
        side = n >> (L - 1 - l)
        c = float(side * side)
        e = 8 if (l == 0 and L > 1 and c64) or fp64 else esz
        ec = 8 if (l == 1 and L > 1 and c64) or fp64 else esz  # storage of the next coarser level
        fine = l == L - 1
        nlo = 2 if (fine and not fp64) else 0
        xin = 2 if fine else 5  # F~ or r
        Kl = sweeps(l)
        prol = 5 * ec / 4.0 / (2 * Kl) if l > 0 else 0.0  # correction from level l - 1
        nst = 3 if (fine and dev) else 0  # moments in the 2-byte store
        smooth = ((5 - nst + nlo) * 2 + xin) * e + nst * 2 * 2 + prol
        cell_sweeps += ne * 2 * Kl * c
        nbytes += ne * 2 * Kl * c * smooth
        if fine and dev:
            nbytes += c * 3 * e  # the FP32 copy of the last sweep of the solve
        if l > 0:
            cell_sweeps += ne * c
            nbytes += ne * c * ((5 - nst + nlo + xin) * e + nst * 2 + 5 * ec / 4.0)
    fine_cells = float(n * n)
    fe = 8 if fp64 else 4
    nbytes += fine_cells * (9 * fe * 2 + fe + 8 + fe + 8 + fe + 2 * fe)
    return cell_sweeps, nbytes


OPT_COARSEST_STORAGE, OPT_COLD_FP64, OPT_COLD_FP32, OPT_SEGMENTS = 1, 2, 4, 32  # biot_params.options flags of include/biot.h


def coarsest_fp64(params):
    """Whether the FP32 path runs the coarsest multigrid level in FP64 (the
    default; FP32 with the option BIOT_OPT_COARSEST_STORAGE)."""
    return not (int(params.get("options", 0)) & OPT_COARSEST_STORAGE)


def precision_label(params, fp64):
    """What the run computes in, from the parameters the library was given."""
    if fp64:
        return "fp64 storage and arithmetic"
    prec = int(params.get("precision", 1))
    store = {3: "; finest m_11, m_s, m_d stored as fp16 deviation", 4: "; finest m_11, m_s, m_d stored as bf16 deviation"}.get(prec, "")
    cells = params["nx"] * params["ny"]
    opt = int(params.get("options", 0))
    cold64 = bool(opt & OPT_COLD_FP64) or (cells >= 2048 * 2048 and not opt & OPT_COLD_FP32)
    return ("fp32 moments and collisions; fp64 residual norms, coupling accumulators and "
            + ("coarsest level" if coarsest_fp64(params) else "no level (coarsest level fp32)")
            + ("; fp64 solve at t = 0" if cold64 else "") + store)


def measured_fp64_peak(torch):
    """FP64 arithmetic peak of this GPU, measured: the best of 3 timed FP64 GEMMs
    of 4096^3 (cuBLAS through torch), in FLOP/s."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return 2.0 * n ** 3 / (best / 1e3)


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


def oracle_strip():
    """The oracle on the benchmark workload restricted to a 512-cell-wide strip:
    the problem does not depend on x, so every cell does the same work as in
    the full grid.  Returns (oracle, cells)."""
    from oracle import oracle as O
    from paper_2409_11382_gb300 import workloads as W
    params, _, _ = W.terzaghi_4097(precision=W.FP64)
    strip = dict(params, nx=512, lx=512 / 4096)
    return O.Oracle(strip, W.top_load_sides(512, W.uniform_load(512))), 512 * params["ny"]


def timed_oracle_step(o, threads):
    """Seconds of one physical step (flow step + elastic solve) of the oracle
    on ``threads`` host threads, and the thread count it actually used."""
    from oracle import oracle as O
    used = O.set_threads(threads)
    t0 = time.perf_counter()
    o.step(1)
    return time.perf_counter() - t0, used


GOLDEN_STRIP = os.path.join(ROOT, "tests", "golden", "terzaghi_4096_strip_fp64.npz")


def accuracy_vs_oracle(oracle_fields, n, params_over=None, precision=None):
    """L-infinity and L2 relative errors of eta and p of the GPU path against the
    FP64 oracle on the benchmark problem, which does not depend on x: after 1,
    10 and 100 steps against the oracle's stored column (tests/golden, written
    by the oracle on a 512-column strip of the same problem), every GPU column
    compared.  Without the stored columns: after 1 step against the live strip
    in ``oracle_fields``."""
    from paper_2409_11382_gb300 import biot, workloads as W
    params, sides, _ = W.terzaghi_4097(n=n, precision=W.FP32 if precision is None else precision)
    params = dict(params, **(params_over or {}))

    def errs(eta, p, eta_o, p_o):
        out = {}
        for name, g, o in (("eta", eta, eta_o), ("p", p, p_o)):
            d = g - o
            out[f"{name}_linf_rel"] = float(np.abs(d).max() / np.abs(o).max())
            out[f"{name}_l2_rel"] = float(np.sqrt((d * d).sum() / (o * o * np.ones_like(g)).sum()))
        return out

    if n == 4096 and os.path.exists(GOLDEN_STRIP):
        gold = np.load(GOLDEN_STRIP)
        per_step = {}
        done = 0
        with biot.Solver(params, sides) as s:
            for k, steps in enumerate(gold["steps"]):
                s.step(int(steps) - done)
                done = int(steps)
                eta, t = s.read_u()
                p, _ = s.read_p()
                assert abs(t - gold["t"][k]) < 1e-12
                per_step[str(int(steps))] = errs(eta, p, gold["eta"][k][:, :, None], gold["p"][k][:, None])
        out = dict(per_step[str(int(gold["steps"][-1]))])
        out["per_step"] = per_step
        out["how"] = (f"after {int(gold['steps'][-1])} steps (also 1 and 10 in per_step), all {n} columns vs the "
                      "FP64 oracle's column of the same x-independent problem (512-column strip)")
        return out
    with biot.Solver(params, sides) as s:
        s.step(1)
        eta, _ = s.read_u()
        p, _ = s.read_p()
    out = errs(eta[:, :, :512], p[:, :512], oracle_fields["eta"], oracle_fields["p"])
    out["how"] = "after 1 step, first 512 columns vs the FP64 oracle on a 512-column strip"
    return out


def cpu_baseline_entry(keep=None):
    """The oracle timed on this host's cores: one step on every core (OpenMP over
    the cells; bitwise the single-thread result), then one on one core."""
    nproc = os.cpu_count() or 1
    o, cells = oracle_strip()
    o.step(0)  # elastic solve at t = 0 (untimed set-up)
    secs_n, used = timed_oracle_step(o, nproc)
    if keep is not None:
        keep["eta"], keep["p"] = o.read_u()[0], o.read_p()[0]
    secs_1, _ = timed_oracle_step(o, 1)
    o.close()
    return {"value": cells / secs_n / 1e6, "unit": "MLUPS", "cores": used, "kind": "oracle", "nproc": nproc,
            "sample": f"1 physical step of the same problem on a 512x4096-cell strip "
                      f"(x-independent solution, same per-cell work), {secs_n:.1f} s, FP64, "
                      f"OpenMP over cells on {used} threads",
            "single_thread": {"value": cells / secs_1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": f"the next step of the same strip on 1 thread, {secs_1:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    nproc = os.cpu_count() or 1
    o, cells = oracle_strip()
    o.step(0)  # elastic solve at t = 0 (untimed set-up)
    used = 1
    for _ in range(args.warmup):
        timed_oracle_step(o, nproc)
    t = []
    for _ in range(args.steps):
        secs, used = timed_oracle_step(o, nproc)
        t.append(secs)
    o.close()
    total = sum(t)
    value = cells * args.steps / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps * (4096 * 4096) / cells,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": "4096x4096", "levels": 10, "ne_fixed": 3, "K": 4, "gamma": 0.75,
                   "precision": "fp64 (the oracle)", "parallelism": "replicas1",
                   "ms_per_step_extrapolated": True,
                   "ms_per_step_from": "the timed 512x4096-cell strip, scaled by cells to 4096x4096",
                   "timed_cells_per_step": cells, "host_threads": used, "nproc": nproc},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": used, "kind": "oracle", "nproc": nproc,
                         "sample": "each step: 1 physical step of the workload restricted to a 512x4096-cell "
                                   "strip (x-independent solution, same per-cell work), OpenMP over cells"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "ms_per_step extrapolated linearly from the strip to 4096x4096 cells",
    }
    print(json.dumps(line), flush=True)
    return 0


def _init_dist(world):
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _finish_dist(world):
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ours(args):
    import torch
    from paper_2409_11382_gb300 import dist as D
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
    fp64 = args.precision == "fp64"
    dev = args.precision in DEV_PRECISIONS
    params, sides, _ = W.terzaghi_4097(n=args.n, precision=W.FP64 if fp64 else DEV_PRECISIONS.get(args.precision, W.FP32))
    if args.coarsest == "fp32":
        params = dict(params, options=int(params.get("options", 0)) | OPT_COARSEST_STORAGE)
    if args.cold != "auto":
        params = dict(params, options=int(params.get("options", 0)) | (OPT_COLD_FP64 if args.cold == "fp64" else OPT_COLD_FP32))
    if args.segments:
        params = dict(params, options=int(params.get("options", 0)) | OPT_SEGMENTS)
    nx, ny = params["nx"], params["ny"]
    cells = nx * ny
    stream = torch.cuda.current_stream()
    solver = biot.Solver(params, sides, stream=stream.cuda_stream)
    # launch shapes (results unchanged); the FP64 path keeps the default shapes
    tuned = solver.autotune() if not (args.no_tune or fp64) else None

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

    ms = D.max_over_ranks(ms, device="cuda")  # slowest rank (no-op on one GPU)

    # ---- end to end through the public API with host buffers ------------------------
    # Each step: H2D of the top-load profile from page-locked memory, the step,
    # and an asynchronous read-out of eta and p into page-locked host arrays
    # (two sets, alternating), whose copy overlaps the next step.  None of the
    # three calls waits for the GPU (biot_step_async); the clock stops after
    # biot_sync, once every step has run and every copy has reached the host.
    e2e_steps = max(1, args.steps)  # as many steps as the device-timed region
    load = W.uniform_load(nx)
    pin = lambda shape: torch.zeros(shape, dtype=torch.float64, pin_memory=True).numpy()
    pin_eta = [pin((2, ny, nx)) for _ in range(2)]
    pin_p = [pin((ny, nx)) for _ in range(2)]
    pin_prof, pin_pprof = pin((2, 2 * nx + 1)), pin((2 * nx + 1,))
    pin_prof[1] = -load
    for k in range(2):  # two untimed iterations: staging buffers, graphs of both flow parities
        solver.set_side_profile(W.TOP, pin_prof, pin_pprof)
        solver.step_async(1)
        solver.read_async(eta=pin_eta[k], p=pin_p[k])
    solver.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        solver.set_side_profile(W.TOP, pin_prof, pin_pprof)
        solver.step_async(1)
        solver.read_async(eta=pin_eta[k % 2], p=pin_p[k % 2])
    solver.sync()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = pin_prof.nbytes + pin_pprof.nbytes
    d2h = pin_eta[0].nbytes + pin_p[0].nbytes
    finite = bool(all(np.isfinite(a).all() for a in pin_eta + pin_p))
    solver.close()

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    value = world * cells * args.steps / (ms / 1e3) / 1e6
    peak, peak_kind = measured_peaks()
    cpu_base, accuracy = None, None
    if args.n == 4096:
        fields = {}
        if not args.no_cpu_baseline:
            cpu_base = cpu_baseline_entry(fields)
        if fields or os.path.exists(GOLDEN_STRIP):
            accuracy = accuracy_vs_oracle(fields, args.n, {"options": params.get("options", 0)}, params["precision"])
    # finest-level smoothing sweep, fixed V-cycle count: the 5 moments that carry
    # state (the ghost moments 12, 21, 22 are elided) in and out, F~ in, with FP32
    # storage also the 2 low parts of the first moments in and out; the
    # prolongated correction (5 coarse moments per 4 cells) once per 2K sweeps
    nm = 5 if params["ne_fixed"] > 0 else 8
    esz = 8.0 if fp64 else 4.0
    nlo = 0 if fp64 else 2
    nst = 3 if dev else 0  # m_11, m_s, m_d as 2-byte values
    bytes_per_cell = ((nm - nst + nlo) * 2 + 2) * esz + nst * 2 * 2 + nm * esz / 4.0 / (2 * params["K"])
    avg_sweep_ms = sweep_ms / max(sweep_n, 1)
    achieved = bytes_per_cell * cells / (avg_sweep_ms / 1e3) / 1e9
    traffic_pc = profiled_traffic_per_cell(PROFILE64 if fp64 else PROFILE)
    hbm_roof = {"kernel": f"k_sweep_mom<{'double,double' if fp64 else 'float,float'}> finest level, smoothing",
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                "bytes_per_cell": bytes_per_cell, "launches": sweep_n, "avg_launch_ms": avg_sweep_ms,
                "traffic": None if traffic_pc is None else traffic_pc * cells}
    roofline, roofline_other = hbm_roof, None
    if fp64:
        # FP64 arithmetic: FP64 instructions per cell from the committed ncu counters
        # against the measured FP64 rate (FP64 GEMM FLOP/s / 2 = FP64 instructions/s,
        # one FMA being two FLOP); this path is built without fused multiply-adds
        inst_pc = profiled_per_cell("fp64_inst_per_cell", PROFILE64)
        peak64 = measured_fp64_peak(torch) / 2.0 / 1e9
        ach64 = None if inst_pc is None else inst_pc * cells / (avg_sweep_ms / 1e3) / 1e9
        roofline = {"kernel": hbm_roof["kernel"], "bound": "fp64", "achieved": ach64, "peak": peak64,
                    "unit": "G FP64-inst/s", "frac": None if ach64 is None else ach64 / peak64,
                    "peak_kind": "measured FP64 GEMM rate (cuBLAS, 4096^3) / 2 FLOP per FMA",
                    "fp64_inst_per_cell": inst_pc, "launches": sweep_n, "avg_launch_ms": avg_sweep_ms,
                    "traffic": hbm_roof["traffic"]}
        roofline_other = hbm_roof
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
        "storage": args.precision,
        "config": {"workload": f"terzaghi_{args.n + 1}x{args.n + 1}_{args.precision}",
                   "cells": f"{nx}x{ny}", "levels": params["levels"],
                   "ne_fixed": params["ne_fixed"], "K": params["K"], "gamma": params["gamma"],
                   "precision": precision_label(params, fp64),
                   "l2": f"state ({st['device_bytes'] / 1e9:.1f} GB) larger than L2; no flush needed",
                   "parallelism": f"replicas{world}",
                   "coarse_sweeps": "cluster segments" if args.segments else "separate graph-launched kernels",
                   "autotuned_strip_rows": tuned},
        "roofline": roofline,
        "cpu_baseline": cpu_base,
        "accuracy": accuracy,
        "e2e": {"value": cells * e2e_steps / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps, "finite": finite},
        "gpu_launches": launches,
        "clocks": clock_info,
        "solver": {"last_ne": st["last_ne"], "last_res": st["last_res"], "diverged": st["diverged"],
                   "device_bytes": st["device_bytes"]},
    }
    if roofline_other is not None:
        line["roofline_hbm"] = roofline_other
    if params["ne_fixed"] > 0:
        sweeps, nb = step_model(params, args.n, fp64, dev)
        t_step = ms / args.steps / 1e3
        line["step"] = {"mlups_sweep": world * sweeps / t_step / 1e6,
                        "algorithmic_bytes_per_step": nb, "achieved_gbs": nb / t_step / 1e9,
                        "frac": nb / t_step / 1e9 / peak,
                        "peak_kind": f"{peak_kind} copy bandwidth",
                        "population_model_frac": (params["ne_fixed"] * 900.0 + 140.0) * cells / t_step / 1e9 / peak,
                        "population_model": "N_E * 0.90 KB + 0.14 KB per fine cell (8 FP32 populations per cell-sweep)"}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def oracle_errors(cases, steps):
    """Max over cases of the L-infinity / L2 relative errors of eta and p against
    the FP64 oracle run for the same number of steps.  cases: [((params, sides), (eta, p))]."""
    from oracle import oracle as O
    from paper_2409_11382_gb300 import workloads as W
    out = {"eta_linf_rel": 0.0, "eta_l2_rel": 0.0, "p_linf_rel": 0.0, "p_l2_rel": 0.0}
    for (params, sides), (eta, p) in cases:
        o = O.Oracle(dict(params, precision=W.FP64), sides)
        o.step(steps)
        eo, po = o.read_u()[0], o.read_p()[0]
        o.close()
        for name, g, r in (("eta", eta, eo), ("p", p, po)):
            out[f"{name}_linf_rel"] = max(out[f"{name}_linf_rel"], float(np.abs(g - r).max() / np.abs(r).max()))
            out[f"{name}_l2_rel"] = max(out[f"{name}_l2_rel"], float(np.linalg.norm(g - r) / np.linalg.norm(r)))
    out["how"] = f"{len(cases)} smallest instance(s) after {steps} steps vs the FP64 oracle"
    return out


def strip_oracle_errors(params, sides_fn, steps, eta, p):
    """L-infinity and L2 relative errors of an x-independent solve (uniform top
    load, mirror sides) against the FP64 oracle run on the narrowest strip of the
    same problem whose hierarchy still coarsens (2^(levels-1) columns): every GPU
    column against the oracle's first column."""
    from oracle import oracle as O
    from paper_2409_11382_gb300 import workloads as W
    w = 1 << (params["levels"] - 1)
    strip = dict(params, nx=w, lx=params["lx"] * w / params["nx"], precision=W.FP64)
    o = O.Oracle(strip, sides_fn(w))
    o.step(steps)
    eo, po = o.read_u()[0][:, :, :1], o.read_p()[0][:, :1]
    o.close()
    out = {}
    for name, g, r in (("eta", eta, eo), ("p", p, po)):
        d = g - r
        out[f"{name}_linf_rel"] = float(np.abs(d).max() / np.abs(r).max())
        out[f"{name}_l2_rel"] = float(np.sqrt((d * d).sum() / (r * r * np.ones_like(g)).sum()))
    return out


def _percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def run_batched(args):
    """64 seeded uneven instances (sides 64..512 cells, random materials and partial
    top loads), FP32, MG(3,4); one CUDA graph per physical step of all instances."""
    import torch
    from paper_2409_11382_gb300 import biot, build as B, dist as D, workloads as W
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    _init_dist(world)
    if rank == 0:
        B.build()
    _barrier(world)
    # weak scaling: every rank advances its own 64 seeded instances
    probs = W.batched_instances(count=args.instances, seed=2409 + 7919 * rank)
    if args.precision in DEV_PRECISIONS:
        probs = [(dict(p, precision=DEV_PRECISIONS[args.precision]), s) for p, s in probs]
    if args.segments:
        probs = [(dict(p, options=int(p.get("options", 0)) | OPT_SEGMENTS), s) for p, s in probs]
    cells = sum(p["nx"] * p["ny"] for p, _ in probs)
    b = biot.Batch(probs)
    b.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    _barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    t0 = time.perf_counter()
    b.step(args.steps)  # one graph launch per step, one read-back at the end
    ev1.record()
    torch.cuda.synchronize()
    _barrier(world)
    secs = D.max_over_ranks(max(time.perf_counter() - t0, ev0.elapsed_time(ev1) / 1e3), device="cuda")
    clock_info = clocks.stop() if clocks else None
    st = b.stats()
    # end to end: each step, H2D of every instance's top-load profile and D2H of
    # eta and p, as in the single-instance line: page-locked buffers, steps and
    # reads queued without waiting (two output sets, alternating), clock stopped
    # after biot_batch_sync
    e2e_steps = max(1, args.steps)  # as many steps as the device-timed region

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy()
        t[:] = a
        return t

    views = [b[i] for i in range(len(b))]
    profs = [(pinned(sides[W.TOP]["eta_profile"]), pinned(sides[W.TOP]["p_profile"])) for _, sides in probs]
    outs = [[(pinned(np.zeros((2, p["ny"], p["nx"]))), pinned(np.zeros((p["ny"], p["nx"])))) for p, _ in probs]
            for _ in range(2)]
    etas = [[eta for eta, _ in o] for o in outs]
    prs = [[pr for _, pr in o] for o in outs]
    for k in range(2):  # two untimed iterations: staging buffers, graphs of both flow parities
        for v, (ep, pp) in zip(views, profs):
            v.set_side_profile(W.TOP, ep, pp)
        b.step_async(1)
        b.read_async(eta=etas[k], p=prs[k])
    b.sync()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for k in range(e2e_steps):
        for v, (ep, pp) in zip(views, profs):
            v.set_side_profile(W.TOP, ep, pp)
        b.step_async(1)
        b.read_async(eta=etas[k % 2], p=prs[k % 2])  # every instance's eta and p, one call
    b.sync()
    torch.cuda.synchronize()
    e2e = time.perf_counter() - t1
    h2d = sum(ep.nbytes + pp.nbytes for ep, pp in profs)
    d2h = e2e_steps * sum(eta.nbytes + pr.nbytes for eta, pr in outs[0])
    e2e_finite = bool(all(np.isfinite(a).all() for o in outs for pair in o for a in pair))
    total_steps = args.warmup + args.steps + 2 + e2e_steps
    small = sorted(range(len(probs)), key=lambda i: probs[i][0]["nx"])[:2]
    got = {i: (b[i].read_u()[0], b[i].read_p()[0]) for i in small}
    b.close()
    accuracy = oracle_errors([(probs[i], got[i]) for i in small], total_steps) if rank == 0 else None
    value = world * cells * args.steps / secs / 1e6
    # step-level roofline: the algorithmic bytes of every instance's step (the
    # per-sweep model of step_model) over the measured time per step
    dev = args.precision in DEV_PRECISIONS
    step_bytes = sum(step_model(p, p["nx"], False, dev)[1] for p, _ in probs)
    peak, peak_kind = measured_peaks()
    achieved = world * step_bytes / (secs / args.steps) / 1e9
    roofline = {"kernel": "whole batched step (every phase launch and the flow steps)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": f"{peak_kind} copy bandwidth (burst)", "bytes_per_step": step_bytes, "traffic": None}
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "roofline": roofline,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "storage": args.precision if args.precision in DEV_PRECISIONS else "fp32",
            "config": {"workload": "batched_64_instances_64-512_fp32", "instances": len(probs),
                       "cells_total": cells, "ne_fixed": 3, "K": 4,
                       "l2": "state of all instances larger than L2; no flush needed",
                       "parallelism": f"replicas{world}",
                       "coarse_sweeps": "cluster segments" if args.segments else "separate graph-launched kernels",
                       "launches_per_step": st["launches_per_step"]},
            "e2e": {"value": cells * e2e_steps / e2e / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h // e2e_steps,
                    "finite": e2e_finite},
            "gpu_launches": st["launches_per_step"] * args.steps,
            "batch": st, "accuracy": accuracy, "clocks": clock_info}
    if rank == 0:
        print(json.dumps(line), flush=True)
    _finish_dist(world)
    return 0


def run_served(args):
    """Seeded Poisson stream of solve requests (sides 64..1024 cells, the 4097^2
    case's materials, 100 steps to T = 0.1, FP32) through the continuous-batching
    server; then the same requests one at a time through the plain FP64 path (and
    the plain FP32 path) with the same arrival times (first come, first served)."""
    import torch
    from paper_2409_11382_gb300 import biot, build as B, workloads as W
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    _init_dist(world)
    if rank == 0:
        B.build()
    _barrier(world)
    reqs = W.served_requests(count=args.requests, seed=11382 + 7919 * rank,
                             mean_service_s=args.mean_service)
    cells_steps = sum(p["nx"] * p["ny"] * round(T / p["dt"]) for _, p, _, T in reqs)
    budget = int(args.budget_gb * (1 << 30))
    # warm-up: kernels, graphs and the allocator on one small request of each size
    for n in sorted({p["nx"] for _, p, _, _ in reqs}):
        _, p, s, T = next(r for r in reqs if r[1]["nx"] == n)
        with biot.Solver(p, s) as sol:
            sol.step(2)
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    with biot.Server(budget, max_resident=args.max_resident) as srv:
        ids = []
        t0 = time.perf_counter()
        for arrival, p, s, T in reqs:
            delay = arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(p, s, T))
        for rid in ids:
            srv.wait(rid, timeout=3600)
        makespan = time.perf_counter() - t0
        infos = [srv.poll(rid) for rid in ids]
        st = srv.stats()
        checks = [srv.fetch(rid) for rid in ids[:2]]
        ismall = min(range(len(reqs)), key=lambda i: reqs[i][1]["nx"])
        ilarge = max(range(len(reqs)), key=lambda i: reqs[i][1]["nx"])
        small_res = srv.fetch(ids[ismall])
        large_res = srv.fetch(ids[ilarge])
    clock_info = clocks.stop() if clocks else None
    lat = [i["t_done"] - i["t_submit"] for i in infos]

    def one_at_a_time(precision):
        finish, lats, busy = 0.0, [], 0.0
        for arrival, p, s, T in reqs:
            t1 = time.perf_counter()
            with biot.Solver(dict(p, precision=precision), s) as sol:
                sol.solve_to(T)
                sol.read_u()
                sol.read_p()
            svc = time.perf_counter() - t1
            busy += svc
            finish = max(arrival, finish) + svc
            lats.append(finish - arrival)
        return {"p50_s": _percentile(lats, 50), "p99_s": _percentile(lats, 99),
                "throughput_mlups": cells_steps / busy / 1e6, "busy_s": busy}

    plain64 = one_at_a_time(W.FP64)
    plain32 = one_at_a_time(W.FP32)
    # the first two served results against their plain FP32 solo runs (same kernels)
    same = True
    for (arrival, p, s, T), (eta, pr, t) in zip(reqs[:2], checks):
        with biot.Solver(p, s) as sol:
            sol.solve_to(T)
            same = same and np.array_equal(eta, sol.read_u()[0]) and np.array_equal(pr, sol.read_p()[0])
    _, sp, ss, sT = reqs[ismall]
    accuracy = oracle_errors([((sp, ss), (small_res[0], small_res[1]))], int(round(sT / sp["dt"]))) if rank == 0 else None
    if rank == 0:
        _, lp, _, lT = reqs[ilarge]
        accuracy = {"smallest": accuracy,
                    "largest": dict(strip_oracle_errors(lp, lambda w: W.top_load_sides(w, W.uniform_load(w)),
                                                        int(round(lT / lp["dt"])), large_res[0], large_res[1]),
                                    how=f"{lp['nx']}^2 request after {int(round(lT / lp['dt']))} steps, every column "
                                        "vs the FP64 oracle on a strip of the same x-independent problem")}
    value = world * cells_steps / makespan / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.requests, "accuracy": accuracy, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served_poisson_64-1024_fp32", "requests": len(reqs),
                       "mean_in_flight_target": 8, "budget_gb": args.budget_gb,
                       "max_resident": args.max_resident, "parallelism": f"replicas{world}"},
            "latency": {"p50_s": _percentile(lat, 50), "p99_s": _percentile(lat, 99),
                        "makespan_s": makespan},
            "plain_fp64_one_at_a_time": plain64, "plain_fp32_one_at_a_time": plain32,
            "served_equals_solo": same, "server": st, "clocks": clock_info}
    if rank == 0:
        print(json.dumps(line), flush=True)
    _finish_dist(world)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip biot_autotune (default launch shapes)")
    ap.add_argument("--n", type=int, default=4096, help="cells per side (4096 = the benchmark workload)")
    ap.add_argument("--workload", choices=["single", "batched", "served"], default="single")
    ap.add_argument("--precision", choices=["fp32", "fp64"] + sorted(DEV_PRECISIONS), default="fp32",
                    help="single: the FP32 path (default), the plain FP64 path, or the FP32 path with the "
                         "16-bit deviation store; batched: fp32 or a deviation store")
    ap.add_argument("--instances", type=int, default=64, help="batched: number of instances")
    ap.add_argument("--coarsest", choices=["fp64", "fp32"], default="fp64",
                    help="single, FP32 path: precision of the coarsest multigrid level")
    ap.add_argument("--cold", choices=["auto", "fp64", "fp32"], default="auto",
                    help="single, FP32 path: the solve at t = 0 on an FP64 copy (auto: from 2048^2 cells)")
    ap.add_argument("--segments", action="store_true",
                    help="the sweeps of the small coarse levels as cluster segments (BIOT_OPT_SEGMENTS)")
    ap.add_argument("--requests", type=int, default=200, help="served: number of requests")
    ap.add_argument("--mean-service", type=float, default=0.05, help="served: assumed mean service time (s)")
    ap.add_argument("--budget-gb", type=float, default=16.0, help="served: device-memory budget")
    ap.add_argument("--max-resident", type=int, default=16, help="served: resident-instance limit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
