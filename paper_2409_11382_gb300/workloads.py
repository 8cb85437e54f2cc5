"""Seeded synthetic workloads shared by the CUDA path and the oracle.

This module only builds inputs: parameter sets and boundary-data profiles of
the consolidation problems used for parity tests and benchmarks.  It holds none
of the method's arithmetic and imports neither the CUDA binding nor the oracle.

A parameter set is a plain dict with the keys
    nx, ny, lx, ly, lam, mu, alpha, c0, kappa, dt, r, levels, K, gamma,
    tol, ne_max, ne_fixed, precision
and ``sides`` is a list of four dicts (bottom, right, top, left) with
``eta_type`` / ``p_type`` (PERIODIC, SYMMETRY, DIRICHLET, NEUMANN) and optional
``eta_profile`` (shape (2, 2n+1): Dirichlet displacement or Neumann traction)
and ``p_profile`` (shape (2n+1,): Dirichlet pressure).  Profile sample k sits
at arc position k*h/2 along the side (even k: cell faces, odd k: centres).

Problem statements: Terzaghi's consolidation problem of §4.2 (quasi-1D, top
load, drained top, fixed bottom) and the step-load 2D extension of §4.3; the
grid sizes, material values and step counts are those of the benchmark
configurations (nodes n -> n-1 cells on the cell-centred lattice).
"""
from __future__ import annotations

import numpy as np

PERIODIC, SYMMETRY, DIRICHLET, NEUMANN = 0, 1, 2, 3
BOTTOM, RIGHT, TOP, LEFT = 0, 1, 2, 3
FP64, FP32, FP32_COARSE64, FP32_DEV16, FP32_DEVBF16 = 0, 1, 2, 3, 4


def _params(n, *, lam, mu, alpha, c0, kappa, dt, levels, K=4, gamma=0.75, r=0.5,
            tol=1e-10, ne_max=100, ne_fixed=0, precision=FP64, ny=None, lx=1.0):
    ny = n if ny is None else ny
    return dict(nx=n, ny=ny, lx=lx, ly=lx * ny / n, lam=lam, mu=mu, alpha=alpha, c0=c0,
                kappa=kappa, dt=dt, r=r, levels=levels, K=K, gamma=gamma, tol=tol,
                ne_max=ne_max, ne_fixed=ne_fixed, precision=precision)


def top_load_sides(nx: int, load: np.ndarray, side_type=SYMMETRY):
    """Bottom: fixed displacement, no flow.  Top: traction (0, -load(x)), p = 0.
    Left/right: ``side_type`` for both fields (SYMMETRY = roller + no flux, or PERIODIC)."""
    eta_top = np.zeros((2, 2 * nx + 1))
    eta_top[1] = -np.asarray(load, dtype=np.float64)
    return [
        dict(eta_type=DIRICHLET, p_type=NEUMANN),
        dict(eta_type=side_type, p_type=side_type),
        dict(eta_type=NEUMANN, p_type=DIRICHLET, eta_profile=eta_top,
             p_profile=np.zeros(2 * nx + 1)),
        dict(eta_type=side_type, p_type=side_type),
    ]


def uniform_load(nx: int, sigma0: float = 1.0) -> np.ndarray:
    return np.full(2 * nx + 1, sigma0)


def step_load(nx: int, x_end: float = 0.5, sigma0: float = 1.0, lx: float = 1.0) -> np.ndarray:
    """sigma0 for x < x_end, sigma0/2 exactly at x_end, 0 beyond (samples at k*h/2)."""
    x = np.arange(2 * nx + 1) * (lx / nx) / 2.0
    v = np.where(x < x_end, sigma0, 0.0)
    v[np.isclose(x, x_end)] = 0.5 * sigma0
    return v


# ---------------------------------------------------------------------------
# Benchmark / parity configurations.
# ---------------------------------------------------------------------------

def terzaghi_33(precision=FP64, side_type=SYMMETRY):
    """Terzaghi consolidation, 33x33 nodes (32x32 cells), unit square,
    lambda = mu = 1, alpha = 1, c0 = 0.1, kappa = 1, unit top load at t = 0+,
    3 levels, residual tolerance 1e-10, 50 steps to T = 0.1."""
    n = 32
    p = _params(n, lam=1.0, mu=1.0, alpha=1.0, c0=0.1, kappa=1.0, dt=0.1 / 50, levels=3,
                tol=1e-10, precision=precision)
    return p, top_load_sides(n, uniform_load(n), side_type), 50


def step_load_257(alpha=1.0, precision=FP64, n=256, ne_fixed=3, steps=200):
    """2D Terzaghi extension, 257x257 nodes (256x256 cells): load 1 on the top
    for x < 0.5, traction-free elsewhere; lambda = mu = 1, c0 = 0.01, kappa = 1,
    6 levels, 200 steps to T = 0.1, fixed MG(3,4)."""
    levels = int(np.log2(n)) - 2
    p = _params(n, lam=1.0, mu=1.0, alpha=alpha, c0=0.01, kappa=1.0, dt=0.1 / 200,
                levels=levels, ne_fixed=ne_fixed, precision=precision)
    return p, top_load_sides(n, step_load(n)), steps


def terzaghi_4097(precision=FP32, n=4096, ne_fixed=3, steps=100):
    """Single large instance, 4097x4097 nodes (4096x4096 cells), same boundary
    conditions as the 33x33 Terzaghi case; lambda = mu = 1, alpha = 1,
    c0 = 0.1, kappa = 1e-2, 10 levels, 100 steps to T = 0.1, fixed MG(3,4)."""
    levels = int(np.log2(n)) - 2
    p = _params(n, lam=1.0, mu=1.0, alpha=1.0, c0=0.1, kappa=1e-2, dt=0.1 / 100,
                levels=levels, ne_fixed=ne_fixed, precision=precision)
    return p, top_load_sides(n, uniform_load(n)), steps


def paper_terzaghi(n: int, alpha: float = 1.0, ne_fixed=3, K=4, side_type=PERIODIC):
    """Terzaghi's problem with the parameters of §4.2: E = 1, nu = 0.8 (plane
    stress), kappa = (25 + 9 alpha^2)/25, load varpi = alpha + (lam+2mu)/alpha so
    that p0 = 1, c0 = 1, dt = dx^2/4, periodic sides, MG(ne_fixed, K)."""
    lam, mu = 20.0 / 9.0, 5.0 / 18.0
    kappa = (25.0 + 9.0 * alpha ** 2) / 25.0
    varpi = alpha + (lam + 2 * mu) / alpha
    h = 1.0 / n
    p = _params(n, lam=lam, mu=mu, alpha=alpha, c0=1.0, kappa=kappa, dt=h * h / 4,
                levels=int(np.log2(n)), K=K, ne_fixed=ne_fixed)
    return p, top_load_sides(n, uniform_load(n, varpi), side_type), varpi


def manufactured_params(n: int, alpha: float, r: float, ne_fixed=3, K=2):
    """Periodic manufactured problem of §4.1: (0,1)^2, lambda = 11/45,
    mu = 11/360, kappa = 1/10, c0 = 1, dt = dx^2, all sides periodic, MG(ne_fixed, K)."""
    h = 1.0 / n
    p = _params(n, lam=11.0 / 45.0, mu=11.0 / 360.0, alpha=alpha, c0=1.0, kappa=0.1,
                dt=h * h, levels=int(np.log2(n)), K=K, r=r, ne_fixed=ne_fixed)
    sides = [dict(eta_type=PERIODIC, p_type=PERIODIC) for _ in range(4)]
    return p, sides


def batched_instances(count: int = 64, seed: int = 2409, max_modulus: float = 2.5, max_coupling: float = 4.0):
    """Seeded uneven instances: side uniform in {64,128,256,512} cells, lambda, mu
    log-uniform [0.1, 10], alpha U[0.5, 1], c0 log-U[1e-3, 1], kappa log-U[1e-3, 1],
    a partial top load on a seeded interval of length >= 1/8, fixed MG(3,4),
    L = log2(N) - 2 levels, FP32.

    The pseudo-time multigrid of the method diverges when the lattice P-wave
    modulus c0 (lambda + 2 mu) exceeds about 3, and the coupled scheme when
    alpha^2 / (c0 (lambda + 2 mu)) is large (checked with the FP64 oracle), so
    draws with c0 (lambda + 2 mu) > max_modulus or alpha^2 / (c0 (lambda + 2 mu))
    > max_coupling are drawn again.  The time step gives a lattice permeability
    kappa dt / (c0 h^2) = 1 (the diffusive scaling dt ~ h^2 of the paper)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = int(rng.choice([64, 128, 256, 512]))
        lam = float(10 ** rng.uniform(-1, 1))
        mu = float(10 ** rng.uniform(-1, 1))
        alpha = float(rng.uniform(0.5, 1.0))
        c0 = float(10 ** rng.uniform(-3, 0))
        kappa = float(10 ** rng.uniform(-3, 0))
        a = float(rng.uniform(0.0, 7.0 / 8.0))
        b = float(rng.uniform(a + 1.0 / 8.0, 1.0))
        modulus = c0 * (lam + 2.0 * mu)
        if modulus > max_modulus or alpha * alpha / modulus > max_coupling:
            continue
        h = 1.0 / n
        x = np.arange(2 * n + 1) * h / 2.0
        load = np.where((x > a) & (x < b), 1.0, 0.0)
        p = _params(n, lam=lam, mu=mu, alpha=alpha, c0=c0, kappa=kappa, dt=c0 * h * h / kappa,
                    levels=int(np.log2(n)) - 2, ne_fixed=3, precision=FP32)
        out.append((p, top_load_sides(n, load)))
    return out


def served_requests(count: int = 200, seed: int = 11382, mean_in_flight: float = 8.0,
                    mean_service_s: float = 0.05, sizes=(64, 128, 256, 512, 1024), steps: int = 100,
                    T: float = 0.1):
    """Seeded Poisson request stream: ``count`` consolidation solves with side
    uniform in ``sizes`` cells (65..1025 nodes), the material values and
    boundary conditions of the 4097x4097 Terzaghi case (lambda = mu = 1,
    alpha = 1, c0 = 0.1, kappa = 1e-2), each to T in ``steps`` steps with fixed
    MG(3,4) and L = log2(N) - 2 levels, FP32.  Inter-arrival times are
    exponential with mean mean_service_s / mean_in_flight.  Returns a list of
    (arrival_s, params, sides, T)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(mean_service_s / mean_in_flight))
        n = int(rng.choice(list(sizes)))
        p = _params(n, lam=1.0, mu=1.0, alpha=1.0, c0=0.1, kappa=1e-2, dt=T / steps,
                    levels=int(np.log2(n)) - 2, ne_fixed=3, precision=FP32)
        out.append((t, p, top_load_sides(n, uniform_load(n)), T))
    return out


def loading_2d(n: int = 128, precision=FP64, ne_fixed=3, K=4):
    """The dimensional two-dimensional loading problem of §4.3: domain (0,100)^2,
    Young's modulus E = 1e5 and Poisson ratio nu = 0.9 in plane stress, so
    lambda = E nu / (1 - nu^2) = 9e6/19 and mu = E / (2 (1 + nu)) = 5e5/19;
    c0 = 1e-6, kappa = 1e-9, alpha = 1, centered coupling, no body force or
    source, zero initial data.  Top: p = 0 and traction
    (0, -1e4 (1 - cos((x + 25) pi / 50))); bottom: fixed displacement, no flow;
    left and right periodic.  Final time 2e6 in N_T = n^2 steps (the paper's
    n = 128, N_T = 16384), MG(3,4) on log2(n) levels as in the paper's own
    experiments.  Returns (params, sides, steps)."""
    lx = 100.0
    p = _params(n, lam=9e6 / 19.0, mu=5e5 / 19.0, alpha=1.0, c0=1e-6, kappa=1e-9,
                dt=2e6 / (n * n), levels=int(np.log2(n)), K=K, ne_fixed=ne_fixed,
                precision=precision, lx=lx)
    x = np.arange(2 * n + 1) * (lx / n) / 2.0
    load = 1e4 * (1.0 - np.cos((x + 25.0) * np.pi / 50.0))
    return p, top_load_sides(n, load, PERIODIC), n * n


def alg1(params: dict, ne: int) -> dict:
    """Alg. 1 -- pseudo-time stepping without multigrid -- as a parameter set:
    one level, no under-relaxation (gamma = 1, so each sweep is one
    ELASTIC_STEP), ne pseudo-time steps per time step (one cycle of ne/2 + ne/2
    sweeps; ne even)."""
    if ne < 2 or ne % 2:
        raise ValueError("ne must be even and >= 2")
    return dict(params, levels=1, gamma=1.0, K=ne // 2, ne_fixed=1)
