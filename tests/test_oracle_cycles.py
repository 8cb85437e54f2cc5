"""Pins of the oracle's multigrid cycle variants and of the central-difference
pressure gradient -- what the paper leaves to future work (§5: W- and F-cycles,
full multigrid) or describes without results (§3.4,
eq. pressure:gradient:alternative), under the definitions stated beside the
code (readings R20-R22).

* A cycle only changes how the correction problem is approached, not the
  discrete fixed point: W- and F-cycles, and solves that open with a
  full-multigrid cycle, converge to the dense direct solution of the affine
  fixed-point map on 8^2 and 16^2 grids, as the V-cycle does.
* W- and F-cycles solve the coarse correction problem more accurately than a
  V-cycle, so they need no more cycles to reach the tolerance; a full-multigrid
  first cycle leaves a smaller residual than a V-cycle from the same start.
* The central difference of eq. pressure:gradient:alternative is exact for a
  linear field in the interior, and the coupled scheme with it stays second
  order on the manufactured problem of §4.1 (the paper observes the same order
  for both gradients).
"""
import numpy as np
import pytest

from oracle import oracle as O
from test_oracle_bruteforce import dense_solution, setup
from test_oracle_coupled import manufactured_errors


def cycles_to_converge(o, n, max_cycles=400):
    o.set_g(np.zeros((n, n, 8)))
    res = [o.vcycle(reset_history=True)]
    while res[-1] >= 1e-14 and len(res) < max_cycles:
        res.append(o.vcycle())
    return np.array(res), o.get_g().ravel()


@pytest.mark.parametrize("n,kind", [(8, "roller"), (16, "mixed")])
def test_w_and_f_cycles_converge_to_the_direct_solution(n, kind):
    o, _ = setup(n, kind)
    g_direct, _ = dense_solution(o, n)
    o.close()
    scale = max(np.abs(g_direct).max(), 1.0)
    count = {}
    for cycle in (0, 1, 2):
        o, _ = setup(n, kind, cycle=cycle)
        res, g = cycles_to_converge(o, n)
        o.close()
        assert res[-1] < 1e-14, cycle
        assert np.abs(g - g_direct).max() < 1e-10 * scale, (cycle, np.abs(g - g_direct).max())
        count[cycle] = len(res)
    assert count[1] <= count[0] and count[2] <= count[0], count


@pytest.mark.parametrize("cycle", [0, 1])
def test_full_multigrid_first_cycle(cycle):
    n, kind = 16, "mixed"
    o, _ = setup(n, kind)
    g_direct, _ = dense_solution(o, n)
    o.close()
    first = {}
    for fmg in (0, 1):
        # one cycle of the elastic solve from the zero iterate
        o, _ = setup(n, kind, cycle=cycle, fmg=fmg, ne_max=1)
        assert o.step(0) == -4  # one cycle, tolerance not reached
        first[fmg] = o.stats()["last_res"]
        o.close()
        # the whole solve converges to the direct solution
        o, _ = setup(n, kind, cycle=cycle, fmg=fmg)
        assert o.step(0) == 0
        g = o.get_g().ravel()
        o.close()
        assert np.abs(g - g_direct).max() < 1e-10 * max(np.abs(g_direct).max(), 1.0)
    assert first[1] < first[0], first


def test_central_gradient_is_exact_for_linear_pressure():
    """F~ = c0 h^2 f - alpha h [grad^c P + grad^c s'_exp / 2]: with flow
    populations at rest on a linear P = a x + b y, zero source and zero
    divergence history, the interior F~ is -alpha h (a, b) exactly."""
    n = 16
    p = dict(nx=n, ny=n, lx=1.0, ly=1.0, lam=1.0, mu=0.5, alpha=0.7, c0=0.3, kappa=0.2, dt=0.01, r=0.5,
             levels=2, K=2, gamma=0.75, tol=1e-12, ne_max=50, ne_fixed=0, pgrad=1)
    sides = [dict(eta_type=O.PERIODIC, p_type=O.PERIODIC) for _ in range(4)]
    sides = [dict(eta_type=O.DIRICHLET, p_type=O.NEUMANN), dict(eta_type=O.SYMMETRY, p_type=O.SYMMETRY),
             dict(eta_type=O.NEUMANN, p_type=O.DIRICHLET), dict(eta_type=O.SYMMETRY, p_type=O.SYMMETRY)]
    a, b = 0.013, -0.021
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x)
    P = 0.4 + a * X + b * Y
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    o = O.Oracle(p, sides)
    o.set_f(P[:, :, None] * w[None, None, :])
    o.prepare_elastic()
    # the explicit force is what the elastic solve sees: recover it through the
    # fixed-point map's action on the zero iterate (F~ enters the first moments)
    g0 = o.fixed_point_map(np.zeros((n, n, 8)))
    o.close()
    h = 1.0 / n
    # eq. moments:inverse: the first moments of STEP(0) carry F~ (m*_10 = F), pulled
    # unchanged from the neighbours away from walls: sum over k of c_k g_k
    c8 = np.array([(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], dtype=float)
    m10 = g0 @ c8[:, 0]
    m01 = g0 @ c8[:, 1]
    inner = (slice(3, n - 3), slice(3, n - 3))
    assert np.allclose(m10[inner], -p["alpha"] * h * a, rtol=1e-12, atol=0)
    assert np.allclose(m01[inner], -p["alpha"] * h * b, rtol=1e-12, atol=0)


def test_central_gradient_keeps_second_order():
    errs = [manufactured_errors(n, 0.5, 0.5, tf=0.25, extra={"pgrad": 1}) for n in (8, 16, 32)]
    ep = np.array([e[0] for e in errs])
    ee = np.array([e[1] for e in errs])
    assert np.all(ep[:-1] / ep[1:] > 3.3) and np.all(ee[:-1] / ee[1:] > 3.3), (ep, ee)


@pytest.mark.parametrize("K_level", [[1, 3], [4, 1, 2], [2, 6, 1]])
def test_per_level_sweep_counts_keep_the_fixed_point(K_level):
    """Reading R23: the smoothing counts per level (K_level[j] on the level j
    below the finest, Alg. 4's K elsewhere) change the iteration, not its fixed
    point."""
    n, kind = 16, "mixed"
    o, _ = setup(n, kind)
    g_direct, _ = dense_solution(o, n)
    o.close()
    o, _ = setup(n, kind, K_level=K_level)
    res, g = cycles_to_converge(o, n)
    o.close()
    assert res[-1] < 1e-14
    assert np.abs(g - g_direct).max() < 1e-10 * max(np.abs(g_direct).max(), 1.0)


def test_per_level_sweep_counts_change_the_contraction():
    """More sweeps on the finest level contract the residual faster per cycle;
    K_level = [K] * L is Alg. 4 with K itself (bitwise)."""
    n, kind = 16, "roller"
    out = {}
    for name, extra in (("K2", {}), ("same", {"K_level": [2, 2, 2]}), ("fine6", {"K_level": [6]})):
        o, _ = setup(n, kind, **extra)
        o.set_g(np.zeros((n, n, 8)))
        out[name] = [o.vcycle(reset_history=(k == 0)) for k in range(6)]
        o.close()
    assert out["K2"] == out["same"]
    assert out["fine6"][-1] < out["K2"][-1]
