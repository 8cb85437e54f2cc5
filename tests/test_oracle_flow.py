"""Pins of the oracle's flow LBM (Alg. 3) with the coupling switched off (alpha = 0).

* mass balance: the collision of eq. pressure:collision with the source of
  eq. pressure:collision:source adds exactly s' = dt s per cell, and periodic,
  bounce-back and mirror walls conserve the rest;
* diffusion: a cosine mode decays like exp(-kappa k^2 t), with the
  second-order convergence of the SRT diffusion LBM (relation eq. pressure:rate);
* halfway anti-bounce-back (eq. BC:pressure) and bounce-back (eq. BC:noFlow)
  reproduce linear / constant steady states exactly.
"""
import numpy as np
import pytest

from oracle import oracle as O

P, S, D, N = O.PERIODIC, O.SYMMETRY, O.DIRICHLET, O.NEUMANN
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def params(n, **kw):
    p = dict(nx=n, ny=n, lx=1.0, ly=1.0, lam=1.0, mu=0.5, alpha=0.0, c0=1.0, kappa=0.1,
             dt=1.0 / n ** 2, r=0.5, levels=1, K=1, gamma=0.75, tol=1e-12, ne_max=100, ne_fixed=1)
    p.update(kw)
    return p


@pytest.mark.parametrize("walls", ["periodic", "mixed"])
def test_mass_balance_is_exact(walls):
    rng = np.random.default_rng(3)
    n = 8
    if walls == "periodic":
        sides = [dict(eta_type=P, p_type=P)] * 4
    else:
        sides = [dict(eta_type=D, p_type=N), dict(eta_type=S, p_type=S),
                 dict(eta_type=N, p_type=N), dict(eta_type=S, p_type=S)]
    p = params(n)
    o = O.Oracle(p, sides)
    o.set_f(rng.random((n, n, 9)))
    s = rng.normal(size=(n, n))
    o.set_sources(None, s)
    for _ in range(3):
        m0 = o.get_f().sum()
        o.step(1)
        m1 = o.get_f().sum()
        assert abs((m1 - m0) - p["dt"] * s.sum()) < 1e-12


def test_diffusion_mode_decays_at_second_order():
    errs = []
    for n in (8, 16, 32):
        p = params(n)
        o = O.Oracle(p, [dict(eta_type=P, p_type=P)] * 4)
        x = (np.arange(n) + 0.5) / n
        X, _ = np.meshgrid(x, x)
        p0 = np.cos(2 * np.pi * X)
        o.set_f(p0[:, :, None] * W9[None, None, :])
        o.step(int(round(0.2 / p["dt"])))
        pp, t = o.read_p()
        exact = np.exp(-4 * np.pi ** 2 * p["kappa"] * t) * p0
        errs.append(np.abs(pp - exact).max() / np.abs(exact).max())
    assert errs[-1] < 5e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a / b < 4.4


def test_dirichlet_pressure_gives_exact_linear_profile():
    n = 8
    p = params(n, kappa=1.0 / 6)  # omega = 1
    top = np.ones(2 * n + 1)
    sides = [dict(eta_type=D, p_type=D), dict(eta_type=P, p_type=P),
             dict(eta_type=N, p_type=D, p_profile=top), dict(eta_type=P, p_type=P)]
    o = O.Oracle(p, sides)
    o.step(3000)
    pp, _ = o.read_p()
    y = (np.arange(n) + 0.5) / n
    np.testing.assert_allclose(pp, np.broadcast_to(y[:, None], pp.shape), atol=1e-12)


def test_no_flow_wall_keeps_dirichlet_value():
    n = 8
    p = params(n, kappa=1.0 / 6, c0=0.5)
    top = np.full(2 * n + 1, 0.8)
    sides = [dict(eta_type=D, p_type=N), dict(eta_type=S, p_type=S),
             dict(eta_type=N, p_type=D, p_profile=top), dict(eta_type=S, p_type=S)]
    o = O.Oracle(p, sides)
    o.step(4000)
    pp, _ = o.read_p()
    np.testing.assert_allclose(pp, 0.8, atol=1e-11)
