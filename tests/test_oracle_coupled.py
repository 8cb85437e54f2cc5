"""Pins of the oracle's coupled scheme (Alg. 5) against the paper's problems.

* Terzaghi's consolidation problem (§4.2) against its series solution: first
  order in dx with dt = dx^2/4, MG(3,4), centered coupling -- as §4.2 reports;
* the periodic manufactured solution (§4.1): second order with MG(3,2) at
  alpha = 0.5, and displacement errors about twice the pressure errors;
* the stability behaviour of §4.1 with MG(4,2): explicit coupling (r = 0)
  diverges at alpha = 0.6, implicit (r = 1) at alpha = 0.8, centered (r = 1/2)
  converges at alpha = 1;
* roller (mirror) side walls give the periodic result for a problem that does
  not depend on x (reading R12);
* Alg. 1 (pseudo-time stepping without multigrid) with N_E = 1.5 N_x pseudo
  steps converges at almost second order on the manufactured problem (§4.1),
  and far too few pseudo steps leave the elasticity error dominant;
* the dimensional two-dimensional loading problem (§4.3): parameters as
  printed, and the behaviour the paper describes for its solution.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_11382_gb300 import workloads as W
from paper_checks import check_loading_2d_statements, loading_2d_snapshots

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PI = np.pi


def test_paper_parameter_values():
    """Plane-stress Lame values and p0 = 1 as printed in §4.1 / §4.2."""
    g = json.load(open(os.path.join(GOLD, "paper_parameters.json")))
    for key, lam_s, mu_s in (("periodic", 11 / 45, 11 / 360), ("terzaghi", 20 / 9, 5 / 18)):
        E, nu = g[key]["E"], g[key]["nu"]
        assert abs(E * nu / (1 - nu ** 2) - lam_s) < 1e-14
        assert abs(E / (2 * (1 + nu)) - mu_s) < 1e-14
    for alpha in (0.8, 0.9, 1.0):
        p, _, varpi = W.paper_terzaghi(8, alpha)
        assert abs(p["lam"] - 20 / 9) < 1e-15 and abs(p["mu"] - 5 / 18) < 1e-15
        assert abs(alpha * varpi / (p["lam"] + 2 * p["mu"] + alpha ** 2) - g["terzaghi"]["p0"]) < 1e-14


def terzaghi_series(x2, t, p0, cf, terms=400):
    k = np.arange(terms)[:, None]
    a = (k + 0.5) * PI
    return p0 * np.sum(2 * (-1.0) ** k / a * np.exp(-a ** 2 * cf * t) * np.cos(a * x2[None, :]), axis=0)


def subsidence_series(t, S0, Sinf, cf, terms=400):
    a = (np.arange(terms) + 0.5) * PI
    return Sinf + (S0 - Sinf) * np.sum(2 / a ** 2 * np.exp(-a ** 2 * cf * t))


def terzaghi_errors(n, alpha=1.0, T=0.05):
    p, sides, varpi = W.paper_terzaghi(n, alpha)
    lam, mu, kap = p["lam"], p["mu"], p["kappa"]
    p0 = alpha * varpi / (lam + 2 * mu + alpha ** 2)
    cf = (lam + 2 * mu) / (lam + 2 * mu + alpha ** 2) * kap
    S0, Sinf = varpi / (lam + 2 * mu + alpha ** 2), varpi / (lam + 2 * mu)
    o = O.Oracle(p, sides)
    x2 = (np.arange(n) + 0.5) / n
    ep = pn = eS = Sn = 0.0
    for _ in range(int(round(T / p["dt"]))):
        assert o.step(1) == 0
        pp, t = o.read_p()
        eta, _ = o.read_u()
        pe = terzaghi_series(x2, t, p0, cf)
        ep += np.sum((pp - pe[:, None]) ** 2) / n ** 2
        pn += np.sum(pe ** 2) / n
        S = -eta[1, -1].mean()
        Se = subsidence_series(t, S0, Sinf, cf)
        eS += (S - Se) ** 2
        Sn += Se ** 2
    return np.sqrt(ep / pn), np.sqrt(eS / Sn)


def test_terzaghi_first_order():
    errs = [terzaghi_errors(n) for n in (8, 16, 32)]
    ep = np.array([e[0] for e in errs])
    eS = np.array([e[1] for e in errs])
    assert ep[-1] < 0.03 and eS[-1] < 0.03
    assert np.all((ep[:-1] / ep[1:] > 1.7) & (ep[:-1] / ep[1:] < 3.0))
    assert np.all((eS[:-1] / eS[1:] > 1.6) & (eS[:-1] / eS[1:] < 3.0))


def manufactured_errors(n, alpha, r, ne=3, K=2, tf=1.0, alg1_ne=None, extra=None):
    p, sides = W.manufactured_params(n, alpha, r, ne_fixed=ne, K=K)
    if alg1_ne is not None:
        p = W.alg1(p, alg1_ne)
    p = dict(p, **(extra or {}))
    lam, mu, kap = p["lam"], p["mu"], p["kappa"]
    o = O.Oracle(p, sides)
    x = (np.arange(n) + 0.5) / n
    X1, X2 = np.meshgrid(x, x)
    sin_sin = np.sin(2 * PI * X1) * np.sin(2 * PI * X2)

    def sources(t):
        a = (1 - np.exp(-8 * PI ** 2 * kap * t)) / 2
        fb = np.zeros((n, n, 2))
        fb[:, :, 0] = a * 16 * PI ** 2 * mu * np.cos(2 * PI * X1) * np.sin(2 * PI * X2)
        s = -8 * PI ** 3 * kap * (16 * alpha * np.exp(-8 * PI ** 2 * kap * t) + (16 * lam + 30 * mu) / alpha) * sin_sin
        return fb, s

    def exact(t):
        a = (1 - np.exp(-8 * PI ** 2 * kap * t)) / 2
        e = np.array([a * 9 * np.cos(2 * PI * X1) * np.sin(2 * PI * X2),
                      a * 7 * np.sin(2 * PI * X1) * np.cos(2 * PI * X2)])
        return e, -(16 * lam + 30 * mu) * PI / alpha * (1 - np.exp(-8 * PI ** 2 * kap * t)) * sin_sin

    o.set_sources(*sources(0.0))
    ep = pn = ee = en = 0.0
    steps = int(round(tf / p["dt"]))
    for i in range(steps):
        o.set_sources(*sources(i * p["dt"]))
        o.step(1)
        o.set_sources(*sources((i + 1) * p["dt"]))
        pp, t = o.read_p()
        eta, _ = o.read_u()
        if not np.isfinite(pp).all() or np.abs(pp).max() > 1e8:
            return np.inf, np.inf
        e_ex, p_ex = exact(t)
        ep += np.sum((pp - p_ex) ** 2)
        pn += np.sum(p_ex ** 2)
        ee += np.sum((eta - e_ex) ** 2)
        en += np.sum(e_ex ** 2)
    return np.sqrt(ep / pn), np.sqrt(ee / en)


def test_manufactured_second_order_weak_coupling():
    errs = [manufactured_errors(n, 0.5, 0.5, tf=0.25) for n in (8, 16, 32)]
    ep = np.array([e[0] for e in errs])
    ee = np.array([e[1] for e in errs])
    assert np.all(ep[:-1] / ep[1:] > 3.3) and np.all(ee[:-1] / ee[1:] > 3.3)
    # displacement error about twice the pressure error (§4.1)
    assert 1.3 < ee[-1] / ep[-1] < 3.0


@pytest.mark.parametrize("alpha,r,stable", [(0.6, 0.0, False), (0.8, 1.0, False), (1.0, 0.5, True)])
def test_coupling_stability_trio(alpha, r, stable):
    ep, ee = manufactured_errors(16, alpha, r, ne=4, K=2, tf=1.0)
    if stable:
        assert ep < 0.05 and ee < 0.1
    else:
        assert not (ep < 1.0)


def test_roller_sides_equal_periodic_sides_for_x_uniform_problem():
    out = []
    for side_type in (W.SYMMETRY, W.PERIODIC):
        p, sides, _ = W.terzaghi_33(side_type=side_type)
        p = dict(p, nx=16, ny=16, levels=2)
        sides = W.top_load_sides(16, W.uniform_load(16), side_type)
        o = O.Oracle(p, sides)
        o.step(5)
        eta, _ = o.read_u()
        pp, _ = o.read_p()
        out.append((eta, pp, o.read_stress()))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * max(1.0, np.abs(b).max()))


def test_alg1_almost_second_order_and_pseudo_step_starvation():
    """§4.1, Alg. 1 without multigrid: N_E = 1.5 N_x pseudo steps give almost
    second-order convergence (alpha = 0.5, centered coupling); with N_E = 2 at
    N_x = 32 (far below the 0.015 N_x^2 transition) the unconverged elasticity
    dominates the error."""
    g = json.load(open(os.path.join(GOLD, "paper_parameters.json")))["alg1_no_multigrid"]
    errs = [manufactured_errors(n, 0.5, 0.5, tf=0.25, alg1_ne=int(g["NE_over_Nx"] * n)) for n in (8, 16, 32)]
    ep = np.array([e[0] for e in errs])
    ee = np.array([e[1] for e in errs])
    assert np.all(ep[:-1] / ep[1:] > 3.0) and np.all(ee[:-1] / ee[1:] > 3.0)
    starved = manufactured_errors(32, 0.5, 0.5, tf=0.25, alg1_ne=2)
    assert starved[1] > 4 * ee[-1]


def test_alg1_is_the_smoother_at_gamma_one_on_one_level():
    """Alg. 1 as a parameter set: one level, gamma = 1, N_E sweeps in one cycle."""
    p, _ = W.manufactured_params(16, 0.5, 0.5)
    q = W.alg1(p, 24)
    assert (q["levels"], q["gamma"], q["K"], q["ne_fixed"]) == (1, 1.0, 12, 1)
    with pytest.raises(ValueError):
        W.alg1(p, 23)


def test_loading_2d_parameters_as_printed():
    g = json.load(open(os.path.join(GOLD, "paper_parameters.json")))["loading_2d"]
    p, sides, steps = W.loading_2d(g["Nx"])
    E, nu = g["E"], g["nu"]
    assert np.isclose(p["lam"], E * nu / (1 - nu ** 2)) and np.isclose(p["lam"], 9e6 / 19)
    assert np.isclose(p["mu"], E / (2 * (1 + nu))) and np.isclose(p["mu"], 5e5 / 19)
    assert (p["c0"], p["kappa"], p["alpha"], p["r"]) == (g["c0"], g["kappa"], g["alpha"], g["r"])
    assert p["lx"] == g["domain"][1] and steps == g["NT"] and np.isclose(p["dt"] * steps, g["tf"])
    assert (p["ne_fixed"], p["K"]) == (3, 4)
    top = sides[W.TOP]["eta_profile"]
    x = np.arange(2 * g["Nx"] + 1) * (p["lx"] / g["Nx"]) / 2
    assert np.allclose(top[0], 0.0)
    assert np.isclose(top[1][np.argmin(abs(x - 25))], -2 * g["load_amplitude"])  # largest load at x1 = 25
    assert np.isclose(top[1][np.argmin(abs(x - 75))], 0.0, atol=1e-9)            # no load at x1 = 75
    assert sides[W.LEFT]["eta_type"] == W.PERIODIC and sides[W.BOTTOM]["eta_type"] == W.DIRICHLET


def test_loading_2d_statements_oracle():
    n = 32
    check_loading_2d_statements(loading_2d_snapshots(O.Oracle, n), n)
