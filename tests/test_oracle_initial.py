"""Pins of the oracle's initial conditions (§3.6, eqs. ICs and ICs:moments).

The paper starts every problem from p = 0 and eta = 0 and chooses the initial
populations so that these physical values hold in the read-outs of
eq. pressure and eq. displacement at t = 0, with a body force f(0) and a
source s(0) present.  The checks below read the oracle's populations before
any elastic solve and evaluate the read-outs from their definitions -- the
moments m_ab = sum_ij i^a j^b g_ij of eqs. moments / moments:stress with the
velocities of Tab. velocities (tests/golden/velocities.txt), not the oracle's
own tables:

  * eta(0) = mbar = m + F/2 = 0 in every cell (eqs. displacement,
    moments:halfForce), with F = eps^2 f_eff(0) = c0 h^2 f(0) the lattice force
    (grad p(0) = 0);
  * sigma(0) = 0: m_s = m_d = m_11 = 0 (eqs. displacement, moments:bared);
  * m_12, m_21 = -F/6 and m_22 = 0, the force-corrected equilibrium of
    eq. ICs:moments;
  * p(0) = sum_i f_i + (dt/2) s(0) = 0 in every cell (eq. pressure), the flow
    populations at rest (zero flux sum_i f_i c_i, f_i proportional to w_i);
  * and, through the public read-out, p at t = 0 is zero when a source acts
    without load (the divergence then stays zero, so s_eff(0) = s(0)).

A wrong sign or coefficient in either initial state, a dropped source or force
term, or swapped components fails one of them.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _velocities():
    rows = []
    for line in open(os.path.join(GOLD, "velocities.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    c9 = np.array([[int(r[1]), int(r[2])] for r in rows])
    w9 = np.array([float(Fraction(r[3])) for r in rows])
    order8 = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    return c9, w9, np.array(order8)


def _moments(g, c8):
    """eqs. moments / moments:stress from the definition, per cell:
    (m_10, m_01, m_11, m_s, m_d, m_12, m_21, m_22)."""
    cx, cy = c8[:, 0].astype(float), c8[:, 1].astype(float)
    raw = lambda a, b: g @ (cx ** a * cy ** b)  # noqa: E731
    m20, m02 = raw(2, 0), raw(0, 2)
    return np.stack([raw(1, 0), raw(0, 1), raw(1, 1), m20 + m02, m20 - m02,
                     raw(1, 2), raw(2, 1), raw(2, 2)], axis=-1)


def _problem(n=16, periodic=True, c0=0.3, dt=0.01, lx=2.0):
    if periodic:
        sides = [dict(eta_type=O.PERIODIC, p_type=O.PERIODIC) for _ in range(4)]
    else:
        sides = [dict(eta_type=O.DIRICHLET, p_type=O.NEUMANN), dict(eta_type=O.SYMMETRY, p_type=O.SYMMETRY),
                 dict(eta_type=O.NEUMANN, p_type=O.DIRICHLET), dict(eta_type=O.SYMMETRY, p_type=O.SYMMETRY)]
    params = dict(nx=n, ny=n, lx=lx, ly=lx, lam=0.7, mu=0.4, alpha=0.9, c0=c0, kappa=0.2, dt=dt, r=0.5,
                  levels=3, K=2, gamma=0.75, tol=1e-12, ne_max=50, ne_fixed=3)
    return params, sides


def _sources(n, seed):
    rng = np.random.default_rng(seed)
    fbody = rng.normal(size=(n, n, 2)) * 3.0   # dimensional body force, 2 per cell
    src = rng.normal(size=(n, n)) + 0.5        # dimensional source
    return fbody, src


@pytest.mark.parametrize("periodic", [True, False])
def test_initial_populations_give_zero_displacement_stress_and_pressure(periodic):
    n = 16
    params, sides = _problem(n, periodic)
    fbody, src = _sources(n, 7 + periodic)
    o = O.Oracle(params, sides)
    o.set_sources(fbody, src)
    o.prepare_elastic()  # initial state; no elastic solve
    g, f = o.get_g(), o.get_f()
    o.close()
    c9, w9, c8 = _velocities()
    h = params["lx"] / n
    F = params["c0"] * h * h * fbody                      # lattice force eps^2 f_eff(0)
    m = _moments(g, c8)
    scale = np.abs(F).max()
    # eta(0) = mbar = m + F/2 = 0
    assert np.abs(m[..., 0:2] + 0.5 * F).max() <= 1e-15 * scale
    assert np.abs(m[..., 0:2]).max() > 0.1 * scale           # the force really enters
    # sigma(0) = 0 and m_22 = 0
    for k in (2, 3, 4, 7):
        assert np.abs(m[..., k]).max() <= 1e-15 * scale
    # m_12, m_21 = -F/6 (force-corrected equilibrium)
    assert np.abs(m[..., 5] + F[..., 0] / 6.0).max() <= 1e-15 * scale
    assert np.abs(m[..., 6] + F[..., 1] / 6.0).max() <= 1e-15 * scale
    # p(0) = sum f + (dt/2) s(0) = 0; the populations at rest with weights w_i
    s0 = params["dt"] * src                                   # lattice source
    total = f.sum(axis=-1)
    assert np.abs(total + 0.5 * s0).max() <= 1e-15 * np.abs(s0).max()
    assert np.abs(f @ c9.astype(float)).max() <= 1e-15 * np.abs(s0).max()
    assert np.abs(f - total[..., None] * w9).max() <= 1e-15 * np.abs(s0).max()


def test_pressure_read_at_t0_is_zero_with_source_and_no_load():
    """Through the public read-out: a uniform source s(0) with no load or body
    force gives no force (no flux, no source gradient), so the elastic solve at
    t = 0 leaves eta = 0 and the divergence zero, and p(0) = sum f + (dt/2) s(0)
    must vanish."""
    n = 16
    params, sides = _problem(n, periodic=False)
    src = np.full((n, n), 1.7)
    o = O.Oracle(params, sides)
    o.set_sources(None, src)
    p, t = o.read_p()
    eta, _ = o.read_u()
    o.close()
    assert t == 0.0
    assert np.abs(eta).max() == 0.0
    assert np.abs(p).max() <= 1e-15 * params["dt"] * np.abs(src).max() / params["c0"]


def test_dropping_the_flow_initial_state_is_detected():
    """The same read-out from populations set to zero (the initial state of
    eq. ICs left out) gives p(0) = (dt/2) s(0) / c0, not zero."""
    n = 16
    params, sides = _problem(n, periodic=False)
    src = np.full((n, n), 1.7)
    o = O.Oracle(params, sides)
    o.set_sources(None, src)
    o.set_f(np.zeros((n, n, 9)))
    p, _ = o.read_p()
    o.close()
    expect = 0.5 * params["dt"] * src / params["c0"]
    assert np.abs(p - expect).max() <= 1e-14 * np.abs(expect).max()
