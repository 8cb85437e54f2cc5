"""Closed-form pins of the oracle's elasticity LBM (alpha = 0: no coupling).

Drained linear-elastic states that the lattice must reproduce at every cell
centre: uniaxial compression under a normal traction (eta varies linearly,
sigma uniform), simple shear under a tangential traction, and a rigid shift
prescribed by Dirichlet data.  Each is run with the loaded wall on each of the
four sides, which pins the traction corrections of eq. BC:traction on every
wall (reading R11), the Dirichlet rule of eq. BC:elasticity (reading R2) and
the stress read-out of eqs. displacement / moments:bared, including the c0
scaling of §2.2.
"""
import numpy as np
import pytest

from oracle import oracle as O

P, S, D, N = O.PERIODIC, O.SYMMETRY, O.DIRICHLET, O.NEUMANN
BOTTOM, RIGHT, TOP, LEFT = O.BOTTOM, O.RIGHT, O.TOP, O.LEFT
OPPOSITE = {BOTTOM: TOP, TOP: BOTTOM, LEFT: RIGHT, RIGHT: LEFT}
NORMAL = {BOTTOM: (0, -1), RIGHT: (1, 0), TOP: (0, 1), LEFT: (-1, 0)}


def params(n, lam=1.3, mu=0.45, c0=1.0, **kw):
    p = dict(nx=n, ny=n, lx=1.0, ly=1.0, lam=lam, mu=mu, alpha=0.0, c0=c0, kappa=1.0,
             dt=1.0 / n ** 2, r=0.5, levels=max(1, int(np.log2(n)) - 1), K=4, gamma=0.75,
             tol=1e-14, ne_max=3000, ne_fixed=0)
    p.update(kw)
    return p


def run(p, sides):
    o = O.Oracle(p, sides)
    assert o.step(0) == 0  # elastic solve at t = 0 only
    eta, _ = o.read_u()
    return eta, o.read_stress()


def coords(n):
    c = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c)  # [y][x]
    return X, Y


@pytest.mark.parametrize("wall", [BOTTOM, RIGHT, TOP, LEFT])
@pytest.mark.parametrize("c0", [1.0, 0.1])
def test_uniaxial_compression_each_wall(wall, c0):
    n = 16
    p = params(n, c0=c0)
    lam, mu, s0 = p["lam"], p["mu"], 0.7
    nrm = np.array(NORMAL[wall])
    prof = np.zeros((2, 2 * n + 1))
    prof[:, :] = (-s0 * nrm)[:, None]          # compressive normal traction t = -s0 n
    lateral = S
    sides = [dict(eta_type=lateral, p_type=lateral) for _ in range(4)]
    sides[wall] = dict(eta_type=N, p_type=D, eta_profile=prof)
    sides[OPPOSITE[wall]] = dict(eta_type=D, p_type=N)
    eta, sig = run(p, sides)
    X, Y = coords(n)
    # distance from the fixed wall along the load direction
    axis = 0 if wall in (LEFT, RIGHT) else 1
    s = {RIGHT: X, LEFT: 1 - X, TOP: Y, BOTTOM: 1 - Y}[wall]
    strain = -s0 / (lam + 2 * mu)
    exact = -nrm[axis] * 0 + strain * s * (1 if wall in (RIGHT, TOP) else -1)
    np.testing.assert_allclose(eta[axis], exact, atol=1e-11)
    np.testing.assert_allclose(eta[1 - axis], 0.0, atol=1e-12)
    s_nn = sig[0] if axis == 0 else sig[2]
    s_tt = sig[2] if axis == 0 else sig[0]
    np.testing.assert_allclose(s_nn, -s0, atol=1e-9)
    np.testing.assert_allclose(s_tt, lam * strain, atol=1e-9)
    np.testing.assert_allclose(sig[1], 0.0, atol=1e-9)


@pytest.mark.parametrize("wall", [BOTTOM, RIGHT, TOP, LEFT])
def test_simple_shear_each_wall(wall):
    n = 16
    p = params(n)
    mu, tau = p["mu"], 0.3
    axis = 0 if wall in (LEFT, RIGHT) else 1
    tang = np.array([0, 1]) if axis == 0 else np.array([1, 0])
    prof = np.zeros((2, 2 * n + 1))
    prof[:, :] = (tau * tang)[:, None]
    sides = [dict(eta_type=P, p_type=P) for _ in range(4)]
    sides[wall] = dict(eta_type=N, p_type=D, eta_profile=prof)
    sides[OPPOSITE[wall]] = dict(eta_type=D, p_type=N)
    eta, sig = run(p, sides)
    X, Y = coords(n)
    s = {RIGHT: X, LEFT: 1 - X, TOP: Y, BOTTOM: 1 - Y}[wall]
    sign = 1.0 if wall in (RIGHT, TOP) else -1.0
    # sigma_12 = t . tangent * (n . axis sign); displacement grows away from the fixed wall
    s12 = tau * sign
    np.testing.assert_allclose(sig[1], s12, atol=1e-9)
    np.testing.assert_allclose(eta[1 - axis], tau * s / mu, atol=1e-10)
    np.testing.assert_allclose(eta[axis], 0.0, atol=1e-12)


@pytest.mark.parametrize("wall", [BOTTOM, RIGHT, TOP, LEFT])
def test_dirichlet_shift_each_wall(wall):
    n = 8
    p = params(n)
    a, b = 0.2, -0.1
    prof = np.zeros((2, 2 * n + 1))
    prof[0], prof[1] = a, b
    sides = [dict(eta_type=P, p_type=P) for _ in range(4)]
    sides[wall] = dict(eta_type=D, p_type=N, eta_profile=prof)
    sides[OPPOSITE[wall]] = dict(eta_type=N, p_type=D)
    eta, sig = run(p, sides)
    np.testing.assert_allclose(eta[0], a, atol=1e-10)
    np.testing.assert_allclose(eta[1], b, atol=1e-10)
    np.testing.assert_allclose(sig, 0.0, atol=1e-8)


def test_lattice_independence_of_domain_scaling():
    """The same physical problem on a domain of size 3 scales as the closed form."""
    n = 16
    p = params(n, lx=3.0, ly=3.0, c0=0.5)
    lam, mu, s0 = p["lam"], p["mu"], 1.1
    prof = np.zeros((2, 2 * n + 1))
    prof[1] = -s0
    sides = [dict(eta_type=D, p_type=N), dict(eta_type=S, p_type=S),
             dict(eta_type=N, p_type=D, eta_profile=prof), dict(eta_type=S, p_type=S)]
    eta, sig = run(p, sides)
    y = (np.arange(n) + 0.5) / n * 3.0
    np.testing.assert_allclose(eta[1], (-s0 * y / (lam + 2 * mu))[:, None] * np.ones((1, n)), atol=1e-10)
    np.testing.assert_allclose(sig[2], -s0, atol=1e-9)
