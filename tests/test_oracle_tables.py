"""Pins of the oracle's lattice tables and single-cell collision (CPU).

The moment map is rebuilt here from its definition (eq. moments:
m_ab = sum_ij i^a j^b g_ij, eq. moments:stress) with the velocities of
Tab. velocities read from tests/golden/, independently of the oracle's code.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append(line.split())
    return rows


def _d2q8_velocities():
    """D2Q8 = the moving velocities of Tab. velocities, in the row order of
    Tab. moments:inverse (10, 01, -10, 0-1, 11, -11, -1-1, 1-1)."""
    rows = _read_table("velocities.txt")
    vel = {(int(r[1]), int(r[2])) for r in rows if r[0] != "0"}
    order = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    assert set(order) == vel
    return order


def moment_matrix():
    """Rows: m_10, m_01, m_11, m_s, m_d, m_12, m_21, m_22 (eqs. moments, moments:stress)."""
    c = _d2q8_velocities()
    def raw(a, b):
        return np.array([float(i ** a * j ** b) for i, j in c])
    m20, m02 = raw(2, 0), raw(0, 2)
    return np.array([raw(1, 0), raw(0, 1), raw(1, 1), m20 + m02, m20 - m02,
                     raw(1, 2), raw(2, 1), raw(2, 2)])


def printed_table():
    rows = _read_table("moments_inverse_table.txt")
    return np.array([[float(v) for v in r[1:]] for r in rows])


def test_velocity_weights_sum_and_isotropy():
    rows = _read_table("velocities.txt")
    w = np.array([float(Fraction(r[3])) for r in rows])
    c = np.array([[int(r[1]), int(r[2])] for r in rows])
    assert abs(w.sum() - 1.0) < 1e-15
    # second-order isotropy: sum w c c^T = c_s^2 I with c_s^2 = 1/3
    assert np.allclose((w[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0), np.eye(2) / 3)


def test_oracle_table_is_printed_table_with_reading_R1():
    """The oracle's table equals the printed one (reading R1 only relabels the
    first two columns as 10, 01)."""
    assert np.array_equal(O.inverse_table(), printed_table())


def test_table_inverts_moment_map_exactly():
    M = moment_matrix()
    T = O.inverse_table()
    assert np.array_equal(M @ T, np.eye(8))
    assert np.array_equal(T @ M, np.eye(8))


def test_printed_header_order_does_not_invert():
    """Taking the printed header (01, 10, ...) literally breaks the inverse, which is
    why the columns are read as (10, 01, ...)."""
    M = moment_matrix()
    T = O.inverse_table()[:, [1, 0, 2, 3, 4, 5, 6, 7]]
    assert not np.allclose(M @ T, np.eye(8))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_collision_in_moment_space(seed):
    """Post-collision moments follow Tab. moments, eqs. moments:halfForce,
    moments:collision, moments:BC and moments:collision:22."""
    rng = np.random.default_rng(seed)
    M = moment_matrix()
    for _ in range(20):
        lam, mu = 10 ** rng.uniform(-2, 1, size=2)
        g = rng.normal(size=8)
        F = rng.normal(size=2)
        gs = O.collide_cell(lam, mu, g, F)
        m, ms = M @ g, M @ gs
        lm = lam + mu
        w_s, w_d = 2 / (3 * lm + 1), 2 / (6 * mu + 1)
        np.testing.assert_allclose(ms[0], m[0] + F[0], atol=1e-13)
        np.testing.assert_allclose(ms[1], m[1] + F[1], atol=1e-13)
        np.testing.assert_allclose(ms[2], (1 - w_d) * m[2], atol=1e-13)
        np.testing.assert_allclose(ms[3], (1 - w_s) * m[3], atol=1e-13)
        np.testing.assert_allclose(ms[4], (1 - w_d) * m[4], atol=1e-13)
        np.testing.assert_allclose(ms[5], (m[0] + F[0] / 2) / 3, atol=1e-13)
        np.testing.assert_allclose(ms[6], (m[1] + F[1] / 2) / 3, atol=1e-13)
        # m_f = m_22 + m_s/(12(lam+mu) - 4) relaxes to 0 with omega_f = 1
        if abs(12 * lm - 4) > 1e-3:
            assert abs(ms[7] + ms[3] / (12 * lm - 4)) < 1e-11 * (1 + abs(ms[3]) / abs(12 * lm - 4))
        np.testing.assert_allclose(ms[7], -m[3] / (12 * lm + 4), atol=1e-13)


def test_moment_22_is_regular_at_lambda_mu_one_third():
    """eq. moments:collision:22 is finite where the m_f definition is singular."""
    gs = O.collide_cell(1.0 / 6, 1.0 / 6, np.arange(1, 9, dtype=float), np.array([0.1, -0.2]))
    assert np.isfinite(gs).all()


def test_bounce_back_weights_match_equilibrium_reading_R2():
    """For the stress-free equilibrium of displacement eta, the populations differ
    across opposite directions by 6 w_ij c_ij . eta with the D2Q9 weights."""
    T = O.inverse_table()
    rng = np.random.default_rng(7)
    rows = _read_table("velocities.txt")
    w9 = {(int(r[1]), int(r[2])): float(Fraction(r[3])) for r in rows}
    c = _d2q8_velocities()
    for _ in range(5):
        eta = rng.normal(size=2)
        m = np.array([eta[0], eta[1], 0, 0, 0, eta[0] / 3, eta[1] / 3, 0])
        g = T @ m
        for k, (i, j) in enumerate(c):
            kb = c.index((-i, -j))
            np.testing.assert_allclose(g[k] - g[kb], 6 * w9[(i, j)] * (i * eta[0] + j * eta[1]), atol=1e-14)


def test_stress_free_displacement_state_is_collision_invariant():
    """A uniform displacement without force is a fixed point of the collision."""
    T = O.inverse_table()
    eta = np.array([0.3, -0.7])
    g = T @ np.array([eta[0], eta[1], 0, 0, 0, eta[0] / 3, eta[1] / 3, 0])
    np.testing.assert_allclose(O.collide_cell(0.5, 0.2, g, np.zeros(2)), g, atol=1e-15)
