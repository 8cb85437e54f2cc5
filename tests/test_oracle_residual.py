"""Pin of the oracle's residual norms (the stopping test of the adaptive
variant, §3.4, and its 2-norm companion).

On one level (no coarse correction) with K = 1, a V-cycle of Alg. 4 is one
smoothing sweep g1 = (1 - gamma) g0 + gamma ELASTIC_STEP(g0) (eq. MG:smoother)
followed by one more, whose start g1 is the iterate the residual is measured
on.  With periodic sides the fullway bounce-back history plays no part, so
the residual r = g1 - ELASTIC_STEP(g1) follows from the oracle's fixed-point
map alone; its max-norm and 2-norm over every population of every cell must be
the ones the V-cycle reports.
"""
import numpy as np

from oracle import oracle as O


def test_vcycle_residual_norms_match_the_fixed_point_map():
    n = 16
    p = dict(nx=n, ny=n, lx=1.0, ly=1.0, lam=0.9, mu=0.5, alpha=0.8, c0=0.4, kappa=0.2, dt=0.01, r=0.5,
             levels=1, K=1, gamma=0.75, tol=1e-14, ne_max=10, ne_fixed=0)
    sides = [dict(eta_type=O.PERIODIC, p_type=O.PERIODIC) for _ in range(4)]
    rng = np.random.default_rng(5)
    o = O.Oracle(p, sides)
    o.set_f(0.01 * rng.normal(size=(n, n, 9)))
    o.prepare_elastic()
    g0 = 0.1 * rng.normal(size=(n, n, 8))
    g1 = 0.25 * g0 + 0.75 * o.fixed_point_map(g0)
    r = g1 - o.fixed_point_map(g1)
    o.set_g(g0)
    res = o.vcycle(reset_history=True)
    st = o.stats()
    o.close()
    assert np.abs(r).max() > 0
    assert abs(res - np.abs(r).max()) <= 1e-14 * np.abs(r).max()
    assert abs(st["last_res"] - res) == 0.0
    assert abs(st["last_res_l2"] - np.linalg.norm(r.ravel())) <= 1e-13 * np.linalg.norm(r.ravel())
    # the two norms bound each other: max <= l2 <= sqrt(8 n^2) max
    assert res <= st["last_res_l2"] <= np.sqrt(8 * n * n) * res
