"""Brute-force pin of the oracle's multigrid (Alg. 4) on tiny grids.

The fixed point of ELASTIC_STEP with the self-dependent force,
g = ELASTIC_STEP(g, F~ + F_*(g)), is an affine map g = A g + b.  Here it is
assembled column by column from the oracle's fixed-point map and solved
directly with LAPACK.  The V-cycles must converge to the same populations
(any error in the restriction, prolongation or coarse operator would change the
convergence but could not move the fixed point, so the test also demands that
every V-cycle reduces the residual).
"""
import numpy as np
import pytest

from oracle import oracle as O

P, S, D, N = O.PERIODIC, O.SYMMETRY, O.DIRICHLET, O.NEUMANN


def setup(n, sides_kind, alpha=1.0, r=0.5, c0=0.3, seed=0, **extra):
    p = dict(nx=n, ny=n, lx=1.0, ly=1.0, lam=1.0, mu=0.5, alpha=alpha, c0=c0, kappa=0.2,
             dt=0.01, r=r, levels=int(np.log2(n)) - 1, K=2, gamma=0.75, tol=1e-14,
             ne_max=2000, ne_fixed=0)
    p.update(extra)
    rng = np.random.default_rng(seed)
    prof = np.zeros((2, 2 * n + 1))
    prof[0] = 0.2 * rng.normal(size=2 * n + 1)
    prof[1] = -1.0 + 0.1 * rng.normal(size=2 * n + 1)
    if sides_kind == "roller":
        sides = [dict(eta_type=D, p_type=N), dict(eta_type=S, p_type=S),
                 dict(eta_type=N, p_type=D, eta_profile=prof), dict(eta_type=S, p_type=S)]
    else:
        bot = np.zeros((2, 2 * n + 1))
        bot[0] = 0.05
        sides = [dict(eta_type=D, p_type=N, eta_profile=bot), dict(eta_type=D, p_type=N),
                 dict(eta_type=N, p_type=D, eta_profile=prof), dict(eta_type=N, p_type=N)]
    o = O.Oracle(p, sides)
    # a non-trivial explicit force: random flow populations and divergence history
    o.set_f(0.01 * rng.normal(size=(n, n, 9)))
    o.prepare_elastic()
    return o, n


def dense_solution(o, n):
    m = 8 * n * n
    b = o.fixed_point_map(np.zeros((n, n, 8))).ravel()
    A = np.empty((m, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        A[:, j] = o.fixed_point_map(e.reshape(n, n, 8)).ravel() - b
    return np.linalg.solve(np.eye(m) - A, b), A


@pytest.mark.parametrize("n,kind", [(8, "roller"), (8, "mixed"), (16, "roller")])
def test_vcycles_converge_to_direct_solution(n, kind):
    o, n = setup(n, kind)
    g_direct, A = dense_solution(o, n)
    assert np.linalg.cond(np.eye(A.shape[0]) - A) < 1e8
    o.set_g(np.zeros((n, n, 8)))
    res = [o.vcycle(reset_history=True)]
    for _ in range(400):
        res.append(o.vcycle())
        if res[-1] < 1e-14:
            break
    res = np.array(res)
    # every V-cycle contracts after the first few (fullway history warm-up)
    assert np.all(res[5:] / res[4:-1] < 1.0)
    g = o.get_g().ravel()
    scale = np.abs(g_direct).max()
    assert np.abs(g - g_direct).max() < 1e-10 * max(scale, 1.0)


def test_fixed_point_map_is_affine_consistent():
    """Superposition check of the assembled map (guards the dense assembly itself)."""
    o, n = setup(8, "roller", seed=3)
    rng = np.random.default_rng(1)
    b = o.fixed_point_map(np.zeros((n, n, 8)))
    x, y = rng.normal(size=(n, n, 8)), rng.normal(size=(n, n, 8))
    lhs = o.fixed_point_map(x + 2 * y) - b
    rhs = (o.fixed_point_map(x) - b) + 2 * (o.fixed_point_map(y) - b)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
