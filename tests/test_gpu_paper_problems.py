"""The paper's test problems on the GPU FP64 path (§4.1, §4.2):

* the periodic manufactured solution converges at second order (weak coupling
  alpha = 0.5, centered scheme, MG(3,2), dt = dx^2);
* the coupling-stability study with MG(4,2): the explicit scheme (r = 0)
  diverges at alpha = 0.6, the implicit one (r = 1) at alpha = 0.8, the
  centered one (r = 1/2) converges at alpha = 1;
* Terzaghi's problem converges at first order to its series solution
  (dt = dx^2/4, MG(3,4), periodic sides);
* Alg. 1 (pseudo-time stepping without multigrid, N_E = 1.5 N_x) matches the
  oracle and converges at almost second order (§4.1);
* the dimensional two-dimensional loading problem (§4.3) matches the oracle
  over its whole time span at 32^2 cells and, at the paper's size (128^2
  cells, 16384 steps), behaves as the paper describes.
The exact solutions are the paper's; the time-dependent sources are uploaded
with biot_set_sources every step, as the oracle's tests do."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402
from paper_checks import check_loading_2d_statements, loading_2d_snapshots  # noqa: E402

PI = np.pi


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def manufactured_errors(n, alpha, r, ne=3, K=2, tf=1.0, alg1_ne=None):
    p, sides = W.manufactured_params(n, alpha, r, ne_fixed=ne, K=K)
    if alg1_ne is not None:
        p = W.alg1(p, alg1_ne)
    lam, mu, kap = p["lam"], p["mu"], p["kappa"]
    x = (np.arange(n) + 0.5) / n
    X1, X2 = np.meshgrid(x, x)
    sin_sin = np.sin(2 * PI * X1) * np.sin(2 * PI * X2)

    def sources(t):
        a = (1 - np.exp(-8 * PI ** 2 * kap * t)) / 2
        fb = np.zeros((2, n, n))
        fb[0] = a * 16 * PI ** 2 * mu * np.cos(2 * PI * X1) * np.sin(2 * PI * X2)
        s = -8 * PI ** 3 * kap * (16 * alpha * np.exp(-8 * PI ** 2 * kap * t) + (16 * lam + 30 * mu) / alpha) * sin_sin
        return fb, s

    def exact(t):
        a = (1 - np.exp(-8 * PI ** 2 * kap * t)) / 2
        e = np.array([a * 9 * np.cos(2 * PI * X1) * np.sin(2 * PI * X2),
                      a * 7 * np.sin(2 * PI * X1) * np.cos(2 * PI * X2)])
        return e, -(16 * lam + 30 * mu) * PI / alpha * (1 - np.exp(-8 * PI ** 2 * kap * t)) * sin_sin

    ep = pn = ee = en = 0.0
    with biot.Solver(p, sides) as g:
        g.set_sources(*sources(0.0))
        for i in range(int(round(tf / p["dt"]))):
            g.set_sources(*sources(i * p["dt"]))
            try:
                g.step(1)
            except biot.BiotError as e:
                assert e.code == biot.ERR_DIVERGED
                return np.inf, np.inf
            g.set_sources(*sources((i + 1) * p["dt"]))
            pp, t = g.read_p()
            eta, _ = g.read_u()
            if not np.isfinite(pp).all() or np.abs(pp).max() > 1e8:
                return np.inf, np.inf
            e_ex, p_ex = exact(t)
            ep += np.sum((pp - p_ex) ** 2)
            pn += np.sum(p_ex ** 2)
            ee += np.sum((eta - e_ex) ** 2)
            en += np.sum(e_ex ** 2)
    return np.sqrt(ep / pn), np.sqrt(ee / en)


def test_manufactured_second_order_on_gpu():
    errs = [manufactured_errors(n, 0.5, 0.5, tf=0.25) for n in (16, 32, 64)]
    ep = np.array([e[0] for e in errs])
    ee = np.array([e[1] for e in errs])
    assert np.all(ep[:-1] / ep[1:] > 3.3) and np.all(ee[:-1] / ee[1:] > 3.3)
    assert 1.3 < ee[-1] / ep[-1] < 3.0  # displacement error about twice the pressure error


@pytest.mark.parametrize("alpha,r,stable", [(0.6, 0.0, False), (0.8, 1.0, False), (1.0, 0.5, True)])
def test_coupling_stability_trio_on_gpu(alpha, r, stable):
    ep, ee = manufactured_errors(16, alpha, r, ne=4, K=2, tf=1.0)
    if stable:
        assert ep < 0.05 and ee < 0.1
    else:
        assert not (ep < 1.0)


def terzaghi_series(x2, t, p0, cf, terms=400):
    k = np.arange(terms)[:, None]
    a = (k + 0.5) * PI
    return p0 * np.sum(2 * (-1.0) ** k / a * np.exp(-a ** 2 * cf * t) * np.cos(a * x2[None, :]), axis=0)


def terzaghi_error(n, alpha=1.0, T=0.05):
    p, sides, varpi = W.paper_terzaghi(n, alpha)
    lam, mu, kap = p["lam"], p["mu"], p["kappa"]
    p0 = alpha * varpi / (lam + 2 * mu + alpha ** 2)
    cf = (lam + 2 * mu) / (lam + 2 * mu + alpha ** 2) * kap
    x2 = (np.arange(n) + 0.5) / n
    ep = pn = 0.0
    with biot.Solver(p, sides) as g:
        for _ in range(int(round(T / p["dt"]))):
            g.step(1)
            pp, t = g.read_p()
            pe = terzaghi_series(x2, t, p0, cf)
            ep += np.sum((pp - pe[:, None]) ** 2) / n ** 2
            pn += np.sum(pe ** 2) / n
    return np.sqrt(ep / pn)


def test_terzaghi_first_order_on_gpu():
    e = np.array([terzaghi_error(n) for n in (16, 32, 64)])
    assert e[-1] < 0.02
    assert np.all((e[:-1] / e[1:] > 1.7) & (e[:-1] / e[1:] < 3.0))


# ---------------------------------------------------------------------------
# Alg. 1 without multigrid (§4.1)
# ---------------------------------------------------------------------------

def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision, tol", [(W.FP64, 1e-12), (W.FP32, 1e-5)])
def test_alg1_matches_oracle(precision, tol):
    """Alg. 1 with N_E = 1.5 N_x = 48 pseudo steps on the 33x33 Terzaghi case
    (one level, gamma = 1): the GPU path against the FP64 oracle after 10 steps."""
    from oracle import oracle as O
    p, sides, _ = W.terzaghi_33(precision=precision)
    p = W.alg1(p, 48)
    with biot.Solver(p, sides) as g:
        g.step(10)
        eta, _ = g.read_u()
        pp, _ = g.read_p()
    ref = O.Oracle(W.alg1(W.terzaghi_33()[0], 48), sides)
    ref.step(10)
    eta_o, _ = ref.read_u()
    p_o, _ = ref.read_p()
    ref.close()
    assert rel(eta, eta_o) < tol and rel(pp, p_o) < tol


def test_alg1_almost_second_order_on_gpu():
    errs = [manufactured_errors(n, 0.5, 0.5, tf=0.25, alg1_ne=int(1.5 * n)) for n in (16, 32, 64)]
    ep = np.array([e[0] for e in errs])
    ee = np.array([e[1] for e in errs])
    assert np.all(ep[:-1] / ep[1:] > 3.0) and np.all(ee[:-1] / ee[1:] > 3.0)


# ---------------------------------------------------------------------------
# Two-dimensional loading problem (§4.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision, tol", [(W.FP64, 1e-12), (W.FP32, 1e-5)])
def test_loading_2d_matches_oracle(precision, tol):
    """32^2 cells, t_f = 2e6 in 1024 steps (the lattice permeability of the
    paper's 128^2 run): eta and p at t = 2e4, 2e5, 2e6 against the oracle."""
    from oracle import oracle as O
    n = 32
    got = loading_2d_snapshots(lambda p, s: biot.Solver(p, s), n, precision)
    ref = loading_2d_snapshots(O.Oracle, n)
    for (t, e, p), (to, eo, po) in zip(got, ref):
        assert t == pytest.approx(to)
        assert rel(e, eo) < tol and rel(p, po) < tol


def test_loading_2d_paper_size_statements():
    """The paper's run: 128^2 cells, 16384 steps to t_f = 2e6, MG(3,4), on the
    FP32 path; the solution behaves as §4.3 describes."""
    n = 128
    check_loading_2d_statements(loading_2d_snapshots(lambda p, s: biot.Solver(p, s), n, W.FP32), n)
