"""The paper's test problems on the GPU FP64 path (§4.1, §4.2):

* the periodic manufactured solution converges at second order (weak coupling
  alpha = 0.5, centered scheme, MG(3,2), dt = dx^2);
* the coupling-stability study with MG(4,2): the explicit scheme (r = 0)
  diverges at alpha = 0.6, the implicit one (r = 1) at alpha = 0.8, the
  centered one (r = 1/2) converges at alpha = 1;
* Terzaghi's problem converges at first order to its series solution
  (dt = dx^2/4, MG(3,4), periodic sides).
The exact solutions are the paper's; the time-dependent sources are uploaded
with biot_set_sources every step, as the oracle's tests do."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402

PI = np.pi


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def manufactured_errors(n, alpha, r, ne=3, K=2, tf=1.0):
    p, sides = W.manufactured_params(n, alpha, r, ne_fixed=ne, K=K)
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
