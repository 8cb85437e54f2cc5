"""Serving (biot_server_*): requests that arrive while others run are admitted
as memory and slots free up, their steps overlap on the GPU, and each result is
the same as the request solved alone (same kernels and arguments: bitwise) and
within the FP32 tolerance (1e-5 relative L-infinity of eta and p) of the FP64
oracle -- checked for one request of every size in the mix."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402

TOL32 = 1e-5


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def alone(params, sides, T):
    with biot.Solver(params, sides) as s:
        s.solve_to(T)
        return s.read_u(), s.read_p()[0]


def test_served_results_equal_solo_runs_and_overlap():
    reqs = W.served_requests(count=8, seed=5, sizes=(64, 128, 256), steps=12, T=0.012)
    budget = sum(biot.estimate_bytes(p, s) for _, p, s, _ in reqs[:3])
    with biot.Server(budget, max_resident=4) as srv:
        ids = []
        t0 = time.perf_counter()
        for arrival, p, s, T in reqs:
            while time.perf_counter() - t0 < arrival * 0.2:
                time.sleep(0.0005)
            ids.append(srv.submit(p, s, T))
        for rid in ids:
            assert srv.wait(rid, timeout=300) == biot.OK
        infos = [srv.poll(rid) for rid in ids]
        results = [srv.fetch(rid) for rid in ids]
        st = srv.stats()
    assert st["peak_resident"] >= 2            # requests were resident together
    assert st["graphs_reused"] >= 1             # a finished request's step graphs served a later one
    assert st["peak_bytes"] <= budget           # admission kept to the budget
    for info in infos:
        assert info["state"] == biot.REQ_DONE
        assert info["t_submit"] <= info["t_start"] <= info["t_done"]
    for (arrival, p, s, T), (eta, pr, t) in zip(reqs, results):
        (eta_a, t_a), p_a = alone(p, s, T)
        assert t == pytest.approx(t_a)
        assert np.array_equal(eta, eta_a) and np.array_equal(pr, p_a)
    # one served result of every size against the FP64 oracle
    seen = set()
    for (arrival, p, s, T), (eta, pr, t) in zip(reqs, results):
        if p["nx"] in seen:
            continue
        seen.add(p["nx"])
        o = O.Oracle(dict(p, precision=W.FP64), s)
        o.solve_to(T)
        eta_o, t_o = o.read_u()
        p_o, _ = o.read_p()
        o.close()
        assert t == pytest.approx(t_o)
        assert rel(eta, eta_o) < TOL32 and rel(pr, p_o) < TOL32, (p["nx"], rel(eta, eta_o), rel(pr, p_o))
    assert len(seen) >= 2


def test_request_larger_than_budget_is_rejected():
    _, p, s, T = W.served_requests(count=1, seed=1, sizes=(256,), steps=2, T=0.002)[0]
    with biot.Server(1 << 20, max_resident=2) as srv:
        with pytest.raises(biot.BiotError) as e:
            srv.submit(p, s, T)
        assert e.value.code == biot.ERR_OOM


def test_estimate_matches_allocation():
    _, p, s, T = W.served_requests(count=1, seed=2, sizes=(128,), steps=2, T=0.002)[0]
    est = biot.estimate_bytes(p, s)
    with biot.Solver(p, s) as sol:
        sol.step(1)
        sol.read_u()
        held = sol.stats()["device_bytes"]
    assert held == est
