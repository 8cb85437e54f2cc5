"""Segments (BIOT_OPT_SEGMENTS): the sweeps of the small coarse levels of a
V-cycle (every level of at most 16 tiles, from the coarsest up) run as one
thread-block-cluster launch per run of sweeps of one storage type, instead of
one launch per sweep.  The per-cell code and every argument are those of the
separate launches, so the results are bitwise the same, with fewer launches.
Covered: the FP32 path (FP64 or FP32 coarsest level, deviation store), the FP64
path, the tolerance mode (ghost moments kept, the V-cycle loop in a graph WHILE
node) and batches (one cluster per instance in each segment launch).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def run(params, sides, steps):
    with biot.Solver(params, sides) as s:
        assert s.step(steps) in (biot.OK, biot.ERR_NOT_CONVERGED)
        return dict(eta=s.read_u()[0], p=s.read_p()[0], sigma=s.read_stress(), st=s.stats())


def cases():
    out = {}
    p, s, _ = W.terzaghi_4097(n=512)                                   # FP32, 7 levels, FP64 8^2
    out["fp32_512"] = (p, s, 3)
    out["fp32_512_coarsest_fp32"] = (dict(p, options=biot.OPT_COARSEST_STORAGE), s, 3)
    out["fp32dev16_512"] = (dict(p, precision=W.FP32_DEV16), s, 3)
    p, s, _ = W.step_load_257(alpha=0.8, precision=W.FP32, n=128)
    out["fp32_step_load_128"] = (dict(p, c0=0.1), s, 4)
    p, s, _ = W.terzaghi_33()                                          # FP64, tolerance mode
    out["fp64_terzaghi_33_tolerance"] = (p, s, 5)
    out["fp64_terzaghi_33_fixed"] = (dict(p, ne_fixed=3), s, 5)
    p, s, _ = W.terzaghi_33(precision=W.FP32)                          # FP32, tolerance mode
    out["fp32_terzaghi_33_tolerance"] = (p, s, 5)
    return out


CASES = cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_segments_bitwise_equal_to_separate_sweeps(name):
    params, sides, steps = CASES[name]
    sep = run(params, sides, steps)
    seg = run(dict(params, options=params.get("options", 0) | biot.OPT_SEGMENTS), sides, steps)
    for k in ("eta", "p", "sigma"):
        assert np.array_equal(seg[k], sep[k]), (name, k)
    assert seg["st"]["total_cycles"] == sep["st"]["total_cycles"]
    assert seg["st"]["kernel_launches"] < sep["st"]["kernel_launches"], name


def test_segments_fp64_match_oracle():
    """The FP64 path with segments against the oracle (1e-12, as every FP64 parity test)."""
    params, sides, _ = W.terzaghi_33()
    params = dict(params, ne_fixed=3, options=biot.OPT_SEGMENTS)
    g = run(params, sides, 5)
    o = O.Oracle(params, sides)
    assert o.step(5) == 0
    for k, f in (("eta", o.read_u), ("p", o.read_p)):
        ref = f()[0]
        assert np.abs(g[k] - ref).max() <= 1e-12 * np.abs(ref).max(), k
    o.close()


def batch_problems():
    probs = W.batched_instances(count=10, seed=5)
    p, s, _ = W.terzaghi_33()
    probs.append((dict(p, ne_fixed=3), s))                             # an FP64 instance
    return probs


def test_batch_segments_bitwise_equal_to_separate_sweeps():
    probs = batch_problems()
    seg_probs = [(dict(p, options=p.get("options", 0) | biot.OPT_SEGMENTS), s) for p, s in probs]
    out = []
    for pr in (seg_probs, probs):
        with biot.Batch(pr) as b:
            assert b.step(2) == biot.OK
            assert b.step(2) == biot.OK
            out.append(([(b[i].read_u()[0], b[i].read_p()[0]) for i in range(len(b))], b.stats()))
    (seg, st_seg), (sep, st_sep) = out
    for i in range(len(probs)):
        assert np.array_equal(seg[i][0], sep[i][0]), i
        assert np.array_equal(seg[i][1], sep[i][1]), i
    assert st_seg["launches_per_step"] < st_sep["launches_per_step"]


def test_served_segments_equal_solo_runs():
    """A server whose requests take segments: the reused executable step graphs
    (cudaGraphExecUpdate) carry the cluster launches, and every result equals
    the request solved alone with separate launches, bitwise."""
    import time
    reqs = W.served_requests(count=6, seed=3, sizes=(64, 128), steps=8, T=0.008)
    reqs = [(a, dict(p, options=p.get("options", 0) | biot.OPT_SEGMENTS), s, T) for a, p, s, T in reqs]
    budget = sum(biot.estimate_bytes(p, s) for _, p, s, _ in reqs[:3])
    with biot.Server(budget, max_resident=3) as srv:
        ids = []
        t0 = time.perf_counter()
        for arrival, p, s, T in reqs:
            while time.perf_counter() - t0 < arrival * 0.2:
                time.sleep(0.0005)
            ids.append(srv.submit(p, s, T))
        for rid in ids:
            assert srv.wait(rid, timeout=300) == biot.OK
        results = [srv.fetch(rid) for rid in ids]
        st = srv.stats()
    assert st["graphs_reused"] >= 1
    for (_, p, s, T), (eta, pr, t) in zip(reqs, results):
        plain = dict(p, options=p["options"] & ~biot.OPT_SEGMENTS)
        with biot.Solver(plain, s) as g:
            g.solve_to(T)
            assert np.array_equal(eta, g.read_u()[0]) and np.array_equal(pr, g.read_p()[0])
