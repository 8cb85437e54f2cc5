"""Batched execution (biot_batch_*): many uneven instances advanced by work-list
launches that span instances and multigrid levels, one CUDA graph per step.

Each instance runs the same sweeps with the same arguments as when stepped
alone.  A level may take another kernel form in the batch (the batch runs
levels above 128^2 as strips, a single instance levels above 256^2), but the
forms share the per-cell arithmetic, whose every rounding the source fixes
(explicit fused multiply-adds and separately rounded products, so no
contraction choice of the compiler can differ between them): results are
bitwise those of the instance alone, FP32 and FP64.  Sampled instances are also
checked against the FP64 oracle (1e-12 FP64, 1e-5 FP32).
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


TOL32 = 1e-5


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def mixed_problems():
    out = []
    p, s, _ = W.step_load_257(alpha=0.8, precision=W.FP32, n=64)
    out.append((dict(p, c0=0.1), s))
    p, s, _ = W.terzaghi_4097(n=128)
    out.append((p, s))
    p, s, _ = W.terzaghi_33()
    out.append((dict(p, ne_fixed=3), s))                      # FP64, 3 levels
    out += W.batched_instances(count=3, seed=7)                # random materials and loads
    p, s, _ = W.step_load_257(alpha=0.5, precision=W.FP32, n=256)
    out.append((dict(p, c0=0.1, ny=128, ly=0.5), s))          # rectangle
    return out


def alone(params, sides, steps):
    with biot.Solver(params, sides) as s:
        s.step(steps)
        return s.read_u()[0], s.read_p()[0], s.stats()


def test_batch_equals_each_instance_alone_bitwise():
    probs = mixed_problems()
    steps = 5
    with biot.Batch(probs) as b:
        assert b.step(2) == biot.OK
        assert b.step(3) == biot.OK
        got = [(b[i].read_u()[0], b[i].read_p()[0], b[i].stats()) for i in range(len(b))]
        st = b.stats()
    assert st["launches_per_step"] > 0 and st["work_items_per_step"] > 0
    for i, (params, sides) in enumerate(probs):
        eta, p, stats = alone(params, sides, steps)
        assert np.array_equal(got[i][0], eta), (i, rel(got[i][0], eta))
        assert np.array_equal(got[i][1], p), (i, rel(got[i][1], p))
        assert got[i][2]["nstep"] == stats["nstep"] == steps
        assert got[i][2]["total_cycles"] == stats["total_cycles"]


def test_batch_matches_oracle():
    p64, s64, _ = W.terzaghi_33()
    p64 = dict(p64, ne_fixed=3)
    p32, s32, _ = W.step_load_257(alpha=1.0, precision=W.FP32, n=64)
    p32 = dict(p32, c0=0.1)
    steps = 4
    with biot.Batch([(p64, s64), (p32, s32)]) as b:
        b.step(steps)
        res = [(b[i].read_u()[0], b[i].read_p()[0]) for i in range(2)]
    for (params, sides), (eta, p), tol in zip([(p64, s64), (p32, s32)], res, (1e-12, 1e-5)):
        o = O.Oracle(params, sides)
        o.step(steps)
        assert rel(eta, o.read_u()[0]) < tol
        assert rel(p, o.read_p()[0]) < tol
        o.close()


def test_batched_workload_64_instances():
    """The 64-instance workload (sides 64..512, seeded materials and loads): every
    instance finite and bitwise equal to its solo run; one instance of every size
    (the first of each) within the FP32 tolerance of the FP64 oracle."""
    probs = W.batched_instances(count=64, seed=2409)
    steps = 4
    with biot.Batch(probs) as b:
        b.step(steps)
        out = [(b[i].read_u()[0], b[i].read_p()[0]) for i in range(len(b))]
    for eta, p in out:
        assert np.isfinite(eta).all() and np.isfinite(p).all()
    first = {}
    for i, (params, _) in enumerate(probs):
        first.setdefault(params["nx"], i)
    assert sorted(first) == [64, 128, 256, 512]
    # every instance against its solo run
    for i, (params, sides) in enumerate(probs):
        eta, p, _ = alone(params, sides, steps)
        assert np.array_equal(out[i][0], eta) and np.array_equal(out[i][1], p), (i, rel(out[i][0], eta))
    for i in first.values():
        params, sides = probs[i]
        o = O.Oracle(dict(params, precision=W.FP64), sides)
        o.step(steps)
        assert rel(out[i][0], o.read_u()[0]) < 1e-5
        assert rel(out[i][1], o.read_p()[0]) < 1e-5
        o.close()


def test_equal_sized_instances_with_own_walls_equal_solo_runs():
    """Instances of one size share every phase launch of a batch, each with its
    own materials and boundary conditions (symmetric and periodic sides; a
    512-column level ends in a part-filled strip), beside a 512 x 128 rectangle
    of another depth: each equals its solo run bitwise and the FP64 oracle
    within the FP32 tolerance."""
    probs = []
    for k, (alpha, c0, side) in enumerate([(1.0, 0.01, W.SYMMETRY), (0.7, 0.05, W.PERIODIC),
                                           (0.9, 0.1, W.SYMMETRY), (0.8, 0.02, W.PERIODIC)]):
        p, _, _ = W.step_load_257(alpha=alpha, precision=W.FP32, n=512)
        probs.append((dict(p, c0=c0), W.top_load_sides(512, W.step_load(512), side)))
    p, _, _ = W.step_load_257(alpha=0.6, precision=W.FP32, n=512)
    probs.append((dict(p, ny=128, ly=0.25, c0=0.03, levels=6), W.top_load_sides(512, W.step_load(512))))
    steps = 3
    with biot.Batch(probs) as b:
        assert b.step(steps) == biot.OK
        out = [(b[i].read_u()[0], b[i].read_p()[0]) for i in range(len(b))]
    for i, (params, sides) in enumerate(probs):
        eta, p, _ = alone(params, sides, steps)
        assert np.array_equal(out[i][0], eta) and np.array_equal(out[i][1], p), (i, rel(out[i][0], eta))
    for i in (1, 4):
        params, sides = probs[i]
        o = O.Oracle(dict(params, precision=W.FP64), sides)
        o.step(steps)
        assert rel(out[i][0], o.read_u()[0]) < 1e-5, i
        assert rel(out[i][1], o.read_p()[0]) < 1e-5, i
        o.close()


def test_batch_rejects_mixed_cycle_counts():
    p1, s1, _ = W.terzaghi_33(precision=W.FP32)
    with pytest.raises(biot.BiotError) as e:
        biot.Batch([(dict(p1, ne_fixed=3), s1), (dict(p1, ne_fixed=2), s1)])
    assert e.value.code == biot.ERR_INVALID_ARG
