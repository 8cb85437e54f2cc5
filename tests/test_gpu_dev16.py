"""The 16-bit deviation store of the FP32 path (BIOT_FP32_DEV16, _DEVBF16):
the finest level's m_11, m_s, m_d -- the deviation of the elastic state from
its equilibrium, whose values for these moments are zero (Tab. moments) --
stored as FP16 or BF16 values times a power of two, collided in FP32.

Checked against the FP64 oracle on the same seeded inputs (relative L-infinity
of eta and p): the 33^2 Terzaghi problem over its 50 steps, the 257^2 step load
after 40 steps, and one instance of every size of the 64-instance batch.  The
bounds are the measured accuracy of each storage with a margin (FP16 keeps 11
significant bits, BF16 8): DEV_TOL below -- measured about 5e-5 (eta) and 3e-4
(p) with FP16, 5e-4 and 2.3e-3 with BF16, against 4e-8 and 7e-7 for FP32
storage on the 257^2 step load.  The pressure error comes mostly through the
divergence D = kD m_s of the coupling.  A checkpoint resumes bitwise, and a
batched instance agrees with its solo run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402

DEVS = {"fp16": W.FP32_DEV16, "bf16": W.FP32_DEVBF16}
DEV_TOL = {"fp16": 1e-3, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def both(params, sides, steps):
    with biot.Solver(params, sides) as s:
        s.step(steps)
        g = (s.read_u()[0], s.read_p()[0])
    o = O.Oracle(dict(params, precision=W.FP64), sides)
    o.step(steps)
    r = (o.read_u()[0], o.read_p()[0])
    o.close()
    return rel(g[0], r[0]), rel(g[1], r[1])


@pytest.mark.parametrize("dev", sorted(DEVS))
def test_dev_store_terzaghi_33_and_step_load_257(dev):
    p, s, steps = W.terzaghi_33(precision=DEVS[dev])
    e1 = both(dict(p, ne_fixed=3), s, steps)
    p, s, _ = W.step_load_257(alpha=1.0, precision=DEVS[dev])
    e2 = both(dict(p, c0=0.1), s, 40)
    p32, s32, _ = W.step_load_257(alpha=1.0, precision=W.FP32)
    e32 = both(dict(p32, c0=0.1), s32, 40)
    print(f"\n{dev}: terzaghi_33 eta/p {e1[0]:.3g}/{e1[1]:.3g}; step_load_257 eta/p {e2[0]:.3g}/{e2[1]:.3g} "
          f"(fp32 {e32[0]:.3g}/{e32[1]:.3g})")
    assert max(e1 + e2) < DEV_TOL[dev], (e1, e2)


@pytest.mark.parametrize("dev", sorted(DEVS))
def test_dev_store_batched_64_instances(dev):
    probs = [(dict(p, precision=DEVS[dev]), s) for p, s in W.batched_instances(count=64, seed=2409)]
    steps = 4
    with biot.Batch(probs) as b:
        b.step(steps)
        out = [(b[i].read_u()[0], b[i].read_p()[0]) for i in range(len(b))]
    for eta, p in out:
        assert np.isfinite(eta).all() and np.isfinite(p).all()
    first = {}
    for i, (params, _) in enumerate(probs):
        first.setdefault(params["nx"], i)
    errs = {}
    for n, i in sorted(first.items()):
        params, sides = probs[i]
        with biot.Solver(params, sides) as s:          # the same instance alone
            s.step(steps)
            solo = (s.read_u()[0], s.read_p()[0])
        # the batch's strip / tile forms may round FP32 differently from the solo
        # run's, and a 16-bit store can turn that into one unit of its own rounding
        assert rel(out[i][0], solo[0]) < DEV_TOL[dev] and rel(out[i][1], solo[1]) < DEV_TOL[dev], n
        o = O.Oracle(dict(params, precision=W.FP64), sides)
        o.step(steps)
        errs[n] = (rel(out[i][0], o.read_u()[0]), rel(out[i][1], o.read_p()[0]))
        o.close()
    print(f"\n{dev} batch vs oracle:", {n: (f"{a:.3g}", f"{b:.3g}") for n, (a, b) in errs.items()})
    assert max(max(e) for e in errs.values()) < DEV_TOL[dev], errs


def test_dev_store_checkpoint_resume_is_bitwise():
    params, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP32_DEV16, n=64)
    params = dict(params, c0=0.1)
    with biot.Solver(params, sides) as a:
        a.step(4)
        blob = a.save()
        a.step(3)
        ref = (a.read_u()[0], a.read_p()[0])
    with biot.Solver(params, sides) as b:
        b.load(blob)
        b.step(3)
        got = (b.read_u()[0], b.read_p()[0])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_dev_store_needs_fixed_cycles():
    p, s, _ = W.terzaghi_33(precision=W.FP32_DEV16)  # tolerance mode
    with pytest.raises(biot.BiotError) as e:
        biot.Solver(p, s)
    assert e.value.code == biot.ERR_INVALID_ARG
