"""GPU tests of biot_read_async / biot_read_wait, the read-out whose host copy
overlaps the following steps.

* Fields issued after step k and waited for after steps k+1, k+2 are bitwise
  the fields biot_read_u / biot_read_p / biot_read_stress return at step k on a
  second instance of the same problem (same kernels, same state).
* A third read in flight reuses the first one's device staging buffer only
  after that buffer's copy is done.
* Asking for the stress grows the staging buffers; a batch instance reads the
  same way; bad calls are rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def pinned(shape):
    return torch.full(shape, np.nan, dtype=torch.float64, pin_memory=True).numpy()


def problem(precision, n=64):
    params, sides, _ = W.step_load_257(alpha=1.0, precision=precision, n=n)
    return dict(params, c0=0.1), sides


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_reads_in_flight_across_steps_equal_synchronous_reads(precision):
    params, sides = problem(precision)
    n = params["nx"]
    outs = [(pinned((2, n, n)), pinned((n, n))) for _ in range(3)]
    times = []
    with biot.Solver(params, sides) as a:
        for eta, p in outs:  # three reads in flight, one per step; nothing waits in between
            a.step(1)
            times.append(a.read_async(eta=eta, p=p))
        a.read_wait()
    with biot.Solver(params, sides) as b:
        for k, (eta, p) in enumerate(outs):
            b.step(1)
            ref_eta, t = b.read_u()
            ref_p, _ = b.read_p()
            assert t == times[k]
            assert np.array_equal(eta, ref_eta) and np.array_equal(p, ref_p), f"read {k}"
    assert not np.array_equal(outs[0][1], outs[2][1])


def test_stress_read_grows_the_staging_buffers():
    params, sides = problem(W.FP32)
    n = params["nx"]
    p_only, eta = pinned((n, n)), pinned((2, n, n))
    sig, p2 = pinned((3, n, n)), pinned((n, n))
    with biot.Solver(params, sides) as s:
        s.step(2)
        s.read_async(p=p_only)               # 3-plane staging buffer
        s.read_async(eta=eta)                # the other slot
        s.read_async(p=p2, sigma=sig)        # back to the first slot, grown to 6 planes
        s.read_wait()
        s.read_wait()                        # nothing in flight: still fine
        ref_sig = s.read_stress()
        ref_p, _ = s.read_p()
        ref_eta, _ = s.read_u()
    assert np.array_equal(sig, ref_sig)
    assert np.array_equal(p_only, ref_p) and np.array_equal(p2, ref_p)
    assert np.array_equal(eta, ref_eta)


def test_batch_instance_reads_asynchronously():
    probs = W.batched_instances(count=3, seed=11)
    with biot.Batch(probs) as b:
        b.step(2)
        outs = []
        for i in range(len(b)):
            p, _ = probs[i]
            eta, pr = pinned((2, p["ny"], p["nx"])), pinned((p["ny"], p["nx"]))
            b[i].read_async(eta=eta, p=pr)
            outs.append((eta, pr))
        for i in range(len(b)):
            b[i].read_wait()
        for i, (eta, pr) in enumerate(outs):
            assert np.array_equal(eta, b[i].read_u()[0]) and np.array_equal(pr, b[i].read_p()[0])


def test_bad_calls_are_rejected():
    params, sides = problem(W.FP64, n=16)
    with biot.Solver(params, sides) as s:
        with pytest.raises(biot.BiotError):
            s.read_async()                   # no output at all
        with pytest.raises(ValueError):
            s.read_async(p=np.zeros((16, 8)))
        s.read_wait()                        # no read issued yet


def test_batch_read_async_equals_instance_reads():
    probs = W.batched_instances(count=4, seed=5)
    with biot.Batch(probs) as b:
        b.step(1)
        etas = [pinned((2, p["ny"], p["nx"])) for p, _ in probs]
        ps = [pinned((p["ny"], p["nx"])) for p, _ in probs]
        ps[2] = None                         # skip one field of one instance
        t = b.read_async(eta=etas, p=ps)
        b.step(1)                            # runs while the copies are in flight
        b.read_wait()
        assert np.array_equal(t, [p["dt"] for p, _ in probs])  # one step taken before the read
        with biot.Batch(probs) as ref:
            ref.step(1)
            for i in range(len(ref)):
                assert np.array_equal(etas[i], ref[i].read_u()[0])
                if ps[i] is not None:
                    assert np.array_equal(ps[i], ref[i].read_p()[0])
