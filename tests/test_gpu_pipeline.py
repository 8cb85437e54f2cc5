"""GPU tests of the pipelined entry points: biot_step_async / biot_sync,
biot_set_side_profile without waiting, and their batch forms.

* A loop that changes the top load every step and never waits (set profile,
  step_async, read_async) gives, step for step, bitwise the fields of the
  same loop run with biot_step and synchronous reads.
* biot_sync reports what biot_step would have: BIOT_ERR_NOT_CONVERGED for a
  tolerance-mode step that hit ne_max, once.
* The batch forms equal biot_batch_step.
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


def loads(n, steps):
    """A different top traction profile for every step (2 x (2n+1) samples)."""
    rng = np.random.default_rng(7)
    out = []
    for _ in range(steps):
        prof = np.zeros((2, 2 * n + 1))
        prof[1] = -(0.5 + rng.random()) * np.ones(2 * n + 1)
        out.append(prof)
    return out


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_pipelined_loop_equals_synchronous_loop(precision):
    params, sides, _ = W.terzaghi_4097(n=64, precision=precision)
    n, steps = params["nx"], 4
    profs = loads(n, steps)
    outs = [(pinned((2, n, n)), pinned((n, n))) for _ in range(steps)]
    with biot.Solver(params, sides) as a:
        for k in range(steps):
            a.set_side_profile(W.TOP, profs[k], None)
            a.step_async(1)
            a.read_async(eta=outs[k][0], p=outs[k][1])
        assert a.sync() == biot.OK
    with biot.Solver(params, sides) as b:
        for k in range(steps):
            b.set_side_profile(W.TOP, profs[k], None)
            b.step(1)
            assert np.array_equal(outs[k][0], b.read_u()[0]), f"eta, step {k}"
            assert np.array_equal(outs[k][1], b.read_p()[0]), f"p, step {k}"


def test_sync_reports_not_converged_once():
    params, sides, _ = W.terzaghi_4097(n=32, precision=W.FP64)
    params = dict(params, ne_fixed=0, ne_max=1, tol=1e-30)  # every step stops at ne_max
    with biot.Solver(params, sides) as s:
        s.step_async(2)
        assert s.sync() == biot.ERR_NOT_CONVERGED
        assert s.sync() == biot.OK           # nothing new since the last report
        assert s.stats()["notconv_steps"] >= 2


def test_batch_step_async_equals_batch_step():
    probs = W.batched_instances(count=3, seed=3)
    with biot.Batch(probs) as a, biot.Batch(probs) as b:
        a.step_async(2)
        assert a.sync() == biot.OK
        b.step(2)
        for i in range(len(a)):
            assert np.array_equal(a[i].read_u()[0], b[i].read_u()[0])
            assert np.array_equal(a[i].read_p()[0], b[i].read_p()[0])
