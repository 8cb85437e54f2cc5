"""GPU test of biot_read_u_noalloc, the displacement read-out that allocates no
device memory.

Callers that cannot allocate when they read results (device memory already
handed to another allocator, or a loop that must not take cudaMalloc's implicit
synchronisation) use this entry point; it stages the values in a static array
of the library instead of the instance's lazily allocated read-out buffer.  It
must return what biot_read_u returns.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402

TOL64 = 1e-12  # the FP64 parity tolerance of the other GPU tests
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_read_u_noalloc_matches_read_u_on_consecutive_calls(precision):
    params, sides, _ = W.step_load_257(alpha=1.0, precision=precision, n=64)
    params = dict(params, c0=0.1)
    tol = TOL64 if precision == W.FP64 else TOL32
    with biot.Solver(params, sides) as s:
        s.step(3)
        first, t1 = s.read_u_noalloc()      # first call on this device sets the array up
        second, t2 = s.read_u_noalloc()     # second call in a row: same state, same values
        ref, t0 = s.read_u()
        assert t0 == t1 == t2
        assert np.isfinite(first).all() and np.abs(ref).max() > 0
        assert rel(first, ref) <= tol and rel(second, ref) <= tol
        s.step(2)                           # new state: the array is overwritten, not stale
        third, _ = s.read_u_noalloc()
        fourth, _ = s.read_u_noalloc()
        ref2, _ = s.read_u()
        assert rel(third, ref2) <= tol and rel(fourth, ref2) <= tol
        assert rel(third, ref) > tol


def test_read_u_noalloc_rejects_grids_beyond_the_static_array():
    n = 1024  # 1024^2 cells > BIOT_NOALLOC_MAX_CELLS
    assert n * n > biot.NOALLOC_MAX_CELLS
    params, sides, _ = W.terzaghi_4097(n=n)
    with biot.Solver(params, sides) as s:
        with pytest.raises(biot.BiotError) as e:
            s.read_u_noalloc()
        assert e.value.code == biot.ERR_INVALID_ARG
        assert "static read-out array" in str(e.value)
