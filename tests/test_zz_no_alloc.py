"""GPU test of biot_read_u_noalloc, the displacement read-out that allocates no
device memory.

Callers that cannot allocate when they read results (device memory already
handed to another allocator, or a loop that must not take cudaMalloc's implicit
synchronisation) use this entry point; it stages the values in a static array
of the library instead of the instance's lazily allocated read-out buffer.  It
must return bitwise what biot_read_u returns (the same read-out kernel) and
leave the device's free memory unchanged.  This file is collected last so that a
run stopping at the first failure has already run every other test.
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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(0)[0]


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_read_u_noalloc_matches_read_u_on_consecutive_calls(precision):
    """Both entry points run the same read-out kernel, so the values are
    bitwise equal; after the first call (the array's address is looked up),
    a call leaves the device's free memory unchanged."""
    params, sides, _ = W.step_load_257(alpha=1.0, precision=precision, n=64)
    params = dict(params, c0=0.1)
    with biot.Solver(params, sides) as s:
        s.step(3)
        ref, t0 = s.read_u()
        first, t1 = s.read_u_noalloc()      # first call on this device sets the array up
        free0 = free_bytes()
        second, t2 = s.read_u_noalloc()     # second call in a row: same state, same values
        assert free_bytes() == free0
        assert t0 == t1 == t2
        assert np.isfinite(first).all() and np.abs(ref).max() > 0
        assert np.array_equal(first, ref) and np.array_equal(second, ref)
        s.step(2)                           # new state: the array is overwritten, not stale
        ref2, _ = s.read_u()
        free1 = free_bytes()
        third, _ = s.read_u_noalloc()
        fourth, _ = s.read_u_noalloc()
        assert free_bytes() == free1
        assert np.array_equal(third, ref2) and np.array_equal(fourth, ref2)
        assert not np.array_equal(third, ref)


def test_read_u_noalloc_refuses_the_allocating_fp64_cold_start():
    """An FP32 instance whose solve at t = 0 runs on an FP64 copy (which
    biot_create allocates) is refused until that solve has run."""
    params, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP32, n=64)
    params = dict(params, c0=0.1, options=biot.OPT_COLD_FP64)
    with biot.Solver(params, sides) as s:
        with pytest.raises(biot.BiotError) as e:
            s.read_u_noalloc()
        assert e.value.code == biot.ERR_INVALID_ARG
        s.step(1)
        ref, _ = s.read_u()
        got, _ = s.read_u_noalloc()
        assert np.array_equal(got, ref)


def test_read_u_noalloc_rejects_grids_beyond_the_static_array():
    n = 1024  # 1024^2 cells > BIOT_NOALLOC_MAX_CELLS
    assert n * n > biot.NOALLOC_MAX_CELLS
    params, sides, _ = W.terzaghi_4097(n=n)
    with biot.Solver(params, sides) as s:
        with pytest.raises(biot.BiotError) as e:
            s.read_u_noalloc()
        assert e.value.code == biot.ERR_INVALID_ARG
        assert "static read-out array" in str(e.value)
