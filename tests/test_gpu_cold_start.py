"""The FP64 cold start of the FP32 path: the solve at t = 0 (three V-cycles from
a zero iterate) runs on an FP64 copy of the problem and its state is narrowed
into the FP32 instance (moments rounded to FP32, the first moments as
double-float).  By default this applies from 2048^2 cells; the option
BIOT_OPT_COLD_FP64 applies it to every grid, so the checks run on a small grid:

* the handed-over state at t = 0 is the FP64 path's state to FP32 rounding;
* the following FP32 steps stay within 1e-5 of the FP64 oracle;
* a served request, whose FP64 copy the server admits within its memory
  budget, gives bitwise the result of the same request solved alone;
* BIOT_OPT_COLD_FP32 keeps the solve at t = 0 on the FP32 path (a different
  rounding, the same tolerance)."""
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


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_fp64_cold_start_handover_steps_and_serving():
    n, steps = 64, 6
    p64, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP64, n=n)
    p64 = dict(p64, c0=0.1)
    p32 = dict(p64, precision=W.FP32, options=biot.OPT_COLD_FP64)
    with biot.Solver(p64, sides) as s:
        e64, _ = s.read_u()
    with biot.Solver(p32, sides) as s:
        e32, _ = s.read_u()                       # the solve at t = 0 on the FP64 copy
        assert rel(e32, e64) < 1e-6
        s.step(steps)
        eta, _ = s.read_u()
        pp, _ = s.read_p()
    ref = O.Oracle(p64, sides)
    ref.step(steps)
    assert rel(eta, ref.read_u()[0]) < 1e-5
    assert rel(pp, ref.read_p()[0]) < 1e-5
    ref.close()
    T = steps * p32["dt"]
    with biot.Solver(p32, sides) as s:
        s.solve_to(T)
        solo = (s.read_u()[0], s.read_p()[0])
    budget = biot.estimate_bytes(p32, sides) + biot.estimate_bytes(p64, sides)
    with biot.Server(budget, max_resident=2) as srv:
        rid = srv.submit(p32, sides, T)
        assert srv.wait(rid, timeout=300) == biot.OK
        eta_s, p_s, _ = srv.fetch(rid)
        st = srv.stats()
    assert np.array_equal(eta_s, solo[0]) and np.array_equal(p_s, solo[1])
    assert st["peak_bytes"] <= budget


def test_fp32_cold_start_option():
    n, steps = 64, 6
    p64, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP64, n=n)
    p64 = dict(p64, c0=0.1)
    out = {}
    for name, opt in (("fp64", biot.OPT_COLD_FP64), ("fp32", biot.OPT_COLD_FP32)):
        with biot.Solver(dict(p64, precision=W.FP32, options=opt), sides) as s:
            s.step(steps)
            out[name] = (s.read_u()[0], s.read_p()[0])
    ref = O.Oracle(p64, sides)
    ref.step(steps)
    eta_o, p_o = ref.read_u()[0], ref.read_p()[0]
    ref.close()
    for name in out:
        assert rel(out[name][0], eta_o) < 1e-5 and rel(out[name][1], p_o) < 1e-5, name
    assert not np.array_equal(out["fp64"][1], out["fp32"][1])  # different cold starts, different rounding


def test_conflicting_options_are_rejected():
    p, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP32, n=64)
    for opt in (biot.OPT_COLD_FP64 | biot.OPT_COLD_FP32, biot.OPT_COARSE_LO_ALL | biot.OPT_COARSE_LO_OFF, 1 << 10):
        with pytest.raises(biot.BiotError) as e:
            biot.Solver(dict(p, options=opt), sides)
        assert e.value.code == biot.ERR_INVALID_ARG
