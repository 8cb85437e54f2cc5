"""The FP64 cold start of the FP32 path: the solve at t = 0 (three V-cycles from
a zero iterate) runs on an FP64 copy of the problem and its state is narrowed
into the FP32 instance (moments rounded to FP32, the first moments as
double-float).  By default this applies from 2048^2 cells; the environment
variable BIOT_COLD_FP64_MIN_CELLS = 0 applies it to every grid, so the checks
run in a child process on a small grid:

* the handed-over state at t = 0 is the FP64 path's state to FP32 rounding;
* the following FP32 steps stay within 1e-5 of the FP64 oracle;
* a served request, whose FP64 copy the server admits within its memory
  budget, gives bitwise the result of the same request solved alone."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2409_11382_gb300 import biot, workloads as W
from oracle import oracle as O

def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())

n, steps = 64, 6
p64, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP64, n=n)
p64 = dict(p64, c0=0.1)
p32 = dict(p64, precision=W.FP32)
out = {}
with biot.Solver(p64, sides) as s:
    e64, _ = s.read_u()
    s.read_p()
with biot.Solver(p32, sides) as s:
    e32, _ = s.read_u()                       # the solve at t = 0 on the FP64 copy
    out["t0_eta"] = rel(e32, e64)
    s.step(steps)
    eta, _ = s.read_u()
    pp, _ = s.read_p()
ref = O.Oracle(p64, sides)
ref.step(steps)
out["eta"] = rel(eta, ref.read_u()[0])
out["p"] = rel(pp, ref.read_p()[0])
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
out["served_equal"] = bool(np.array_equal(eta_s, solo[0]) and np.array_equal(p_s, solo[1]))
out["peak_ok"] = bool(st["peak_bytes"] <= budget)
print(json.dumps(out))
"""


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()


def test_fp64_cold_start_handover_steps_and_serving():
    env = dict(os.environ, BIOT_COLD_FP64_MIN_CELLS="0")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["t0_eta"] < 1e-6
    assert res["eta"] < 1e-5 and res["p"] < 1e-5
    assert res["served_equal"] and res["peak_ok"]
