"""Checks of the paper's problems shared by the oracle's and the GPU path's tests
(test helpers only: the solver class under test is passed in)."""
import json
import os

import numpy as np

from paper_2409_11382_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def loading_2d_snapshots(solver_cls, n, precision=W.FP64):
    """(t, eta, p) at the paper's three snapshot times t = 2e4, 2e5, 2e6."""
    g = json.load(open(os.path.join(GOLD, "paper_parameters.json")))["loading_2d"]
    p, sides, steps = W.loading_2d(n, precision=precision)
    marks = [int(round(t / p["dt"])) for t in g["snapshot_times"]]
    out = []
    s = solver_cls(p, sides)
    done = 0
    for m in marks:
        s.step(m - done)
        done = m
        eta, t = s.read_u()
        pp, _ = s.read_p()
        out.append((t, eta, pp))
    s.close()
    return out


def check_loading_2d_statements(snaps, n):
    """§4.3's description of the solution: the heavily loaded left half subsides
    while the surface on the right is lifted; the material expands horizontally
    from the left half to the right one; early on the pressure is large below
    the left half of the surface and low below the right half; the pressure
    decays over time and the whole surface subsides further."""
    x = (np.arange(n) + 0.5) * 100.0 / n
    i25, i50, i75 = (int(np.argmin(abs(x - v))) for v in (25.0, 50.0, 75.0))
    depth = n - 1 - int(round(5.0 * n / 100.0))  # about 5 units below the surface
    (t1, e1, p1), (t2, e2, p2), (t3, e3, p3) = snaps
    for _, e, p in snaps:
        assert np.isfinite(e).all() and np.isfinite(p).all()
    top1 = e1[:, -1, :]
    assert top1[1, i25] < 0.0 < top1[1, i75]
    assert abs(x[int(np.argmin(top1[1]))] - 25.0) < 12.5
    assert e1[0, :, i50].mean() > 0.0  # net horizontal displacement across x1 = 50 (left to right)
    assert p1[depth, i25] > 2.0 * p1[depth, i75]
    assert p1.max() > p2.max() > p3.max()
    assert e3[1, -1, :].mean() < e2[1, -1, :].mean() < top1[1].mean()
