"""Write the FP64 oracle's reference columns of the 4097x4097 Terzaghi problem.

The problem of the 4097x4097-node benchmark (4096^2 cells, lambda = mu = 1,
alpha = 1, c0 = 0.1, kappa = 1e-2, dt = 1e-3, 10 levels, fixed MG(3,4), top
load 1 at t = 0+, roller sides) does not depend on x: the roller sides are
mirrors, so every column of the lattice carries the same solution.  The oracle
therefore runs a strip of 512 columns -- the narrowest strip whose 10-level
hierarchy still coarsens 2x2 down to one coarse column -- for 100 physical
steps, and this script stores one column of eta and p after steps 1, 10 and
100.  The GPU tests compare every column of the full 4096^2 run against it.

Calls only the oracle (and the seeded input builder of the workloads module):

    python tests/golden/make_terzaghi_4096_strip.py [--threads N]

Output: tests/golden/terzaghi_4096_strip_fp64.npz with
    steps   (3,)          1, 10, 100
    t       (3,)          the time of each state
    eta     (3, 2, 4096)  displacement column (components x rows)
    p       (3, 4096)     pressure column
    spread  (3,)          max over fields of |column x - column 0| in the strip
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2409_11382_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "terzaghi_4096_strip_fp64.npz")
STEPS = (1, 10, 100)
STRIP = 512


def strip_problem():
    params, _, _ = W.terzaghi_4097(precision=W.FP64)
    strip = dict(params, nx=STRIP, lx=STRIP / params["nx"])
    return strip, W.top_load_sides(STRIP, W.uniform_load(STRIP))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    used = O.set_threads(args.threads)
    params, sides = strip_problem()
    o = O.Oracle(params, sides)
    etas, ps, ts, spreads = [], [], [], []
    done = 0
    t0 = time.time()
    for target in STEPS:
        assert o.step(target - done) == 0
        done = target
        eta, t = o.read_u()
        p, _ = o.read_p()
        spread = max(float(np.abs(eta - eta[:, :, :1]).max()), float(np.abs(p - p[:, :1]).max()))
        etas.append(eta[:, :, 0].copy())
        ps.append(p[:, 0].copy())
        ts.append(t)
        spreads.append(spread)
        print(f"step {target}: t = {t:.4g}, column spread {spread:.3g}, "
              f"{time.time() - t0:.0f} s on {used} thread(s)", flush=True)
    o.close()
    np.savez_compressed(OUT, steps=np.array(STEPS), t=np.array(ts), eta=np.array(etas), p=np.array(ps),
                        spread=np.array(spreads))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
