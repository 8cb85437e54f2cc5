"""The oracle's spread under a reordering of its FP64 sums, shared by the CPU
pin (test_oracle_rounding.py) and the FP64 GPU parity test at 1024 rows.

The same oracle source, compiled so that the compiler may reorder FP64 sums
(the oracle's "reassociated" build flavour), gives another, equally valid
rounding of the same scheme.  The problem is the x-independent Terzaghi
problem of the 4097x4097 benchmark on a strip of columns (roller sides make
every column equal)."""
import numpy as np

from oracle import oracle as O
from paper_2409_11382_gb300 import workloads as W


def strip(n, cols):
    """The n x n benchmark problem (log2(n) - 2 levels, FP64) on a strip of
    `cols` columns, the narrowest width its hierarchy coarsens to one column."""
    p, _, _ = W.terzaghi_4097(n=n, precision=W.FP64)
    return dict(p, nx=cols, lx=cols / n), W.top_load_sides(cols, W.uniform_load(cols))


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def oracle_fields(params, sides, steps, flavour="standard"):
    o = O.Oracle(params, sides, flavour=flavour)
    assert o.step(steps) == 0
    out = (o.read_u()[0], o.read_p()[0])
    o.close()
    return out


def rounding_spread(params, sides, steps=1):
    """Relative L-infinity difference of eta and p (the larger) between the two
    builds, and the standard build's fields."""
    std = oracle_fields(params, sides, steps)
    alt = oracle_fields(params, sides, steps, "reassociated")
    return max(rel(alt[k], std[k]) for k in (0, 1)), std
