"""The algorithmic byte model of bench.py (host arithmetic, no GPU): the finest
smoothing sweep's bytes per cell, written out by hand, and the step total as
the sum over levels of the per-sweep counts the model documents."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2409_11382_gb300 import workloads as W  # noqa: E402


def test_step_model_terzaghi_4096_fp32():
    p, _, _ = W.terzaghi_4097()
    n, L, K, ne = 4096, p["levels"], p["K"], p["ne_fixed"]
    sweeps, nb = bench.step_model(p, n, fp64=False)
    # cell-sweeps: ne V-cycles of (2K + 1) sweeps per level above the coarsest, 2K there
    cells = [float((n >> (L - 1 - l)) ** 2) for l in range(L)]
    expect_sweeps = ne * (sum((2 * K + 1) * c for c in cells[1:]) + 2 * K * cells[0])
    assert sweeps == pytest.approx(expect_sweeps)
    # finest smoothing: 5 moments + 2 low parts in and out, F~ in (FP32), plus the
    # correction from the 2048^2 level (5 FP32 moments per 4 cells) once per 2K sweeps
    finest = ((5 + 2) * 2 + 2) * 4 + 5 * 4 / 4 / (2 * K)
    assert finest == pytest.approx(64.625)
    fine = cells[-1]
    restrict_fine = (5 + 2 + 2) * 4 + 5 * 4 / 4
    coarse = 0.0
    for l in range(L - 1):  # coarse levels in FP32, the coarsest (l = 0) in FP64
        e = 8 if l == 0 else 4
        ec = 8 if l == 1 else 4  # the storage of the next coarser level (prolongation, restriction)
        prol = 5 * ec / 4 / (2 * K) if l > 0 else 0.0
        coarse += ne * 2 * K * cells[l] * ((5 * 2 + 5) * e + prol)
        if l > 0:
            coarse += ne * cells[l] * ((5 + 5) * e + 5 * ec / 4)
    # flow: 9 f in and out, m_s, D(t - dt) (FP64), previous difference in;
    # D(t) (FP64), new difference, F~ (2) out
    flow = fine * (9 * 4 * 2 + 4 + 8 + 4 + 8 + 4 + 2 * 4)
    assert flow / fine == 108
    expect = ne * 2 * K * fine * finest + ne * fine * restrict_fine + coarse + flow
    assert nb == pytest.approx(expect)
    assert nb / fine == pytest.approx(2312, abs=1.0)


def test_step_model_follows_the_coarsest_precision_option():
    p, _, _ = W.terzaghi_4097()
    _, nb64 = bench.step_model(p, 4096, fp64=False)
    _, nb32 = bench.step_model(dict(p, options=bench.OPT_COARSEST_STORAGE), 4096, fp64=False)
    # the 8^2 level's bytes double and its prolongation into 16^2 doubles
    assert 0 < nb64 - nb32 < 1e-5 * nb32


def test_precision_label_states_what_runs():
    p, _, _ = W.terzaghi_4097()
    assert "coarsest level" in bench.precision_label(p, False)
    assert "coarsest level fp32" in bench.precision_label(dict(p, options=bench.OPT_COARSEST_STORAGE), False)
    assert bench.precision_label(p, True) == "fp64 storage and arithmetic"


def test_step_model_fp64_has_no_low_parts():
    p, _, _ = W.terzaghi_4097(precision=W.FP64)
    _, nb64 = bench.step_model(p, 4096, fp64=True)
    _, nb32 = bench.step_model(dict(p, precision=W.FP32), 4096, fp64=False)
    assert nb64 > 1.5 * nb32
