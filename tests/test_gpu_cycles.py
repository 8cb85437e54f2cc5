"""GPU parity of the multigrid cycle variants (W- and F-cycles, a leading
full-multigrid cycle) and of the central-difference pressure gradient
(eq. pressure:gradient:alternative) against the FP64 oracle, which implements
the same definitions (readings R20-R22): FP64 at 1e-12 with the same number of
cycles in every step (tolerance mode), FP32 at 1e-5 (fixed cycles)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402
from test_gpu_parity import CASES  # noqa: E402

TOL64, TOL32 = 1e-12, 1e-5
VARIANTS = {"W": dict(cycle=1), "F": dict(cycle=2), "FMG-V": dict(fmg=1), "FMG-W": dict(cycle=1, fmg=1),
            "central": dict(pgrad=1), "F-FMG-central": dict(cycle=2, fmg=1, pgrad=1)}


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_11382_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run_both(params, sides, steps):
    g = biot.Solver(params, sides)
    o = O.Oracle(params, sides)
    nes = []
    for _ in range(steps):
        g.step(1)
        o.step(1)
        nes.append((g.stats()["last_ne"], o.stats()["last_ne"]))
    out = (rel(g.read_u()[0], o.read_u()[0]), rel(g.read_p()[0], o.read_p()[0]),
           rel(g.read_stress(), o.read_stress()))
    g.close()
    o.close()
    return out, nes


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_terzaghi_33_fp64_tolerance_mode(name):
    params, sides, _ = W.terzaghi_33()
    params = dict(params, **VARIANTS[name])
    errs, nes = run_both(params, sides, 12)
    assert all(a == b for a, b in nes), nes
    assert max(errs) < TOL64, errs


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_terzaghi_33_fp32_fixed_cycles(name):
    params, sides, _ = W.terzaghi_33(precision=W.FP32)
    params = dict(params, ne_fixed=3, **VARIANTS[name])
    errs, _ = run_both(params, sides, 12)
    assert errs[0] < TOL32 and errs[1] < TOL32, errs


@pytest.mark.parametrize("name", ["W", "FMG-W", "F-FMG-central"])
def test_ragged_mixed_walls_fp64(name):
    params, sides = CASES["ragged_48x40_L3_mixed"]()
    params = dict(params, **VARIANTS[name])
    errs, nes = run_both(params, sides, 4)
    assert all(a == b for a, b in nes), nes
    assert max(errs) < TOL64, errs


def test_batch_takes_v_cycles_only():
    p, s, _ = W.terzaghi_33(precision=W.FP32)
    for extra in (dict(cycle=1), dict(fmg=1)):
        with pytest.raises(biot.BiotError) as e:
            biot.Batch([(dict(p, ne_fixed=3, **extra), s)])
        assert e.value.code == biot.ERR_INVALID_ARG
