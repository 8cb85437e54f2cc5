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


@pytest.mark.parametrize("K_level", [[2, 6, 1], [1, 3]])
def test_per_level_sweep_counts_fp64_and_fp32(K_level):
    params, sides, _ = W.terzaghi_33()
    errs, nes = run_both(dict(params, K_level=K_level), sides, 8)
    assert all(a == b for a, b in nes), nes
    assert max(errs) < TOL64, errs
    p32, s32, _ = W.terzaghi_33(precision=W.FP32)
    errs, _ = run_both(dict(p32, ne_fixed=3, K_level=K_level), s32, 8)
    assert errs[0] < TOL32 and errs[1] < TOL32, errs


def test_batch_with_per_level_sweep_counts():
    """Instances with different per-level counts share one batch: each equals
    its solo run (FP64 bitwise) and the oracle."""
    p64, s64, _ = W.terzaghi_33()
    probs = [(dict(p64, ne_fixed=3, K_level=[2, 6, 1]), s64), (dict(p64, ne_fixed=3, K_level=[5]), s64),
             (dict(p64, ne_fixed=3), s64)]
    with biot.Batch(probs) as b:
        b.step(4)
        got = [(b[i].read_u()[0], b[i].read_p()[0]) for i in range(len(b))]
    for (params, sides), (eta, p) in zip(probs, got):
        with biot.Solver(params, sides) as s:
            s.step(4)
            assert np.array_equal(eta, s.read_u()[0]) and np.array_equal(p, s.read_p()[0])
        o = O.Oracle(params, sides)
        o.step(4)
        assert rel(eta, o.read_u()[0]) < TOL64 and rel(p, o.read_p()[0]) < TOL64
        o.close()


def test_autotuned_sweep_counts():
    """biot_autotune_sweeps returns a count per level, keeps the iteration
    converging, and the instance with the counts applied still matches the
    oracle run with the same counts."""
    params, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP64, n=128)
    params = dict(params, c0=0.1)
    with biot.Solver(params, sides) as s:
        tuned = s.autotune_sweeps(apply=True)
        assert len(tuned["K_level"]) == params["levels"]
        assert all(1 <= k <= 8 for k in tuned["K_level"])
        assert 0 < tuned["rho"] < 1 and tuned["ms_per_cycle"] > 0
        s.step(3)
        eta, p = s.read_u()[0], s.read_p()[0]
    o = O.Oracle(dict(params, K_level=tuned["K_level"]), sides)
    o.step(3)
    assert rel(eta, o.read_u()[0]) < TOL64 and rel(p, o.read_p()[0]) < TOL64
    o.close()
