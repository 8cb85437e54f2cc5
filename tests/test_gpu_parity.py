"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (relative L-infinity of eta and p, as the product states them):
  * FP64 path: 1e-12 -- same algorithm, only the rounding order differs;
  * FP32 path: 1e-5  -- FP32 populations, FP64 coupling accumulators.
Both sides get identical seeded inputs from paper_2409_11382_gb300.workloads.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2409_11382_gb300 import biot, workloads as W  # noqa: E402

TOL64 = 1e-12
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


def run_both(params, sides, steps, sources=None, per_step=False):
    g = biot.Solver(params, sides)
    o = O.Oracle(params, sides)
    if sources is not None:
        g.set_sources(*sources)
        o.set_sources(np.ascontiguousarray(np.moveaxis(sources[0], 0, -1)) if sources[0] is not None else None,
                      sources[1])
    codes = []
    if per_step:
        for _ in range(steps):
            codes.append((g.step(1), o.step(1), g.stats()["last_ne"], o.stats()["last_ne"]))
    else:
        codes.append((g.step(steps), o.step(steps), None, None))
    out = dict(eta=(g.read_u()[0], o.read_u()[0]), p=(g.read_p()[0], o.read_p()[0]),
               sigma=(g.read_stress(), o.read_stress()), codes=codes,
               t=(g.read_u()[1], o.read_u()[1]), gstats=g.stats(), ostats=o.stats())
    g.close()
    o.close()
    return out


def test_terzaghi_33_fp64_tolerance_mode_matches_oracle():
    """33x33 nodes, FP64, residual tolerance 1e-10, 50 steps to T = 0.1."""
    params, sides, steps = W.terzaghi_33()
    r = run_both(params, sides, steps, per_step=True)
    for gc, oc, gne, one in r["codes"]:
        assert gc == oc == 0
        assert gne == one  # identical number of V-cycles in every step
    assert r["t"][0] == r["t"][1] == pytest.approx(0.1)
    assert rel(*r["eta"]) < TOL64
    assert rel(*r["p"]) < TOL64
    assert rel(*r["sigma"]) < TOL64
    assert r["gstats"]["total_cycles"] == r["ostats"]["total_cycles"]


def test_terzaghi_33_fp32_fixed_cycles_within_1e5():
    params, sides, steps = W.terzaghi_33(precision=W.FP32)
    params = dict(params, ne_fixed=3)
    r = run_both(params, sides, steps)
    assert rel(*r["eta"]) < TOL32
    assert rel(*r["p"]) < TOL32
    assert rel(*r["sigma"]) < TOL32


def test_residual_norms_match_oracle():
    """The FP64 stopping-test norm max|g - ELASTIC_STEP(g)| and its FP64 2-norm
    over every population, after one V-cycle per step (far from convergence, so
    the values do not sit at the rounding floor)."""
    params, sides, _ = W.terzaghi_33()
    params = dict(params, tol=1e-300, ne_max=1)
    g = biot.Solver(params, sides)
    o = O.Oracle(params, sides)
    for _ in range(3):
        assert g.step(1) == biot.ERR_NOT_CONVERGED
        assert o.step(1) == -4
        gs, os_ = g.stats(), o.stats()
        assert gs["last_res"] > 1e-8
        assert abs(gs["last_res"] - os_["last_res"]) <= 1e-9 * os_["last_res"]
        assert abs(gs["last_res_l2"] - os_["last_res_l2"]) <= 1e-9 * os_["last_res_l2"]
    g.close()
    o.close()


@pytest.mark.parametrize("alpha", [0.5, 1.0])
def test_step_load_257_as_specified_fp64(alpha):
    """257x257, c0 = 0.01: the scheme is unstable for this storage coefficient; the
    FP64 path must follow the oracle step for step while the modes grow."""
    params, sides, _ = W.step_load_257(alpha=alpha)
    r = run_both(params, sides, 12)
    assert rel(*r["eta"]) < 1e-11
    assert rel(*r["p"]) < 1e-11


@pytest.mark.parametrize("alpha", [0.5, 1.0])
def test_step_load_257_stable_variant_fp32_vs_oracle(alpha):
    """257x257 step load with c0 = 0.1 (stable): FP32 populations within 1e-5 of
    the FP64 oracle after 40 of the 200 steps."""
    params, sides, _ = W.step_load_257(alpha=alpha, precision=W.FP32)
    params = dict(params, c0=0.1)
    r = run_both(params, sides, 40)
    assert rel(*r["eta"]) < TOL32
    assert rel(*r["p"]) < TOL32


@pytest.mark.parametrize("alpha", [0.5, 1.0])
def test_step_load_257_stable_variant_full_run_fp64_and_fp32(alpha):
    """All 200 steps of the 257x257 step load with c0 = 0.1 (the stable variant):
    one oracle run, against which the FP64 path holds 1e-12 and the FP32 path
    1e-5 in eta, p and sigma."""
    params, sides, steps = W.step_load_257(alpha=alpha)
    params = dict(params, c0=0.1)
    o = O.Oracle(params, sides)
    assert o.step(steps) == 0
    ref = dict(eta=o.read_u()[0], p=o.read_p()[0], sigma=o.read_stress())
    o.close()
    for precision, tol in ((W.FP64, TOL64), (W.FP32, TOL32)):
        with biot.Solver(dict(params, precision=precision), sides) as g:
            assert g.step(steps) == biot.OK
            got = dict(eta=g.read_u()[0], p=g.read_p()[0], sigma=g.read_stress())
        for k in ref:
            assert rel(got[k], ref[k]) < tol, (precision, k, rel(got[k], ref[k]))


# ---------------------------------------------------------------------------
# edge cases: ragged tiles, rectangles, odd coarse grids, single level,
# every boundary type on every side, periodic with sources
# ---------------------------------------------------------------------------

def _generic(nx, ny, levels, sides, precision=W.FP64, **kw):
    p = dict(nx=nx, ny=ny, lx=1.0, ly=ny / nx, lam=0.8, mu=0.6, alpha=0.9, c0=0.5, kappa=0.3,
             dt=0.02, r=0.5, levels=levels, K=3, gamma=0.75, tol=1e-11, ne_max=200,
             ne_fixed=0, precision=precision)
    p.update(kw)
    return p, sides


def _profiles(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=(2, 2 * n + 1)), 0.1 * rng.normal(size=2 * n + 1)


def _sides_mixed(nx, ny, seed=0):
    eb, pb = _profiles(nx, seed, 0.01)
    et, pt = _profiles(nx, seed + 1)
    er, pr = _profiles(ny, seed + 2, 0.5)
    el, pl = _profiles(ny, seed + 3, 0.01)
    return [dict(eta_type=W.DIRICHLET, p_type=W.NEUMANN, eta_profile=eb),
            dict(eta_type=W.NEUMANN, p_type=W.DIRICHLET, eta_profile=er, p_profile=pr),
            dict(eta_type=W.NEUMANN, p_type=W.DIRICHLET, eta_profile=et, p_profile=pt),
            dict(eta_type=W.DIRICHLET, p_type=W.NEUMANN, eta_profile=el)]


CASES = {
    "ragged_48x40_L3_mixed": lambda: _generic(48, 40, 3, _sides_mixed(48, 40)),
    "odd_coarse_24x24_L4": lambda: _generic(24, 24, 4, _sides_mixed(24, 24, 5)),
    "single_level_8x16": lambda: _generic(8, 16, 1, _sides_mixed(8, 16, 7), K=2, ne_fixed=40),
    "symmetry_top_traction_sides": lambda: _generic(32, 32, 3, [
        dict(eta_type=W.SYMMETRY, p_type=W.SYMMETRY),
        dict(eta_type=W.NEUMANN, p_type=W.DIRICHLET, eta_profile=_profiles(32, 11)[0]),
        dict(eta_type=W.SYMMETRY, p_type=W.SYMMETRY),
        dict(eta_type=W.DIRICHLET, p_type=W.NEUMANN)]),
    "periodic_x_dirichlet_y": lambda: _generic(64, 32, 4, [
        dict(eta_type=W.DIRICHLET, p_type=W.DIRICHLET, eta_profile=_profiles(64, 3, 0.01)[0], p_profile=_profiles(64, 3)[1]),
        dict(eta_type=W.PERIODIC, p_type=W.PERIODIC),
        dict(eta_type=W.NEUMANN, p_type=W.NEUMANN, eta_profile=_profiles(64, 4)[0]),
        dict(eta_type=W.PERIODIC, p_type=W.PERIODIC)]),
    "all_symmetry_pressure_dirichlet_top": lambda: _generic(32, 32, 3, [
        dict(eta_type=W.SYMMETRY, p_type=W.SYMMETRY),
        dict(eta_type=W.SYMMETRY, p_type=W.SYMMETRY),
        dict(eta_type=W.NEUMANN, p_type=W.DIRICHLET, eta_profile=_profiles(32, 9)[0], p_profile=np.ones(65)),
        dict(eta_type=W.SYMMETRY, p_type=W.SYMMETRY)]),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_edge_cases(case, precision):
    params, sides = CASES[case]()
    params = dict(params, precision=precision)
    if precision == W.FP32:
        params["ne_fixed"] = params["ne_fixed"] or 4
    r = run_both(params, sides, 6)
    tol = TOL64 if precision == W.FP64 else TOL32
    errs = {k: rel(*r[k]) for k in ("eta", "p", "sigma")}
    assert max(errs.values()) < tol, (case, errs)


def test_periodic_manufactured_sources_fp64():
    n = 32
    params, sides = W.manufactured_params(n, alpha=1.0, r=0.5, ne_fixed=4, K=2)
    rng = np.random.default_rng(0)
    fb = rng.normal(size=(2, n, n))
    s = rng.normal(size=(n, n))
    r = run_both(params, sides, 10, sources=(fb, s))
    assert rel(*r["eta"]) < TOL64
    assert rel(*r["p"]) < TOL64


def test_repeatable_bitwise():
    params, sides, _ = W.terzaghi_33(precision=W.FP32)
    params = dict(params, ne_fixed=3)
    outs = []
    for _ in range(2):
        with biot.Solver(params, sides) as s:
            s.step(7)
            outs.append((s.read_u()[0], s.read_p()[0]))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_divergence_is_reported():
    """Explicit coupling at alpha = 1 on the manufactured problem diverges (§4.1);
    the solver reports it instead of returning garbage."""
    n = 16
    params, sides = W.manufactured_params(n, alpha=1.0, r=0.0, ne_fixed=4, K=2)
    params = dict(params, dt=params["dt"] * 50)
    with biot.Solver(params, sides) as s:
        s.set_sources(None, 1e3 * np.random.default_rng(0).normal(size=(n, n)))
        code = None
        for _ in range(5000):
            try:
                s.step(1)
            except biot.BiotError as e:
                code = e.code
                break
        assert code == biot.ERR_DIVERGED
        assert s.stats()["diverged"] == 1


# ---------------------------------------------------------------------------
# full size, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------

def test_terzaghi_4097_full_size_fp32():
    """4097x4097 nodes, FP32, 10 levels, MG(3,4).  The problem does not depend on x,
    so (a) every column must be identical and (b) a 512-cell-wide strip of the same
    problem -- which the oracle can afford -- must give the same column."""
    steps = 2
    params, sides, _ = W.terzaghi_4097()
    with biot.Solver(params, sides) as s:
        s.step(steps)
        eta, _ = s.read_u()
        p, _ = s.read_p()
    col_eta, col_p = eta[:, :, :1], p[:, :1]
    assert np.abs(eta - col_eta).max() <= 1e-12 * np.abs(eta).max()
    assert np.abs(p - col_p).max() <= 1e-12 * np.abs(p).max()
    strip = dict(params, nx=512, lx=512 / 4096, precision=W.FP64)
    ref = O.Oracle(strip, W.top_load_sides(512, W.uniform_load(512)))
    ref.step(steps)
    eta_o, _ = ref.read_u()
    p_o, _ = ref.read_p()
    assert rel(eta[:, :, :512], eta_o) < TOL32
    assert rel(p[:, :512], p_o) < TOL32


GOLD_STRIP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "terzaghi_4096_strip_fp64.npz")


@pytest.mark.parametrize("coarsest", ["fp64", "fp32"])
def test_terzaghi_4097_100_steps_fp32_vs_stored_oracle_columns(coarsest):
    """The 4097x4097-node problem over its 100 steps: every column of the FP32
    path within 1e-5 (relative L-infinity of eta and p) of the FP64 oracle's
    column (stored by tests/golden/make_terzaghi_4096_strip.py) after 1, 10 and
    100 steps, with the FP64 coarsest level (default) and with the FP32 one."""
    gold = np.load(GOLD_STRIP)
    params, sides, _ = W.terzaghi_4097()
    if coarsest == "fp32":
        params = dict(params, options=biot.OPT_COARSEST_STORAGE)
    done = 0
    errs = []
    with biot.Solver(params, sides) as s:
        for k, steps in enumerate(gold["steps"]):
            s.step(int(steps) - done)
            done = int(steps)
            eta, t = s.read_u()
            p, _ = s.read_p()
            assert t == pytest.approx(float(gold["t"][k]))
            errs.append((int(steps), rel(eta, gold["eta"][k][:, :, None]), rel(p, gold["p"][k][:, None])))
    assert all(e < TOL32 and q < TOL32 for _, e, q in errs), errs


def test_tolerance_mode_device_loop_matches_host_loop():
    """Tolerance mode: the V-cycle loop of a step runs on the device (a CUDA-graph
    WHILE node whose condition a stopping-test kernel sets) and gives bitwise the
    result, and the same V-cycle counts, as the host-driven loop."""
    params, sides, _ = W.terzaghi_33()
    out = []
    for direct in (False, True):
        with biot.Solver(params, sides) as s:
            if direct:
                s.sweep_timing(True)  # instrumentation forces direct launches and the host loop
            nes = []
            for _ in range(6):
                s.step(1)
                nes.append(s.stats()["last_ne"])
            s.step(4)
            st = s.stats()
            out.append((s.read_u()[0], s.read_p()[0], nes, st["total_cycles"], st["last_ne"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and min(out[0][2]) >= 1
    assert out[0][3] == out[1][3] and out[0][4] == out[1][4]


def test_tolerance_mode_not_converged_is_reported_from_the_device_loop():
    params, sides, _ = W.terzaghi_33()
    params = dict(params, tol=1e-30, ne_max=2)  # unreachable tolerance
    with biot.Solver(params, sides) as s:
        assert s.step(1) == biot.ERR_NOT_CONVERGED   # first solve: host loop
        assert s.step(3) == biot.ERR_NOT_CONVERGED   # device loop
        st = s.stats()
        assert st["last_ne"] == 2 and st["notconv_steps"] == 5  # t = 0 solve + 4 steps


def test_autotuned_launch_shapes_do_not_change_results():
    """biot_autotune picks strip heights per level and sweep mode; the arithmetic
    per cell is the same for every strip height, so results are bitwise equal."""
    params, sides, _ = W.step_load_257(alpha=1.0, precision=W.FP32, n=1024, ne_fixed=3)
    params = dict(params, c0=0.1)
    out = []
    for tune in (False, True):
        with biot.Solver(params, sides) as s:
            if tune:
                shapes = s.autotune()
                assert shapes and all(r >= 2 and r % 2 == 0 for r, _ in shapes.values())
            s.step(2)
            out.append((s.read_u()[0], s.read_p()[0]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_graph_replay_matches_direct_launches():
    """Fixed-cycle steps replayed from captured CUDA graphs (both flow-buffer
    parities) give bitwise the result of launching every kernel directly."""
    params, sides, _ = W.step_load_257(alpha=0.5, precision=W.FP32, n=64)
    params = dict(params, c0=0.1)
    out = []
    for direct in (False, True):
        with biot.Solver(params, sides) as s:
            if direct:
                s.sweep_timing(True)  # instrumentation forces direct launches
            s.step(3)
            s.step(4)
            out.append((s.read_u()[0], s.read_p()[0], s.stats()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2]["total_cycles"] == out[1][2]["total_cycles"]
    assert out[0][2]["kernel_launches"] == out[1][2]["kernel_launches"]


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_checkpoint_resume_is_bitwise(precision):
    """Saving after k steps and resuming in a fresh instance gives bitwise the
    uninterrupted run (§5 checkpoint / resume)."""
    params, sides, _ = W.step_load_257(alpha=1.0, precision=precision, n=64)
    params = dict(params, c0=0.1)
    with biot.Solver(params, sides) as a:
        a.step(4)
        blob = a.save()
        a.step(3)
        ref = (a.read_u(), a.read_p()[0], a.stats()["total_cycles"])
    with biot.Solver(params, sides) as b:
        b.load(blob)
        assert b.read_u()[1] == pytest.approx(4 * params["dt"])
        b.step(3)
        got = (b.read_u(), b.read_p()[0], b.stats()["total_cycles"])
    assert np.array_equal(got[0][0], ref[0][0]) and got[0][1] == ref[0][1]
    assert np.array_equal(got[1], ref[1]) and got[2] == ref[2]
    with biot.Solver(dict(params, nx=32, ny=32, levels=3), W.top_load_sides(32, W.step_load(32))) as c:
        with pytest.raises(biot.BiotError) as e:
            c.load(blob)
        assert e.value.code == biot.ERR_INVALID_ARG


def test_fp64_at_1024_rows_within_the_oracles_rounding_spread():
    """The FP64 path on a 128-column strip of the 1024^2 benchmark problem
    (8 levels), one step: at this size reordering the oracle's own FP64 sums
    moves its result by about 1e-12, so the GPU is held to three times that
    spread (and to 1e-12 where the spread is smaller)."""
    from rounding_checks import rel, rounding_spread, strip
    params, sides = strip(1024, 128)
    spread, (eta_o, p_o) = rounding_spread(params, sides)
    with biot.Solver(params, sides) as g:
        assert g.step(1) == biot.OK
        eta, p = g.read_u()[0], g.read_p()[0]
    gap = max(rel(eta, eta_o), rel(p, p_o))
    assert gap <= max(TOL64, 3 * spread), (gap, spread)
