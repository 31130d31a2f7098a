"""GPU (sm_103a) parity against the FP64 CPU oracle, through the C ABI.

FP64 path: every active leaf's nine coefficients within 1e-9 (m, m^2/s) of
the oracle and identical active-cell sets, step by step.  FP32 free-surface
path: depth within 1e-3 m of the FP64 oracle and wet-extent CSI >= 0.99.
Sizes span several blocks with ragged tails; full-size runs (1024 x 1024
valley, the benchmark workload) are checked on properties that hold at any
size and on the static active set, which the oracle computes at full size."""
import numpy as np
import pytest

import oracle as O
from paper_2107_02750_gb300 import synth as S
from util import average_raster, oracle_sim

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32_H = 1e-3


def gpu_sim(p, precision=0, **over):
    import paper_2107_02750_gb300 as M
    return M.solver_from_problem(p, precision=precision, **over)


def assert_same_leaves(g, o, tol=TOL64, what=""):
    lg, ig, jg, cg = g.read_active()
    lo, io, jo, co = o.leaves()
    assert len(lg) == len(lo), f"{what}: {len(lg)} active leaves on the GPU, {len(lo)} in the oracle"
    np.testing.assert_array_equal(lg, lo)
    np.testing.assert_array_equal(ig, io)
    np.testing.assert_array_equal(jg, jo)
    err = np.abs(cg - co).max() if len(cg) else 0.0
    assert err <= tol, f"{what}: max |GPU - oracle| = {err:.3e}"
    return err


def run_parity(p, nsteps, check_every=1, precision=0):
    g, o = gpu_sim(p, precision), oracle_sim(p)
    assert_same_leaves(g, o, what="initial")
    for k in range(nsteps):
        dg = g.dg2_step()
        do = o.step()
        assert abs(dg - do) <= 1e-9 * max(do, 1e-300), (k, dg, do)
        if (k + 1) % check_every == 0 or k + 1 == nsteps:
            assert_same_leaves(g, o, what=f"step {k + 1}")
    return g, o


def test_circular_dam_break_128_uniform_f64_full_run():
    """128 x 128 circular dam break to t = 5 s (about 77 steps): lockstep for
    the first 60 steps, then both run to 5 s (last step clamped)."""
    p = S.dam_break_circular()
    g, o = run_parity(p, 60, check_every=10)
    g.run_to_time(5.0)
    o.run_to(5.0)
    t, steps = g.get_time()
    assert steps == o.steps and abs(t - 5.0) < 1e-12
    assert_same_leaves(g, o, what="t = 5 s")
    v = g.get_volume()
    assert abs(v["volume"] - o.diag()["volume"]) <= 1e-12 * v["volume"]
    assert v["n_clip"] == 0


def test_circular_dam_break_128_mra_lossless_at_zero_epsilon():
    """MRA at L = 7, epsilon = 0: encode then decode keeps every finest
    coefficient (the GPU gathers scale coefficients, so exactly)."""
    p = S.dam_break_circular(L=7, eps=0.0, mode=S.ADAPTIVE)
    g = gpu_sim(p)
    l0, i0, j0, c0 = g.read_active()
    g.mra_encode()
    n = g.mra_adapt(0.0)
    l1, i1, j1, c1 = g.read_active()
    assert n == 128 * 128 and (l1 == 7).all()
    np.testing.assert_array_equal(c1, c0)
    o = oracle_sim(p)
    o.adapt()
    assert_same_leaves(g, o, tol=1e-13, what="after adapt")


@pytest.mark.parametrize("islands", [False, True])
def test_lake_at_rest_uniform_f64(islands):
    p = S.lake_at_rest(n=48, islands=islands)
    g, o = run_parity(p, 60, check_every=20)
    _, _, _, c = g.read_active()
    assert np.abs(c[:, 3:]).max() <= 1e-12


def test_uniform_valley_inflow_rain_f64():
    p = S.valley(n=96, L=5, mode=S.UNIFORM, peak_Q=120.0, t_peak=100.0)
    p.rain_rate, p.rain_t_end = 2e-4, 50.0
    g, o = run_parity(p, 150, check_every=25)
    vg, vo = g.get_volume(), o.diag()
    for key in ("volume", "v_in", "v_out", "v_rain"):
        assert abs(vg[key] - vo[key]) <= 1e-9 * max(1.0, abs(vo[key])), key
    assert vg["v_in"] > 0


def test_static_valley_f64():
    p = S.valley(n=128, L=7, mode=S.STATIC, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    g, o = run_parity(p, 120, check_every=20)
    lev, _, _, _ = g.read_active()
    assert len(np.unique(lev)) >= 3


def test_static_valley_reflux_f64():
    """Reflux interface rule: lockstep parity with the oracle and the mass
    budget closed to round-off on the GPU."""
    p = S.valley(n=128, L=7, mode=S.STATIC, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    p.iface_rule = 1
    v0 = gpu_sim(p).get_volume()["volume"]
    g, o = run_parity(p, 120, check_every=20)
    v = g.get_volume()
    assert v["n_clip"] == 0 and v["v_clip"] == 0.0
    budget = v0 + v["v_in"] - v["v_out"] + v["v_rain"]
    assert abs(v["volume"] - budget) <= 1e-12 * v["volume"]
    assert v["v_in"] > 0


@pytest.mark.parametrize("rule", [0, 1])
def test_urban_window_256_static_rain_f64_and_f32(rule):
    """Urban-like DEM (random-walk terrain, 8 m blocks off a 100 m road grid,
    per-cell Manning n 0.013 / 0.035), static grid from one MRA of the
    topography at eps = 1e-2, uniform rain: a 256 x 256 window at dx = 2 m.
    The rain rate is raised to 3.6 m/h so that water ponds and flows within
    the 100-step lockstep horizon.  FP64 against the oracle under both
    interface rules; FP32 against FP64 on depth and wet extent.  The reflux
    rule closes the mass budget (FP64 to round-off); the paper rule moves
    mass at coarse/fine faces, and its drift is only bounded here."""
    p = S.urban(n=256, L=8, rain_mm_per_h=3600.0, rain_hours=1.0)
    p.iface_rule = rule
    assert np.ndim(p.n_manning) == 2 and len(np.unique(p.n_manning)) == 2
    g, o = run_parity(p, 100, check_every=20)
    lev, _, _, c = g.read_active()
    assert len(np.unique(lev)) >= 3 and len(lev) < p.nx * p.ny
    assert (c[:, 0] > 1e-2).sum() > 100  # ponded water
    # FP32 against FP64 on cell-average depths at t = 8 s (a rain film of
    # about 8 mm), the FP32 run taking the FP64 run's time steps
    # (mwdg_dg2_step_dt), so that the comparison sees the FP32 arithmetic
    # alone: max <= 1e-3 m (the FP32 path's accuracy target).  A nearly dry leaf cut by a
    # wall can be stored as flat depth in one precision and as flat free
    # surface in the other (its average agrees, its plane does not), so
    # planes are not compared pointwise here.  Later in the horizon the bar
    # is not met (test_urban_window_256_f32_end_of_horizon).
    d64, f = gpu_sim(p), gpu_sim(p, precision=1)
    t = 0.0
    while t < 8.0:
        dt = d64.dg2_step()
        f.dg2_step_dt(dt)
        t += dt
    a32, a64 = average_raster(f), average_raster(d64)
    assert np.abs(a32 - a64).max() <= TOL32_H
    assert g.get_volume()["n_clip"] == 0
    for sim, tol in ((g, 1e-12), (f, 1e-5)):
        v = sim.get_volume()  # dry start: the budget is rain + inflow - outflow
        drift = abs(v["volume"] - (v["v_in"] - v["v_out"] + v["v_rain"])) / v["volume"]
        assert drift <= (tol if rule == 1 else 0.1), drift


@pytest.mark.xfail(strict=True, reason="on the urban window the FP32 path does not hold 1e-3 m to the end of the "
                   "100-step horizon even on the FP64 run's steps: max 0.025-0.028 m (cell averages) where rain "
                   "films against the 8 m walls are within rounding of the 1e-3 m dry depth and the two "
                   "precisions take different wet/dry branches")
def test_urban_window_256_f32_end_of_horizon():
    """FP32 against FP64 on the urban window (reflux rule) after 100 steps on
    the FP64 run's time steps, held to the FP32 path's accuracy target: max depth error
    <= 1e-3 m and CSI >= 0.99 (known not to be met)."""
    p = S.urban(n=256, L=8, rain_mm_per_h=3600.0, rain_hours=1.0)
    p.iface_rule = 1
    d64, f = gpu_sim(p), gpu_sim(p, precision=1)
    for _ in range(100):
        f.dg2_step_dt(d64.dg2_step())
    a32, a64 = average_raster(f), average_raster(d64)
    assert O.extent_scores(a32, a64)[2] >= 0.99
    assert np.abs(a32 - a64).max() <= TOL32_H


def test_gauges_match_fields_and_oracle():
    """mwdg_read_gauges at seeded cells equals the finest-resolution fields
    there, and the oracle's fields (FP64, adaptive valley)."""
    p = S.valley(n=128, L=7, mode=S.ADAPTIVE, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    g, o = run_parity(p, 40, check_every=40)
    rng = np.random.default_rng(5)
    cells = np.stack([rng.integers(0, p.nx, 37), rng.integers(0, p.ny, 37)], axis=1)
    cells[0] = (0, 0)
    cells[1] = (p.nx - 1, p.ny - 1)
    hg, ug, vg = g.read_gauges(cells)
    hf, uf, vf = g.read_fields()
    ho, uo, vo = o.fields()
    for a, f, r in ((hg, hf, ho), (ug, uf, uo), (vg, vf, vo)):
        np.testing.assert_array_equal(a, f[cells[:, 1], cells[:, 0]])
        assert np.abs(a - r[cells[:, 1], cells[:, 0]]).max() <= 1e-9
    assert g.read_gauges(np.zeros((0, 2)))[0].shape == (0,)
    import paper_2107_02750_gb300 as M
    with pytest.raises(M.MwdgError):
        g.read_gauges([[p.nx, 0]])


def test_adaptive_valley_f64():
    p = S.valley(n=128, L=7, mode=S.ADAPTIVE, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    g, o = run_parity(p, 120, check_every=5)
    lev, _, _, c = g.read_active()
    assert len(np.unique(lev)) >= 2 and len(lev) < 128 * 128 // 2
    assert (c[:, 0] > 1e-3).sum() > 20  # the flood has entered


@pytest.mark.parametrize("mode", [S.UNIFORM, S.STATIC, S.ADAPTIVE])
def test_graph_replay_on_own_stream_f64(mode):
    """On a non-default stream each step is one captured CUDA graph replay;
    the results are those of the oracle (and of direct launches)."""
    import torch
    st = torch.cuda.Stream()
    p = S.valley(n=128, L=7, mode=mode, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    g, o = gpu_sim(p, stream=st.cuda_stream), oracle_sim(p)
    for k in range(60):
        dg = g.dg2_step()
        do = o.step()
        assert abs(dg - do) <= 1e-9 * do, (k, dg, do)
    assert_same_leaves(g, o, what="after 60 graph steps")
    # a run of queued steps without host synchronisation, then the budget
    g.run_steps(20)
    for _ in range(20):
        o.step()
    assert_same_leaves(g, o, what="after 20 queued steps")
    assert g.launch_count() > 0


def test_adaptive_lake_at_rest_islands_f64():
    p = S.lake_at_rest(n=64, L=4, islands=True, mode=S.ADAPTIVE, eps=1e-2)
    g, o = run_parity(p, 40, check_every=10)
    _, _, _, c = g.read_active()
    assert np.abs(c[:, 3:]).max() <= 1e-12


@pytest.mark.parametrize("mode", [S.UNIFORM, S.STATIC, S.ADAPTIVE])
def test_ragged_non_square_grid_f64(mode):
    """M x N = 25 x 9 coarsest elements at L = 2 (100 x 36 finest): level
    sizes are not multiples of any block size, and M != N."""
    base = S.valley(n=128, L=7, mode=mode, peak_Q=100.0, t_peak=60.0)
    p = S.crop(base, 0, 40, 100, 36, L=2)
    p.mode = mode
    run_parity(p, 40, check_every=10)


def test_degenerate_grids_f64():
    # a single element, wet, with friction and walls
    nv = np.ones((2, 2))
    p = S.Problem("one", 1, 1, 0, 5.0, np.zeros((2, 2)), 2.0 * nv, 0.5 * nv, np.zeros((2, 2)),
                  n_manning=0.03)
    run_parity(p, 10)
    # a dry domain: nothing moves, dt is dt_max
    p = S.Problem("dry", 4, 4, 2, 1.0, np.random.default_rng(0).uniform(0, 1, (17, 17)),
                  np.zeros((17, 17)), np.zeros((17, 17)), np.zeros((17, 17)), mode=S.ADAPTIVE)
    g, o = run_parity(p, 5)
    t, _ = g.get_time()
    assert abs(t - 5 * p.dt_max) < 1e-12


def _lockstep_to(g, o, t_end, check_every):
    """both step (CFL steps) until the oracle reaches t_end; every dt within
    1e-9 relative, the leaves compared every check_every steps and at the end"""
    k = 0
    while o.t < t_end:
        dg = g.dg2_step()
        do = o.step()
        assert abs(dg - do) <= 1e-9 * do, (k, dg, do)
        k += 1
        if k % check_every == 0:
            assert_same_leaves(g, o, what=f"step {k}, t = {o.t:.1f} s")
    assert_same_leaves(g, o, what=f"t = {o.t:.1f} s")
    return k


def test_valley_window_through_the_inflow_mwdg2_10min_f64():
    """The rapid-flow valley (1024 x 1024, dx = 10 m) cropped to the 256 x 256
    window through the inflow, MWDG2 at L = 8 and eps = 1e-3, 10 min of the
    hydrograph's rise in lockstep with the oracle: every dt within 1e-9
    relative, identical active sets and coefficients within 1e-9 every 100
    steps.  No depth is clipped on the GPU and the mass budget closes to
    round-off with no clipped volume in it."""
    p = S.crop(S.valley(n=1024), 0, 1024 // 2 - 128, 256, 256, L=8)
    g, o = gpu_sim(p), oracle_sim(p)
    v0 = g.get_volume()["volume"]
    k = _lockstep_to(g, o, 600.0, 100)
    assert k > 1000
    v = g.get_volume()
    assert v["n_clip"] == 0 and v["v_clip"] == 0.0
    assert abs(v["volume"] - (v0 + v["v_in"] - v["v_out"])) <= 1e-12 * v["volume"]
    assert v["v_in"] > 4.0e4


@pytest.mark.parametrize("mode", [S.UNIFORM, S.ADAPTIVE])
def test_valley_window_2h_keeps_depths_nonnegative_f64(mode):
    """The valley window through the inflow over the configuration's whole 2 h
    (the hydrograph's rise, peak and recession; MWDG2 refines and coarsens
    around the shrinking flood): no depth is clipped, and the mass budget,
    with no clipped volume in it, closes to round-off on the uniform grid
    and to the drift of the interface rule at MWDG2's coarse/fine faces
    (each side's flux from its own view, Sect. 2.3: about 1e-7 of the
    inflow over the run)."""
    from dataclasses import replace
    full = S.valley(n=1024)
    p = replace(S.crop(full, 0, 1024 // 2 - 128, 256, 256, L=8 if mode == S.ADAPTIVE else 0), mode=mode)
    g = gpu_sim(p)
    g.run_to_time(7200.0)
    v = g.get_volume()
    assert v["n_clip"] == 0 and v["v_clip"] == 0.0
    tol = 1e-11 if mode == S.UNIFORM else 1e-6
    assert abs(v["volume"] - (v["v_in"] - v["v_out"])) <= tol * v["v_in"]


def test_full_valley_benchmark_configuration_f64():
    """The benchmark's own configuration: the 1024 x 1024 valley at L = 10,
    eps = 1e-3 (five levels of 16 x 16 MRA tiles, a coarse tail of 341 nodes
    run by the first block of later kernels, about 240,000 leaves in two
    waves of the leaf kernels), from t = 0 with the hydrograph peaking at
    120 s, 60 steps in lockstep with the oracle.""" 
    p = S.valley(n=1024, L=10, mode=S.ADAPTIVE, eps=1e-3, peak_Q=400.0, t_peak=120.0)
    g, o = gpu_sim(p), oracle_sim(p)
    assert_same_leaves(g, o, what="initial")
    for k in range(60):
        dg = g.dg2_step()
        do = o.step()
        assert abs(dg - do) <= 1e-9 * do, (k, dg, do)
        if (k + 1) % 20 == 0:
            assert_same_leaves(g, o, what=f"step {k + 1}")
    lev, _, _, c = g.read_active()
    assert len(np.unique(lev)) >= 2 and len(lev) > 200000
    assert (c[:, 0] > 1e-3).sum() > 10  # the flood has entered
    assert g.get_volume()["n_clip"] == 0


def test_urban_window_static_2min_f64():
    """The slow-to-gradual urban configuration (2048 x 2048 at dx = 2 m, 8 m
    blocks off a road grid, 50 mm/h of rain) cropped to a 512 x 512 window,
    static grid from the topography at eps = 1e-2 (reflux rule), 2 min of
    rain in lockstep with the oracle.  No depth is clipped and the budget
    (rain in, nothing out) closes to round-off."""
    p = S.crop(S.urban(), 768, 768, 512, 512, L=9)
    p.iface_rule = 1
    g, o = gpu_sim(p), oracle_sim(p)
    lev, _, _, _ = g.read_active()
    assert len(np.unique(lev)) >= 3 and len(lev) < 512 * 512 // 2
    _lockstep_to(g, o, 120.0, 200)
    v = g.get_volume()
    assert v["n_clip"] == 0 and v["v_clip"] == 0.0
    assert abs(v["volume"] - v["v_rain"]) <= 1e-12 * v["volume"]


def test_invalid_inputs_are_rejected():
    import paper_2107_02750_gb300 as M
    with pytest.raises(M.MwdgError) as e:
        M.Solver(M=1, N=1, L=16, dx=1.0)
    assert e.value.status == -2
    s = M.Solver(M=2, N=2, L=2, dx=1.0)
    z = np.zeros((9, 9))
    z[3, 3] = np.nan
    with pytest.raises(M.MwdgError) as e:
        s.load_dem(z)
    assert e.value.status == -4
    with pytest.raises(M.MwdgError) as e:
        s.dg2_step()
    assert e.value.status == -6


# ---------------------------------------------------------------------------
# FP32 free-surface path against the FP64 oracle
# ---------------------------------------------------------------------------
def _depths_close(g, o, wet=0.01):
    hg, _, _ = g.read_fields()
    ho, _, _ = o.fields()
    err = np.abs(hg - ho).max()
    _, _, csi = O.extent_scores(hg, ho, wet)
    return err, csi


def test_f32_uniform_dam_break():
    p = S.dam_break_circular()
    g, o = gpu_sim(p, precision=1), oracle_sim(p)
    g.run_to_time(5.0)
    o.run_to(5.0)
    err, csi = _depths_close(g, o)
    assert err <= TOL32_H and csi >= 0.99


@pytest.mark.parametrize("mode", [S.STATIC, S.ADAPTIVE])
def test_f32_valley(mode):
    p = S.valley(n=128, L=7, mode=mode, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    g, o = gpu_sim(p, precision=1), oracle_sim(p)
    g.run_to_time(80.0)
    o.run_to(80.0)
    err, csi = _depths_close(g, o)
    assert err <= TOL32_H, err
    assert csi >= 0.99, csi


def test_f32_lake_at_rest_islands_stays_at_rest():
    p = S.lake_at_rest(n=64, islands=True)
    g = gpu_sim(p, precision=1)
    g.run_steps(500)
    _, u, v = g.read_fields()
    assert np.abs(u).max() < 1e-4 and np.abs(v).max() < 1e-4


# ---------------------------------------------------------------------------
# Full size: the 1024 x 1024 valley of the benchmark
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def valley_full():
    return S.valley(n=1024, L=10, mode=S.STATIC, eps=1e-3)


def test_full_size_static_active_set_matches_oracle(valley_full):
    p = valley_full
    g = gpu_sim(p)
    o = oracle_sim(p)
    lg, ig, jg, _ = g.read_active()
    lo, io, jo, _ = o.leaves()
    np.testing.assert_array_equal(lg, lo)
    np.testing.assert_array_equal(ig, io)
    np.testing.assert_array_equal(jg, jo)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_adaptive_mass_budget(valley_full, precision):
    p = S.valley(n=1024, L=10, mode=S.ADAPTIVE, eps=1e-3, peak_Q=400.0, t_peak=120.0)
    g = gpu_sim(p, precision=precision)
    v0 = g.get_volume()["volume"]
    g.run_to_time(90.0)
    v = g.get_volume()
    if precision == 0:
        assert v["n_clip"] == 0 and v["v_clip"] == 0.0
    else:  # FP32: a draining leaf's own rounding, far below the budget's tolerance
        assert v["v_clip"] <= 1e-7 * v["v_in"]
    budget = v0 + v["v_in"] - v["v_out"] + v["v_rain"]
    tol = 1e-9 if precision == 0 else 1e-4
    assert abs(v["volume"] - budget) <= tol * max(1.0, v["volume"]), (v, budget)
    assert v["v_in"] > 0
    # active leaves tile the domain
    lev, i, j, _ = g.read_active()
    area = np.sum(4.0 ** (10 - lev.astype(np.float64)))
    assert area == 1024 * 1024


def _f32_on_f64_steps(p, t_end):
    """FP64 and FP32 runs of p to t_end, the FP32 run taking the FP64 run's
    CFL steps (mwdg_dg2_step_dt): (FP64 depth raster, FP32 depth raster,
    FP64 volume, FP32 volume)"""
    a, b = gpu_sim(p, precision=0), gpu_sim(p, precision=1)
    t = 0.0
    while t < t_end:
        dt = a.dg2_step()
        b.dg2_step_dt(dt)
        t += dt
    ha, _, _ = a.read_fields()
    hb, _, _ = b.read_fields()
    return ha, hb, a.get_volume()["volume"], b.get_volume()["volume"]


def test_full_size_f32_on_f64_steps_meets_the_bar_before_the_front():
    """Benchmark workload, 1024 x 1024 MWDG2: FP32 against FP64 on the GPU at
    t = 120 s with the FP32 run on the FP64 run's time steps, so that the
    comparison sees the FP32 arithmetic alone: max depth error <= 1e-3 m and
    CSI >= 0.99 (the FP32 path's accuracy target), volumes within 1e-6 relative."""
    p = S.valley(n=1024, L=10, mode=S.ADAPTIVE, eps=1e-3)
    ha, hb, va, vb = _f32_on_f64_steps(p, 120.0)
    assert ((ha > 0.01) | (hb > 0.01)).sum() > 0
    assert np.abs(ha - hb).max() <= TOL32_H
    assert O.extent_scores(hb, ha)[2] >= 0.99
    assert abs(vb - va) <= 1e-6 * va


@pytest.mark.xfail(strict=True, reason="the FP32 path does not meet the 1e-3 m / CSI 0.99 bar once the flood "
                   "front runs down the channel: at 300 s, on the FP64 run's own steps, max 1.15 m and CSI "
                   "0.94 over about 100 wet cells (a leaf within rounding of the 1e-3 m dry depth takes the "
                   "other wet/dry branch and the front moves by a cell); CSI is back above 0.99 from 900 s on "
                   "while the maximum stays at 0.1-0.5 m")
def test_full_size_f32_on_f64_steps_after_the_front_forms():
    """The same comparison at t = 300 s, held to the same bar (known not to be
    met; the benchmark reports the figures over the run)."""
    p = S.valley(n=1024, L=10, mode=S.ADAPTIVE, eps=1e-3)
    ha, hb, va, vb = _f32_on_f64_steps(p, 300.0)
    assert np.abs(ha - hb).max() <= TOL32_H
    assert O.extent_scores(hb, ha)[2] >= 0.99


# ---------------------------------------------------------------------------
# FV1 (Sect. 2.1.2) and HWFV1 (Sect. 2.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [S.UNIFORM, S.STATIC, S.ADAPTIVE])
def test_fv1_valley_f64(mode):
    """FV1 (uniform, static graded) and HWFV1 (adaptive, Haar MRA) on the
    valley with inflow: lockstep parity with the oracle."""
    kw = dict(n=128, L=7, mode=mode, peak_Q=200.0, t_peak=100.0)
    if mode != S.UNIFORM:
        # Haar details of sloping terrain do not vanish (multiwavelet ones do
        # for planes), so HWFV1 needs a larger epsilon to coarsen this valley
        kw["eps"] = 1e-2 if mode == S.STATIC else 5e-2
    p = S.fv1(S.valley(**kw))
    g, o = run_parity(p, 120, check_every=20)
    lev, _, _, c = g.read_active()
    assert np.abs(c[:, [1, 2, 4, 5, 7, 8]]).max() == 0.0  # piecewise constant
    assert (c[:, 0] > 1e-3).sum() > 20
    if mode != S.UNIFORM:
        assert len(np.unique(lev)) >= 2
    vg, vo = g.get_volume(), o.diag()
    for key in ("volume", "v_in", "v_out"):
        assert abs(vg[key] - vo[key]) <= 1e-9 * max(1.0, abs(vo[key])), key


def test_fv1_dam_break_and_lake_f64_f32():
    """Uniform FV1 circular dam break in lockstep (FP64) and FP32 against it;
    FV1 lake at rest with islands stays at rest on the GPU."""
    p = S.fv1(S.dam_break_circular())
    g, o = run_parity(p, 60, check_every=20)
    f = gpu_sim(p, precision=1)
    f.run_to_time(g.get_time()[0])
    h32, _, _ = f.read_fields()
    h64, _, _ = g.read_fields()
    assert np.abs(h32 - h64).max() <= TOL32_H
    q = S.fv1(S.lake_at_rest(n=48, islands=True))
    for prec, tol in ((0, 1e-12), (1, 1e-5)):
        s = gpu_sim(q, precision=prec)
        s.run_steps(200)
        _, _, _, c = s.read_active()
        assert np.abs(c[:, 3:]).max() <= tol, prec


# ---------------------------------------------------------------------------
# ACC (local inertial, Sect. 2.1.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [S.UNIFORM, S.STATIC])
def test_acc_valley_f64(mode):
    """ACC on the valley with inflow and rain, uniform and static graded grid
    (half-face discharges aggregated): lockstep parity with the oracle and the
    mass budget."""
    p = S.acc(S.valley(n=128, L=7, mode=mode, eps=1e-2, peak_Q=200.0, t_peak=100.0))
    p.rain_rate, p.rain_t_end = 1e-4, 1e9
    v0 = gpu_sim(p).get_volume()["volume"]
    g, o = run_parity(p, 150, check_every=25)
    lev, _, _, c = g.read_active()
    assert (c[:, 0] > 1e-3).sum() > 20
    if mode == S.STATIC:
        assert len(np.unique(lev)) >= 3
    v, vo = g.get_volume(), o.diag()
    for key in ("volume", "v_in", "v_out", "v_rain", "v_clip"):
        assert abs(v[key] - vo[key]) <= 1e-9 * max(1.0, abs(vo[key])), key
    budget = v0 + v["v_in"] - v["v_out"] + v["v_rain"] + v["v_clip"]
    assert abs(v["volume"] - budget) <= 1e-12 * v["volume"]


def test_acc_channel_and_lake_f64_f32():
    """ACC sloped channel (open outlet) in lockstep with the oracle; FP32
    against FP64; lake at rest with islands exact in both precisions."""
    p = S.acc(S.sloped_channel(nx=128, ny=4, dx=10.0, slope=1e-3, q_in=2.0, n_manning=0.03))
    p.dt_max = 5.0
    g, o = run_parity(p, 200, check_every=50)
    f = gpu_sim(p, precision=1)
    f.run_to_time(g.get_time()[0])
    h32, _, _ = f.read_fields()
    h64, _, _ = g.read_fields()
    assert np.abs(h32 - h64).max() <= TOL32_H
    q = S.acc(S.lake_at_rest(n=48, islands=True))
    for prec in (0, 1):
        s = gpu_sim(q, precision=prec)
        _, _, _, c0 = s.read_active()
        s.run_steps(200)
        _, _, _, c = s.read_active()
        assert np.abs(c[:, 3:]).max() == 0.0, prec
        np.testing.assert_array_equal(c[:, 0], c0[:, 0])


@pytest.mark.parametrize("coarse_nodes", [64, 1024])
def test_adaptive_coarse_level_schedules_f64(coarse_nodes):
    """The coarsest MRA levels (those of at most `coarse_nodes` nodes) run in
    one block: with 256 (the default) and 64 the flux views' coarse levels
    are encoded by the first block of each stage update and the
    regularisation's by the first block of the decode; with 1024 on this
    pyramid (levels of 1024 nodes, more than one pass of a block) every pass
    keeps them in its last block, as loops over the levels.  Each schedule
    gives the oracle's steps."""
    p = S.valley(n=128, L=7, mode=S.ADAPTIVE, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    g, o = gpu_sim(p), oracle_sim(p)
    g.set_launch_shape(coarse_nodes=coarse_nodes)
    assert g.launch_shape()[1] == coarse_nodes
    for k in range(60):
        dg = g.dg2_step()
        do = o.step()
        assert abs(dg - do) <= 1e-9 * do, (k, dg, do)
        if (k + 1) % 20 == 0:
            assert_same_leaves(g, o, what=f"coarse_nodes {coarse_nodes}, step {k + 1}")


def test_grown_launch_shape_keeps_results_and_volume():
    """A launch shape larger than the one the context was created with (the
    volume's per-block partial sums keep their size; the volume launch uses
    no more blocks than they hold): steps and the FP64 volume equal those of
    the default shape."""
    import paper_2107_02750_gb300 as M
    p = S.valley(n=128, L=7, mode=S.ADAPTIVE, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    a, b = gpu_sim(p), gpu_sim(p)
    b.set_launch_shape(grid_leaves=8192)
    assert b.launch_shape()[0] == 8192 and a.launch_shape()[0] < 8192
    for s in (a, b):
        s.run_steps(30)
    la, _, _, ca = a.read_active()
    lb, _, _, cb = b.read_active()
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(ca, cb)
    va, vb = a.get_volume()["volume"], b.get_volume()["volume"]
    assert abs(va - vb) <= 1e-12 * va
