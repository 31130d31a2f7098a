"""Pins of the oracle's DG2 step (Eq. 1-4, Sect. 2.1.1, 2.2.1, 2.3) against
what the mathematics fixes: lake at rest over rough terrain (C-property, also
with emerging islands and on static / adaptive grids), Ritter and Stoker
dam-break closed forms, D4 symmetry and volume conservation of the circular
dam break, the mass budget with inflow and rain, MWDG2 at epsilon = 0 against
uniform DG2, and the friction ODE's closed-form decay."""
import numpy as np
import pytest

import oracle as O
from paper_2107_02750_gb300 import synth as S
from util import oracle_sim, ritter_depth, stoker_depth

G = 9.80665


@pytest.mark.parametrize("islands", [False, True])
def test_lake_at_rest_uniform(islands):
    p = S.lake_at_rest(n=32, islands=islands)
    s = oracle_sim(p)
    _, _, _, c0 = s.leaves()
    for _ in range(1000):
        s.step()
    _, _, _, c = s.leaves()
    h = c[:, 0]
    wet = h > 1e-3
    assert np.abs(c[:, 3:]).max() <= 1e-12
    assert np.abs(h[wet] - c0[wet, 0]).max() <= 1e-12
    if islands:
        assert (~wet).sum() > 0


@pytest.mark.parametrize("mode", [S.STATIC, S.ADAPTIVE])
def test_lake_at_rest_nonuniform(mode):
    p = S.lake_at_rest(n=32, L=3, islands=True, mode=mode, eps=1e-2)
    s = oracle_sim(p)
    for _ in range(300):
        s.step()
    lev, _, _, c = s.leaves()
    assert np.abs(c[:, 3:]).max() <= 1e-12
    if mode == S.STATIC:
        assert len(np.unique(lev)) > 1


def _strip_profile(s, p):
    h, _, _ = s.fields()
    return h.mean(axis=0)


@pytest.mark.parametrize("kind", ["ritter", "stoker"])
def test_dam_break_closed_forms(kind):
    hR = 0.0 if kind == "ritter" else 0.1
    errs = []
    for nx, dx in ((100, 1.0), (200, 0.5)):
        p = S.dam_break_strip(nx=nx, ny=4, dx=dx, h_left=1.0, h_right=hR)
        s = oracle_sim(p, dt_max=1.0)
        T = 6.0
        s.run_to(T)
        x = (np.arange(nx) + 0.5) * dx
        prof = _strip_profile(s, p)
        if kind == "ritter":
            exact = ritter_depth(x, T, 50.0, 1.0, G)
        else:
            exact = stoker_depth(x, T, 50.0, 1.0, hR, G)
        errs.append(np.mean(np.abs(prof - exact)))
        # y-invariance of the strip
        h, _, _ = s.fields()
        assert np.abs(h - h[0:1, :]).max() < 1e-12
    assert errs[1] < errs[0]
    assert errs[1] < (0.0045 if kind == "ritter" else 0.0035)
    assert errs[1] < 0.75 * errs[0]


def test_circular_dam_break_symmetry_and_volume():
    p = S.dam_break_circular()
    s = oracle_sim(p)
    v0 = s.diag()["volume"]
    s.run_to(5.0)
    d = s.diag()
    assert abs(d["volume"] - v0) <= 1e-12 * v0
    assert d["n_clip"] == 0
    h, _, _ = s.fields()
    assert np.abs(h - h.T).max() <= 1e-12
    assert np.abs(h - h[:, ::-1]).max() <= 1e-12
    assert np.abs(h - h[::-1, :]).max() <= 1e-12
    assert 60 <= s.steps <= 90


def test_mass_budget_with_inflow_and_rain():
    p = S.valley(n=64, L=6, mode=S.UNIFORM, dx=10.0, peak_Q=50.0, t_peak=60.0)
    p.rain_rate, p.rain_t_end = 1e-4, 40.0
    s = oracle_sim(p)
    v0 = s.diag()["volume"]
    s.run_to(120.0)
    d = s.diag()
    assert d["n_clip"] == 0 and d["v_clip"] == 0.0
    budget = v0 + d["v_in"] - d["v_out"] + d["v_rain"]
    assert abs(d["volume"] - budget) <= 1e-12 * max(1.0, d["volume"])
    assert d["v_in"] > 0 and d["v_rain"] > 0


@pytest.mark.parametrize("rule", [0, 1])
def test_static_mass_budget_by_interface_rule(rule):
    """Static graded valley with inflow: the reflux rule closes the mass
    budget to round-off (each coarse/fine face moves the same mass on both
    sides); the paper rule (each side from its own view) does not, and its
    drift is what the reflux rule removes."""
    p = S.valley(n=64, L=6, mode=S.STATIC, eps=1e-2, dx=10.0, peak_Q=80.0, t_peak=60.0)
    p.iface_rule = rule
    s = oracle_sim(p)
    lev, _, _, _ = s.leaves()
    assert len(np.unique(lev)) >= 2  # coarse/fine faces exist
    v0 = s.diag()["volume"]
    s.run_to(150.0)
    d = s.diag()
    assert d["n_clip"] == 0 and d["v_clip"] == 0.0
    budget = v0 + d["v_in"] - d["v_out"] + d["v_rain"]
    drift = abs(d["volume"] - budget) / max(1.0, d["volume"])
    assert d["v_in"] > 0
    if rule == 1:
        assert drift <= 1e-12, drift
    else:
        assert drift > 1e-10, drift


def test_reflux_equals_paper_rule_on_uniform_grid():
    p = S.valley(n=32, L=5, mode=S.UNIFORM, dx=10.0, peak_Q=40.0, t_peak=30.0)
    a = oracle_sim(p)
    p.iface_rule = 1
    b = oracle_sim(p)
    for _ in range(30):
        assert a.step() == b.step()
    np.testing.assert_array_equal(a.leaves()[3], b.leaves()[3])


def test_mwdg2_at_zero_epsilon_equals_uniform():
    pu = S.dam_break_circular(n=64, radius=6.0, L=6, mode=S.UNIFORM)
    pa = S.dam_break_circular(n=64, radius=6.0, L=6, mode=S.ADAPTIVE, eps=0.0)
    su, sa = oracle_sim(pu), oracle_sim(pa)
    for _ in range(20):
        dtu = su.step()
        dta = sa.step()
        assert abs(dtu - dta) <= 1e-13 * dtu
    lu, iu, ju, cu = su.leaves()
    la, ia, ja, ca = sa.leaves()
    np.testing.assert_array_equal(la, lu)
    np.testing.assert_array_equal(ia, iu)
    np.testing.assert_array_equal(ja, ju)
    assert np.abs(ca - cu).max() <= 1e-12


def test_friction_decay_matches_ode():
    """Uniform state, open boundaries: only friction acts.  The exact solution
    of dq/dt = -g n^2 q |q| / h^(7/3) at constant depth is
    1/q = 1/q0 + g n^2 t / h^(7/3); the split linearised-implicit update
    reproduces it exactly at any time step (1/q grows by dt g n^2 / h^(7/3)
    per step), so it must match to round-off for two step sizes."""
    n, h, q0, T = 0.05, 2.0, 1.5, 40.0
    for dtm in (0.7, 0.1):
        nv = 9
        p = S.Problem("fr", 8, 8, 0, 10.0, np.zeros((nv, nv)), np.full((nv, nv), h),
                      np.full((nv, nv), q0), np.zeros((nv, nv)), n_manning=n,
                      bc=(S.OPEN,) * 4, dt_max=dtm)
        s = oracle_sim(p)
        s.run_to(T)
        _, _, _, c = s.leaves()
        q_exact = 1.0 / (1.0 / q0 + G * n * n * T / h ** (7.0 / 3.0))
        assert abs(s.t - T) < 1e-12
        assert np.abs(c[:, 0] - h).max() < 1e-12
        assert np.abs(c[:, 3] - q_exact).max() < 1e-12
        assert q_exact < 0.9 * q0


def test_limiter_keeps_averages_within_initial_bounds():
    """Wet-bed dam break with the minmod limiter: no new extrema of the cell
    averages of h (and no clipping)."""
    p = S.dam_break_strip(nx=120, ny=4, dx=0.5, h_left=2.0, h_right=0.5)
    s = oracle_sim(p)
    s.run_to(3.0)
    _, _, _, c = s.leaves()
    assert c[:, 0].max() <= 2.0 + 1e-12 and c[:, 0].min() >= 0.5 - 1e-12
    assert s.diag()["n_clip"] == 0


def test_metrics():
    assert O.rmse([1, 2, 3], [1, 2, 3]) == 0.0
    assert abs(O.rmse([0, 0], [3, 4]) - np.sqrt(12.5)) < 1e-15
    h = np.array([[0, 1], [1, 1]], float)
    r = np.array([[1, 1], [0, 1]], float)
    H, F, C = O.extent_scores(h, r)
    assert (H, F, C) == (2 / 3, 1 / 3, 2 / 4)


def _planar_case(Lf=4, M=4, R=1.0):
    """A planar bed with one compactly supported bump, a planar free surface
    and planar discharges; returns the vertex fields of a grid of cell size
    `dx` and the bump's zone (the box, one finest cell wider than the bump's
    support, outside which bed, depth and discharges are exactly planar)."""
    xb, yb, rb = 21.5, 22.5, 1.5

    def fields(dx, n):
        x = np.arange(n + 1) * dx
        X, Y = np.meshgrid(x, x)
        r2 = ((X - xb) ** 2 + (Y - yb) ** 2) / rb ** 2
        z = 0.02 * X + 0.01 * Y + 0.8 * np.maximum(0.0, 1.0 - r2) ** 2
        eta = 3.0 + 0.01 * X - 0.005 * Y
        qx = 0.4 + 0.01 * Y - 0.005 * X
        qy = -0.3 + 0.008 * X + 0.002 * Y
        return z, eta - z, qx, qy

    zone = (xb - rb - R, xb + rb + R, yb - rb - R, yb + rb + R)
    return fields, zone


@pytest.mark.parametrize("mode", [S.STATIC, S.ADAPTIVE])
def test_interface_rule_on_planar_data_equals_the_uniform_grid_of_each_level(mode):
    """Pin of the interface rule on non-homogeneous faces (Sect. 2.3): each
    leaf evaluates its faces from its neighbours' views at its own level
    (the encoding of finer neighbours, the prolongation of a coarser one;
    on static grids the coarse side averages the two finer interface
    values).  Encoding and prolongation reproduce a plane exactly, and
    minmod keeps a plane's slopes, so on globally planar data one stage of
    Eq. 4a on the non-uniform grid must equal, leaf by leaf, the same stage
    on the uniform grid of the leaf's own level.  Only leaves whose stencil
    (the leaf and its four face neighbours at its level) stays clear of the
    bump that makes the grid non-uniform are compared; the test requires
    many of them to border a leaf of another level."""
    Lf, M, R, dt = 4, 4, 1.0, 0.05
    fields, (x0, x1, y0, y1) = _planar_case(Lf, M, R)
    n = M << Lf
    z, h, qx, qy = fields(R, n)
    s = O.Sim(M=M, N=M, L=Lf, R=R, mode=mode, eps=1e-3)
    s.load_dem(z)
    s.load_roughness(np.zeros((n, n)))
    s.load_initial(h, qx, qy)
    s.init_grid()
    if mode == S.ADAPTIVE:
        s.adapt()
    lev, ii, jj, before = s.leaves()
    s.stage(dt)
    lev2, ii2, jj2, after = s.leaves()
    assert np.array_equal(lev, lev2) and np.array_equal(ii, ii2) and np.array_equal(jj, jj2)
    assert len(np.unique(lev)) >= 3
    Lop = (after - before) / dt

    # the uniform grid of each level present
    ref = {}
    for l in np.unique(lev):
        dxl = R * (1 << (Lf - l))
        nl = M << l
        zl, hl, qxl, qyl = fields(dxl, nl)
        u = O.Sim(M=M, N=M, L=int(l), R=dxl, mode=S.UNIFORM)
        u.load_dem(zl)
        u.load_roughness(np.zeros((nl, nl)))
        u.load_initial(hl, qxl, qyl)
        u.init_grid()
        _, ui, uj, ub = u.leaves()
        u.stage(dt)
        _, _, _, ua = u.leaves()
        ref[int(l)] = {(int(a), int(b)): (ub[k], (ua[k] - ub[k]) / dt) for k, (a, b) in enumerate(zip(ui, uj))}

    # level of the leaf covering each finest cell, to find mixed-level faces
    cover = np.full((n, n), -1)
    for l, a, b in zip(lev, ii, jj):
        f = 1 << (Lf - l)
        cover[b * f:(b + 1) * f, a * f:(a + 1) * f] = l
    compared = mixed = coarse_side = 0
    for k, (l, a, b) in enumerate(zip(lev, ii, jj)):
        dxl = R * (1 << (Lf - l))
        bx0, bx1, by0, by1 = (a - 1) * dxl, (a + 2) * dxl, (b - 1) * dxl, (b + 2) * dxl
        if bx0 < x1 and bx1 > x0 and by0 < y1 and by1 > y0:
            continue  # the stencil reaches the bump
        ub, uL = ref[int(l)][(int(a), int(b))]
        np.testing.assert_allclose(before[k], ub, rtol=0, atol=1e-12)
        np.testing.assert_allclose(Lop[k], uL, rtol=0, atol=1e-9 * max(1.0, np.abs(uL).max()))
        compared += 1
        f = 1 << (Lf - l)
        ring = []
        if a > 0:
            ring.append(cover[b * f:(b + 1) * f, a * f - 1])
        if (a + 1) * f < n:
            ring.append(cover[b * f:(b + 1) * f, (a + 1) * f])
        if b > 0:
            ring.append(cover[b * f - 1, a * f:(a + 1) * f])
        if (b + 1) * f < n:
            ring.append(cover[(b + 1) * f, a * f:(a + 1) * f])
        if any(np.any(r != l) for r in ring):
            mixed += 1
        if any(np.any(r > l) for r in ring):
            coarse_side += 1
    assert compared >= 20 and mixed >= 8 and coarse_side >= 4, (compared, mixed, coarse_side)


def test_dg2_relaxes_to_manning_normal_depth():
    """Steady uniform flow down a constant slope S with Manning friction:
    the bed-slope force g h S balances the resistance g n^2 u |u| / h^(1/3),
    so the unit discharge is q = h^(5/3) S^(1/2) / n and the depth away
    from the ends is h_n = (q n / S^(1/2))^(3/5) (Manning's formula).  The
    split implicit friction reaches it up to an O(dt) error of the split.
    Started 20 % too deep, the DG2 step (bed source, revisions, friction,
    inflow ghost, open outlet) must drain to h_n and carry the inflow
    through.  The discharge is read after the two stages and before the
    next friction step, so it sits half a step's bed-slope increment
    (dt g h S / 2, 0.2 % of q here) above the face flux that mass
    conservation ties to the inflow."""
    q_in, S_, n_m = 2.0, 1e-3, 0.03
    hn = (q_in * n_m / np.sqrt(S_)) ** 0.6
    p = S.sloped_channel(nx=200, ny=4, dx=10.0, slope=S_, q_in=q_in, n_manning=n_m)
    p.h_vert = np.full_like(p.z_vert, 1.2 * hn)
    p.qx_vert = np.full_like(p.z_vert, q_in)
    s = oracle_sim(p)
    h0, _, _ = s.fields()
    s.run_to(3600.0)
    h, u, v = s.fields()
    reach = slice(40, 160)
    assert np.abs(h0[:, reach] / hn - 1.2).max() < 1e-12
    assert np.abs(h[:, reach] / hn - 1.0).max() < 0.01, (h[:, reach].min(), h[:, reach].max(), hn)
    assert np.abs(h[:, reach] * u[:, reach] / q_in - 1.0).max() < 5e-3
    assert np.abs(v).max() < 1e-9


def test_cfl_time_step_closed_forms():
    """The time step (Sect. 2.1.1, Courant number 0.33 for DG2): C times the
    minimum over wet leaves of dx / (|u| + sqrt(g h)) in both directions,
    with the inflow ghost at critical depth (dx / (q / h_c + sqrt(g h_c)),
    h_c = (q^2 / g)^(1/3)) as one more candidate, at most dt_max and never
    past the end time."""
    g, C = 9.80665, 0.33
    n = 8
    ones = np.ones((n + 1, n + 1))
    # uniform flow: the faster of the two directions decides
    p = S.Problem("cfl", n, n, 0, 5.0, 0.0 * ones, 2.0 * ones, 3.0 * ones, -1.0 * ones, bc=(S.WALL,) * 4)
    s = oracle_sim(p, dt_max=10.0)
    want = C * min(5.0 / (1.5 + np.sqrt(g * 2.0)), 5.0 / (0.5 + np.sqrt(g * 2.0)))
    assert abs(s.step() - want) <= 1e-15 * want
    # dt_max and the end time clamp it
    s = oracle_sim(p, dt_max=0.1)
    assert s.step() == 0.1
    s = oracle_sim(p, dt_max=10.0)
    assert abs(s.step(0.05) - 0.05) <= 1e-17
    # a static graded grid: brute force over its leaves (dx per level)
    q = S.valley(n=64, L=6, mode=S.STATIC, eps=1e-2, peak_Q=0.0)
    x = np.linspace(0.0, 1.0, 65)
    X, Y = np.meshgrid(x, x)
    q.h_vert = 1.0 + 0.5 * X
    q.qx_vert = 0.8 * np.sin(3.0 * Y)
    q.qy_vert = 0.3 + 0.2 * X * Y
    q.inflow_edge = -1
    s = oracle_sim(q, dt_max=100.0)
    lev, _, _, c = s.leaves()
    assert len(np.unique(lev)) > 1
    dx = q.dx * 2.0 ** (q.L - lev)
    h = c[:, 0]
    cel = np.sqrt(g * h)
    want = C * np.min(np.minimum(dx / (np.abs(c[:, 3] / h) + cel), dx / (np.abs(c[:, 6] / h) + cel)))
    assert abs(s.step() - want) <= 1e-14 * want
    # a dry domain: only the inflow ghost's critical-depth speed counts
    d = S.Problem("dry_inflow", n, n, 0, 2.0, 0.0 * ones, 0.0 * ones, 0.0 * ones, 0.0 * ones,
                  bc=(S.WALL,) * 4, inflow_edge=S.WEST, inflow_c0=2, inflow_c1=5,
                  inflow_t=np.array([0.0, 100.0]), inflow_Q=np.array([4.0, 4.0]))
    s = oracle_sim(d, dt_max=100.0)
    qu = 4.0 / (4 * 2.0)  # unit discharge over the four inflow cells
    hc = (qu * qu / g) ** (1.0 / 3.0)
    want = C * 2.0 / (qu / hc + np.sqrt(g * hc))
    assert abs(s.step() - want) <= 1e-12 * want
