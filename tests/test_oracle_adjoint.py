"""Pins of the FP64 adjoint oracle (oracle/dg2_adjoint.py) on the CPU.

The oracle restates the uniform-grid DG2 step in PyTorch tensor operations
and differentiates it with reverse-mode automatic differentiation.  Pinned
here against things outside itself:
  * the C oracle's step, bit for bit, over the same time steps (dam break
    with dry fronts, a flowing reach with inflow and an open edge, rain on
    partly wet rough terrain);
  * central finite differences of the C oracle's fixed-dt step, with respect
    to per-cell Manning n, DEM vertex heights, hydrograph knots and initial
    depth and discharge vertices;
  * still water: no sensitivity to Manning n or to a hydrograph that does not
    flow.
"""
import math
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import dg2_adjoint as A
from paper_2107_02750_gb300 import synth as S

from util import oracle_sim


def grid_of(p):
    return A.Grid(nx=p.nx, ny=p.ny, dx=p.dx, limiter=p.limiter, bc=tuple(p.bc), inflow_edge=p.inflow_edge,
                  inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, rain_rate=p.rain_rate,
                  rain_t_end=p.rain_t_end, knot_t=list(map(float, p.inflow_t)))


def state(sim, p):
    _, _, _, co = sim.leaves()
    return co.T.reshape(9, p.ny, p.nx).copy()


def bed(sim, p):
    return sim.z_level(0)[0].reshape(3, p.ny, p.nx).copy()


def knots(p):
    return p.inflow_Q if len(p.inflow_Q) else np.zeros(1)


def _cases():
    reach, _ = S.adjoint_reach(n=24)
    dam = S.dam_break_circular(n=32, L=0, radius=6.0, h_out=0.0)
    lake = S.lake_at_rest(n=24, L=0, islands=True)
    rain = replace(lake, rain_rate=2e-3, rain_t_end=5.0, n_manning=0.03)
    rect = S.crop(S.adjoint_reach(n=64)[0], 0, 18, 40, 28, 0)
    return [("reach", reach, 30), ("dam_dry", dam, 30), ("rain_islands", rain, 20), ("rect_40x28", rect, 20)]


@pytest.mark.parametrize("name,p,K", _cases(), ids=[c[0] for c in _cases()])
def test_forward_is_the_c_oracle_bit_for_bit(name, p, K):
    s = oracle_sim(p)
    U0, z = state(s, p), bed(s, p)
    dts = [s.step() for _ in range(K)]
    want = state(s, p)
    got = A.forward(U0, z, p.n_cell(), knots(p), dts, 0.0, grid_of(p))
    assert np.array_equal(got, want), np.abs(got - want).max()


def _fd(p, dts, seed, make, delta):
    def J(q):
        s = oracle_sim(q)
        for dt in dts:
            s.step_dt(dt)
        return float((state(s, q) * seed).sum())
    return (J(make(+delta)) - J(make(-delta))) / (2.0 * delta)


def test_gradients_match_central_differences_of_the_c_oracle():
    """Gauge-depth objective J = sum of h0 at 16 gauge cells after 40 steps
    (about 22 s) of the flowing reach.  Steps: 1e-6 n for Manning n, 1e-6 m
    for heights, 1e-6 Q for knots.  Steps of 1e-4 relative move a branch
    (the inflow ghost's critical depth against the boundary cell's limit, a
    wet/dry face near the inlet) within the window, and the difference then
    straddles that kink; as the step shrinks the differences converge to the
    gradient.  The bar is 1e-4 relative; agreement is near 1e-8."""
    p, gauges = S.adjoint_reach(n=24)
    s = oracle_sim(p)
    U0, z = state(s, p), bed(s, p)
    dts = [s.step() for _ in range(40)]
    seed = np.zeros((9, p.ny, p.nx))
    for j, i in gauges:
        seed[0, j, i] += 1.0
    P = grid_of(p)
    G = A.gradients(U0, z, p.n_cell(), p.inflow_Q, dts, 0.0, P, seed, z_vert=p.z_vert)
    Gi = _init_vertex_gradients(p, z, dts, seed, P)
    checks = []
    gn = G["gn"]
    for j, i in np.argwhere(np.abs(gn) > 1e-2 * np.abs(gn).max())[:4]:
        def mk(d, j=j, i=i):
            nm = p.n_cell().copy()
            nm[j, i] += d
            return replace(p, n_manning=nm)
        checks.append(("n", gn[j, i], _fd(p, dts, seed, mk, 1e-6 * p.n_cell()[j, i])))
    for k in (0, 1):
        def mk(d, k=k):
            Q = p.inflow_Q.copy()
            Q[k] += d
            return replace(p, inflow_Q=Q)
        checks.append(("Q", G["gQ"][k], _fd(p, dts, seed, mk, 1e-6 * p.inflow_Q[k])))
    gzv = G["gzv"]
    for j, i in np.argwhere(np.abs(gzv) > 2e-2 * np.abs(gzv).max())[::7][:6]:
        def mk(d, j=j, i=i):
            zz = p.z_vert.copy()
            zz[j, i] += d
            return replace(p, z_vert=zz)
        checks.append(("z", gzv[j, i], _fd(p, dts, seed, mk, 1e-6)))
    for name, field in (("h", "h_vert"), ("qx", "qx_vert")):
        g = Gi[name]
        for j, i in np.argwhere(np.abs(g) > 2e-2 * np.abs(g).max())[::5][:3]:
            def mk(d, j=j, i=i, field=field):
                a = getattr(p, field).copy()
                a[j, i] += d
                return replace(p, **{field: a})
            checks.append((name, g[j, i], _fd(p, dts, seed, mk, 1e-6)))
    assert len(checks) >= 15
    for name, ad, fd in checks:
        assert ad != 0.0, name
        assert abs(ad - fd) <= 1e-4 * abs(ad), (name, ad, fd)


def _init_vertex_gradients(p, z, dts, seed, P):
    """gradients with respect to the initial depth and discharge vertex
    rasters: U0 is their projection (Eq. 8)"""
    hv = torch.tensor(p.h_vert, dtype=torch.float64, requires_grad=True)
    qxv = torch.tensor(p.qx_vert, dtype=torch.float64, requires_grad=True)
    qyv = torch.tensor(p.qy_vert, dtype=torch.float64, requires_grad=True)
    U0 = torch.stack(A.project(hv) + A.project(qxv) + A.project(qyv))
    UK = A.run(U0, torch.tensor(z), torch.tensor(p.n_cell()), torch.tensor(p.inflow_Q), dts, 0.0, P)
    (UK * torch.tensor(seed)).sum().backward()
    return {"h": hv.grad.numpy(), "qx": qxv.grad.numpy(), "qy": qyv.grad.numpy()}


def test_still_water_has_no_sensitivity_to_manning_or_inflow():
    """Lake at rest with islands, an inflow edge whose hydrograph is zero:
    nothing moves, so the final state does not depend on the knots (exact
    zeros) nor on n (zero up to the rounding-level discharges, about 1e-16,
    that the still state carries)."""
    p = replace(S.lake_at_rest(n=16, L=0, islands=True), n_manning=0.03, inflow_edge=S.WEST, inflow_c0=4,
                inflow_c1=9, inflow_t=np.array([0.0, 100.0]), inflow_Q=np.array([0.0, 0.0]))
    s = oracle_sim(p)
    U0, z = state(s, p), bed(s, p)
    dts = [s.step() for _ in range(10)]
    assert np.abs(state(s, p)[0] - U0[0]).max() < 1e-12
    seed = np.random.default_rng(7).standard_normal((9, p.ny, p.nx))
    G = A.gradients(U0, z, p.n_cell(), p.inflow_Q, dts, 0.0, grid_of(p), seed)
    assert np.abs(G["gn"]).max() < 1e-20
    assert np.all(G["gQ"] == 0.0)
    assert np.all(np.isfinite(G["gU0"])) and np.all(np.isfinite(G["gz"]))


def test_valley_crop_gradients_converge_to_central_differences():
    """The 64 x 64 window at the inlet of the 1024 x 1024 valley, a seeded
    weighting of every cell's depth after 60 steps (the gauges lie beyond the
    reach of the inflow's first minute): for Manning n, bed vertices and knots, the
    central differences of the C oracle with steps 1e-6, 1e-7, 1e-8
    (relative, or metres) come within 1e-4 of the gradient as the step
    shrinks below the nearest branch switch."""
    p, gauges = S.adjoint_reach(n=64, crop_of=1024)
    s = oracle_sim(p)
    U0, z = state(s, p), bed(s, p)
    dts = [s.step() for _ in range(60)]
    seed = np.zeros((9, p.ny, p.nx))
    seed[0] = np.random.default_rng(5).standard_normal((p.ny, p.nx))
    G = A.gradients(U0, z, p.n_cell(), p.inflow_Q, dts, 0.0, grid_of(p), seed, z_vert=p.z_vert)
    kq = int(np.argmax(np.abs(G["gQ"])))
    assert abs(G["gQ"][kq]) > 1e-6

    def best(ad, make, scale):
        fs = [_fd(p, dts, seed, make, r * scale) for r in (1e-6, 1e-7, 1e-8)]
        return min(fs, key=lambda f: abs(f - ad))

    checks = []
    gn = G["gn"]
    for j, i in np.argwhere(np.abs(gn) > 1e-2 * np.abs(gn).max())[::17][:2]:
        def mk(d, j=j, i=i):
            nm = p.n_cell().copy()
            nm[j, i] += d
            return replace(p, n_manning=nm)
        checks.append(("n", gn[j, i], best(gn[j, i], mk, p.n_cell()[j, i])))
    def mkq(d):
        Q = p.inflow_Q.copy()
        Q[kq] += d
        return replace(p, inflow_Q=Q)
    checks.append(("Q", G["gQ"][kq], best(G["gQ"][kq], mkq, p.inflow_Q[kq])))
    gzv = G["gzv"]
    for j, i in np.argwhere(np.abs(gzv) > 2e-2 * np.abs(gzv).max())[::23][:2]:
        def mk(d, j=j, i=i):
            zz = p.z_vert.copy()
            zz[j, i] += d
            return replace(p, z_vert=zz)
        checks.append(("z", gzv[j, i], best(gzv[j, i], mk, 1.0)))
    for name, ad, fd in checks:
        assert ad != 0.0, name
        assert abs(ad - fd) <= 1e-4 * abs(ad), (name, ad, fd)


def test_limiter_hand_examples():
    """Stage-input limiting on a 3 x 1 strip, evaluated by hand (minmod on the
    interface offsets sqrt3 v1 against the neighbour differences of the
    averages; the restated limiter is the C oracle's, bit for bit, through
    the forward-step test above):
      cell 1: a = 0.75, forward 0.5, backward 0.25 -> 0.25 (smallest, same sign)
      cell 0: a = 0.125, forward 0.25 (one neighbour) -> kept
      cell 2: a = -0.1, backward 0.5 (opposite signs) -> 0
    (dyadic averages, so the differences are exact)
    and a cell with h0 below h_dry is reduced to a flat free surface over
    its planar bed: h1 = -z1, discharge slopes zero, the flux view flat."""
    s3 = math.sqrt(3.0)
    P = A.Grid(nx=3, ny=1, dx=1.0)
    X = np.zeros((9, 1, 3))
    X[0, 0] = [1.0, 1.25, 1.75]
    X[1, 0] = [0.125 / s3, 0.75 / s3, -0.1 / s3]
    X[3, 0] = [0.1, 0.1, 0.1]
    X[4, 0] = [0.0, 0.02 / s3, 0.0]       # qx slope, differences 0 and 0: limited to 0
    z = np.zeros((3, 1, 3))
    w_st, w_fx, ze = A.limit([torch.tensor(x) for x in X], [torch.tensor(x) for x in z], P)
    slope = w_st[1].numpy()[0]
    assert slope[1] == 0.25 / s3
    assert slope[0] == 0.125 / s3
    assert slope[2] == 0.0
    assert w_st[4].numpy()[0, 1] == 0.0
    # partial-wet reduction
    X2 = np.zeros((9, 1, 3))
    X2[0, 0] = [1.0, 0.0005, 1.0]
    X2[1, 0] = [0.0, 0.3, 0.0]
    X2[3, 0] = [0.0, 0.001, 0.0]
    X2[4, 0] = [0.0, 0.2, 0.0]
    z2 = np.zeros((3, 1, 3))
    z2[1, 0] = [0.0, 0.25, 0.0]
    w_st, w_fx, ze = A.limit([torch.tensor(x) for x in X2], [torch.tensor(x) for x in z2], P)
    assert w_st[1].numpy()[0, 1] == -0.25 and w_st[4].numpy()[0, 1] == 0.0
    assert w_st[3].numpy()[0, 1] == 0.001
    assert w_fx[1].numpy()[0, 1] == 0.0 and ze[1].numpy()[0, 1] == 0.0
