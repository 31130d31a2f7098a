"""Pins of the non-uniform-grid adjoint oracle
(oracle/dg2_adjoint_nonuniform.py): its forward is the C oracle's DG2 step
bit for bit on static graded grids (three and five levels) and on MWDG2
grids frozen after a regridding, with leaves next to refined nodes and to
nodes below coarser leaves; its reverse-mode gradients equal central
differences of the C oracle's fixed-dt steps with respect to DEM vertices,
the Manning raster, initial depth vertices (static) and hydrograph knots."""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import dg2_adjoint_nonuniform as AS
from paper_2107_02750_gb300 import synth as S
from util import oracle_sim


def static_reach(n, Ls, eps):
    """the flowing reach of the uniform adjoint tests on a static graded grid
    built from its own DEM (Sect. 2.2.1)"""
    p, _ = S.adjoint_reach(n=n)
    return replace(p, mode=S.STATIC, L=Ls, M=n >> Ls, N=n >> Ls, eps=eps)


def grid_of(p, lev, ii, jj, mode="static"):
    return AS.grid_from_leaves(p.M, p.N, p.L, p.dx, lev, ii, jj, mode=mode, bc=p.bc, inflow_edge=p.inflow_edge,
                               inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, rain_rate=p.rain_rate,
                               rain_t_end=p.rain_t_end, knot_t=list(p.inflow_t))


def t64(a, grad=False):
    return torch.tensor(np.array(a, dtype=np.float64)).requires_grad_(grad)


def mixed_faces(lev, ii, jj, L, n):
    """leaf faces whose neighbour is finer (the two-children mean) and
    coarser (the prolongation)"""
    cover = np.full((n, n), -1)
    for l, a, b in zip(lev, ii, jj):
        w = 1 << (L - l)
        cover[b * w:(b + 1) * w, a * w:(a + 1) * w] = l
    finer = coarser = 0
    for l, a, b in zip(lev, ii, jj):
        w = 1 << (L - l)
        ring = []
        if a > 0:
            ring.append(cover[b * w:(b + 1) * w, a * w - 1])
        if (a + 1) * w < n:
            ring.append(cover[b * w:(b + 1) * w, (a + 1) * w])
        if b > 0:
            ring.append(cover[b * w - 1, a * w:(a + 1) * w])
        if (b + 1) * w < n:
            ring.append(cover[(b + 1) * w, a * w:(a + 1) * w])
        finer += sum(int(np.any(r > l)) for r in ring)
        coarser += sum(int(np.any(r < l)) for r in ring)
    return finer, coarser


@pytest.mark.parametrize("n,Ls,eps", [(32, 3, 5e-2), (64, 5, 1e-1)])
def test_static_forward_is_the_c_oracle_bit_for_bit(n, Ls, eps):
    p = static_reach(n, Ls, eps)
    s = oracle_sim(p)
    lev, ii, jj, c0 = s.leaves()
    assert len(np.unique(lev)) >= 3
    finer, coarser = mixed_faces(lev, ii, jj, Ls, n)
    assert finer >= 10 and coarser >= 10, (finer, coarser)
    dts = [s.step() for _ in range(8)]
    _, _, _, cK = s.leaves()
    G = grid_of(p, lev, ii, jj)
    U, _, _ = AS.inputs(t64(p.z_vert), t64(p.n_cell()), t64(p.h_vert), t64(p.qx_vert), t64(p.qy_vert), G)
    assert np.array_equal(AS.leaves_of(U, G).numpy(), c0)
    out = AS.run(t64(p.z_vert), t64(p.n_cell()), t64(p.h_vert), t64(p.qx_vert), t64(p.qy_vert),
                 t64(p.inflow_Q), dts, 0.0, G).detach().numpy()
    assert np.array_equal(out, cK), np.abs(out - cK).max()
    assert (cK[:, 3] != c0[:, 3]).any()  # the state has moved


def test_static_gradients_match_central_differences_of_the_c_oracle():
    p = static_reach(32, 3, 5e-2)
    s = oracle_sim(p)
    lev, ii, jj, _ = s.leaves()
    dts = [s.step() for _ in range(6)]
    G = grid_of(p, lev, ii, jj)
    W = np.random.default_rng(7).normal(size=(len(lev), 9))
    zv, nf, hv, Q = t64(p.z_vert, True), t64(p.n_cell(), True), t64(p.h_vert, True), t64(p.inflow_Q, True)
    out = AS.run(zv, nf, hv, t64(p.qx_vert), t64(p.qy_vert), Q, dts, 0.0, G)
    (out * torch.as_tensor(W)).sum().backward()

    def c_loss(pp):
        o = oracle_sim(pp)
        l2, i2, j2, _ = o.leaves()
        assert np.array_equal(l2, lev) and np.array_equal(i2, ii) and np.array_equal(j2, jj)
        for dt in dts:
            o.step_dt(dt)
        return float((o.leaves()[3] * W).sum())

    def central(field, idx, ad):
        best = None
        for h in (1e-5, 1e-6, 1e-7):  # the best of three steps dodges branch kinks
            a = np.array(getattr(p, field), dtype=np.float64)
            b = a.copy()
            a[idx] += h
            b[idx] -= h
            d = (c_loss(replace(p, **{field: a})) - c_loss(replace(p, **{field: b}))) / (2 * h)
            if best is None or abs(d - ad) < abs(best - ad):
                best = d
        return best

    checked = 0
    for field, tens in (("z_vert", zv), ("n_manning", nf), ("h_vert", hv), ("inflow_Q", Q)):
        g = tens.grad.numpy()
        assert np.abs(g).max() > 0, field
        for f in np.argsort(-np.abs(g).ravel())[:3]:
            idx = np.unravel_index(f, g.shape)
            d = central(field, idx, g[idx])
            assert abs(d - g[idx]) <= 1e-4 * abs(g[idx]) + 1e-9, (field, idx, g[idx], d)
            checked += 1
    assert checked == 12


def adaptive_reach(n, Ls, eps):
    p, _ = S.adjoint_reach(n=n)
    return replace(p, mode=S.ADAPTIVE, L=Ls, M=n >> Ls, N=n >> Ls, eps=eps)


def frozen_start(p):
    """the C oracle after one MWDG2 regridding, and a time step of 0.8 times
    the CFL choice on that state"""
    s = oracle_sim(p)
    s.adapt()
    probe = oracle_sim(p)
    dt = 0.8 * probe.step()
    return s, dt


@pytest.mark.parametrize("n,Ls,eps", [(32, 3, 5e-2), (64, 4, 2e-2)])
def test_frozen_mwdg2_forward_is_the_c_oracle_bit_for_bit(n, Ls, eps):
    """On an MWDG2 grid frozen after its regridding, refined neighbours are
    seen through the encoding of their leaves' views and nodes below coarser
    leaves through prolongation (Sect. 2.3); the restatement started from
    the C oracle's leaves equals its frozen steps bit for bit."""
    p = adaptive_reach(n, Ls, eps)
    s, dt = frozen_start(p)
    lev, ii, jj, c0 = s.leaves()
    assert len(np.unique(lev)) >= 2
    finer, coarser = mixed_faces(lev, ii, jj, Ls, n)
    assert finer >= 10 and coarser >= 10, (finer, coarser)
    dts = [dt] * 8
    for d in dts:
        s.step_frozen(d)
    l2, _, _, cK = s.leaves()
    assert np.array_equal(l2, lev)
    G = grid_of(p, lev, ii, jj, mode="adaptive")
    out = AS.run_from(t64(c0), t64(p.z_vert), t64(p.n_cell()), t64(p.inflow_Q), dts, 0.0, G).detach().numpy()
    assert np.array_equal(out, cK), np.abs(out - cK).max()
    assert (cK[:, 3] != c0[:, 3]).any()


def test_frozen_mwdg2_gradients_match_central_differences_of_the_c_oracle():
    p = adaptive_reach(32, 3, 5e-2)
    s, dt = frozen_start(p)
    lev, ii, jj, c0 = s.leaves()
    dts = [dt] * 6
    G = grid_of(p, lev, ii, jj, mode="adaptive")
    W = np.random.default_rng(9).normal(size=(len(lev), 9))
    zv, nf, Q = t64(p.z_vert, True), t64(p.n_cell(), True), t64(p.inflow_Q, True)
    out = AS.run_from(t64(c0), zv, nf, Q, dts, 0.0, G)
    (out * torch.as_tensor(W)).sum().backward()

    def c_loss(pp):
        o = oracle_sim(pp)
        o.adapt()
        l2, i2, j2, u0 = o.leaves()
        assert np.array_equal(l2, lev) and np.array_equal(i2, ii) and np.array_equal(j2, jj)
        assert np.array_equal(u0, c0)
        for d in dts:
            o.step_frozen(d)
        return float((o.leaves()[3] * W).sum())

    checked = 0
    for field, tens in (("z_vert", zv), ("n_manning", nf), ("inflow_Q", Q)):
        g = tens.grad.numpy()
        assert np.abs(g).max() > 0, field
        for f in np.argsort(-np.abs(g).ravel())[:3]:
            idx = np.unravel_index(f, g.shape)
            best = None
            for h in (1e-5, 1e-6, 1e-7):
                a = np.array(getattr(p, field), dtype=np.float64)
                b = a.copy()
                a[idx] += h
                b[idx] -= h
                d = (c_loss(replace(p, **{field: a})) - c_loss(replace(p, **{field: b}))) / (2 * h)
                if best is None or abs(d - g[idx]) < abs(best - g[idx]):
                    best = d
            assert abs(best - g[idx]) <= 1e-4 * abs(g[idx]) + 1e-9, (field, idx, g[idx], best)
            checked += 1
    assert checked == 9


@pytest.mark.parametrize("mode", ["static", "adaptive"])
def test_view_reverse_table_is_the_transpose_of_the_views(mode):
    """The reverse table of the views (what the non-uniform reverse kernels
    gather by owner) applied to random face cotangents equals autograd of
    the oracle's view construction: leaves, static two-children means,
    MWDG2 encodes of refined subtrees, prolongations below coarser leaves."""
    n, Ls, eps = 32, 3, 5e-2
    p = static_reach(n, Ls, eps) if mode == "static" else adaptive_reach(n, Ls, eps)
    s = oracle_sim(p)
    if mode == "adaptive":
        s.adapt()
    lev, ii, jj, _ = s.leaves()
    G = grid_of(p, lev, ii, jj, mode=mode)
    nl = len(lev)
    rng = np.random.default_rng(3)
    planes = torch.tensor(rng.normal(size=(nl, 12)), requires_grad=True)
    dense = AS.dense_from_leaves(planes[:, :9], G)
    beds = AS.dense_from_leaves(torch.cat([planes[:, 9:], torch.zeros(nl, 6, dtype=torch.float64)], 1), G)
    V = AS.build_views(dense, [b[:3] for b in beds], G)
    cot = rng.normal(size=(nl, 4, 4))
    index = {(int(l), int(a), int(b)): k for k, (l, a, b) in enumerate(zip(lev, ii, jj))}
    loss = torch.zeros((), dtype=torch.float64)
    for l in range(Ls + 1):
        if not bool(G.leaf[l].any()):
            continue
        for f in range(4):
            fo = f ^ 1
            axis, step = AS._STEP[f]
            view = AS._limits(V[l][:9], V[l][9:], fo)
            if mode == "static" and l + 1 <= Ls:
                c1, c2 = AS._PAIR[f]
                fine = AS._limits(V[l + 1][:9], V[l + 1][9:], fo)
                avg = [0.5 * (AS._children(q)[c1] + AS._children(q)[c2]) for q in fine]
                view = [AS._w(G.sig[l], avg[q], view[q]) for q in range(4)]
            nb = [AS._shift(q, axis, step) for q in view]
            ins = AS._inside(G, l, f)
            for (ll, a, b), k in index.items():
                if ll == l and bool(ins[b, a]):
                    for q in range(4):
                        loss = loss + float(cot[k, f, q]) * nb[q][b, a]
    loss.backward()
    ref = planes.grad.numpy()
    got = np.zeros((nl, 12))
    table = AS.view_reverse_table(G)
    for k, f, owner, w in table:
        for q in range(4):
            got[owner, 3 * q:3 * q + 3] += w * cot[k, f, q]
    assert len(table) > 4 * nl // 2
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def steep_slope_adaptive():
    """a dam break over a steep dry slope (48 x 48 cells of 2 m, the bed
    falling 30 % to the east) on an MWDG2 grid of 3 x 3 roots and 4 levels:
    the front refines coarse leaves whose depth planes would give children of
    negative depth"""
    n, dx, slope = 48, 2.0, 0.3
    x = np.arange(n + 1) * dx
    X, Y = np.meshgrid(x, x)
    z = slope * (n * dx - X) + 0.5 * slope * Y + 0.5 * S.fractal_surface(n + 1, 7, 4.0)
    eta = np.where(X <= 0.2 * n * dx, z.max() + 2.0 - 0.3 * slope * X, z)
    zeros = np.zeros_like(z)
    return S.Problem("steep_slope", 3, 3, 4, dx, z, eta, zeros, zeros.copy(), is_eta=True, n_manning=0.02,
                     bc=(S.WALL, S.OPEN, S.WALL, S.WALL), mode=S.ADAPTIVE, eps=1e-2)


def _refined_below_negative(c_before, G1, G2):
    """G1 leaves that G2 refines and whose depth plane would give a child a
    negative average (the refinement's scaling at work)"""
    count = 0
    index = {}
    k = 0
    for l in range(G1.L + 1):
        for j, i in torch.nonzero(G1.leaf[l], as_tuple=False).tolist():
            index[(l, i, j)] = k
            k += 1
    for (l, i, j), k in index.items():
        if l == G1.L or not bool(G2.sig[l][j, i]):
            continue
        sp = c_before[k, 0:3]
        for c in range(4):
            sx = 1.0 if c & 1 else -1.0
            sy = 1.0 if c & 2 else -1.0
            if (sp[0] + (AS.HALF_S3 * sx) * sp[1]) + (AS.HALF_S3 * sy) * sp[2] < 0.0:
                count += 1
                break
    return count


@pytest.mark.parametrize("case", ["reach_32_L3", "steep_slope_L4"])
def test_regrid_is_the_c_oracle_adaptation_bit_for_bit(case):
    """The restated state transfer of the MWDG2 adaptation, given the grid
    the C oracle chose, reproduces the C oracle's new leaves bit for bit:
    leaves kept, coarsened (Eq. 9) and refined (Eq. 10 with the depth
    planes kept non-negative for the children)."""
    # the state moves over frozen steps after an adaptation, so that the
    # next adaptation changes the grid
    if case == "reach_32_L3":
        p = adaptive_reach(32, 3, 5e-2)
        s, dt = frozen_start(p)
        K = 12
    else:
        p = steep_slope_adaptive()
        s = oracle_sim(p)
        for _ in range(2):   # a few cycles in, the front refines coarse, partly wet leaves
            dt, K = s.step(), 3
            for _ in range(K):
                s.step_frozen(dt)
            s.adapt()
        s.step()
        K = 3
    for _ in range(K):
        s.step_frozen(dt)
    l1, i1, j1, c_before = s.leaves()
    s.adapt()
    l2, i2, j2, c_after = s.leaves()
    G1 = grid_of(p, l1, i1, j1, mode="adaptive")
    G2 = grid_of(p, l2, i2, j2, mode="adaptive")
    moved = sum(int((G1.leaf[l] != G2.leaf[l]).sum()) for l in range(p.L + 1))
    assert moved > 0
    got = AS.regrid(t64(c_before), G1, G2).detach().numpy()
    assert np.array_equal(got, c_after), np.abs(got - c_after).max()
    if case == "steep_slope_L4":
        assert _refined_below_negative(c_before, G1, G2) > 0


def test_refinement_keeps_children_non_negative_and_the_average():
    """The refinement's depth plane: children's averages are non-negative,
    their mean is the parent's average, and a plane whose children are all
    non-negative is prolonged unchanged (Zhang & Shu's scaling leaves it)."""
    rng = np.random.default_rng(4)
    sp = [torch.tensor(rng.uniform(0.0, 1.0, 500)), torch.tensor(rng.normal(0.0, 1.0, 500)),
          torch.tensor(rng.normal(0.0, 1.0, 500))]
    sp[0][:20] = 0.0          # planes without content lose their slopes
    out = AS.depth_plane_for_children(sp)
    kids = []
    for c in range(4):
        sx = 1.0 if c & 1 else -1.0
        sy = 1.0 if c & 2 else -1.0
        kids.append((out[0] + (AS.HALF_S3 * sx) * out[1]) + (AS.HALF_S3 * sy) * out[2])
    kids = torch.stack(kids)
    assert float(kids.min()) >= -1e-15
    assert torch.allclose(kids.mean(dim=0), sp[0], rtol=0, atol=1e-15)
    orig = torch.stack([(sp[0] + (AS.HALF_S3 * (1.0 if c & 1 else -1.0)) * sp[1]) +
                        (AS.HALF_S3 * (1.0 if c & 2 else -1.0)) * sp[2] for c in range(4)])
    fine = orig.min(dim=0).values >= 0.0
    assert bool(fine.any()) and bool((~fine).any())
    assert torch.equal(out[1][fine], sp[1][fine]) and torch.equal(out[2][fine], sp[2][fine])
    assert bool((out[1][:20] == 0.0).all()) and bool((out[2][:20] == 0.0).all())
    # the smallest child of a scaled plane is exactly at zero depth (up to rounding)
    scaled = ~fine & (sp[0] > 0.0)
    assert float(kids.min(dim=0).values[scaled].abs().max()) <= 1e-15


def test_refrozen_chain_gradients_match_central_differences_of_the_c_oracle():
    """Two frozen MWDG2 segments with the C oracle's regridding between them:
    reverse-mode gradients through the restated segments and transfer equal
    central differences of the C oracle (the same grids chosen under the
    perturbation)."""
    p = adaptive_reach(32, 3, 5e-2)
    s, dt = frozen_start(p)
    l1, i1, j1, c0 = s.leaves()
    K1, K2 = 4, 4
    for _ in range(K1):
        s.step_frozen(dt)
    s.adapt()
    l2, i2, j2, _ = s.leaves()
    G1 = grid_of(p, l1, i1, j1, mode="adaptive")
    G2 = grid_of(p, l2, i2, j2, mode="adaptive")
    assert sum(int((G1.leaf[l] != G2.leaf[l]).sum()) for l in range(p.L + 1)) > 0
    W = np.random.default_rng(17).normal(size=(len(l2), 9))
    zv, nf, Q = t64(p.z_vert, True), t64(p.n_cell(), True), t64(p.inflow_Q, True)
    mid = AS.run_from(t64(c0), zv, nf, Q, [dt] * K1, 0.0, G1)
    out = AS.run_from(AS.regrid(mid, G1, G2), zv, nf, Q, [dt] * K2, K1 * dt, G2)
    (out * torch.as_tensor(W)).sum().backward()

    def c_loss(pp):
        o = oracle_sim(pp)
        o.adapt()
        assert np.array_equal(o.leaves()[0], l1)
        for _ in range(K1):
            o.step_frozen(dt)
        o.adapt()
        lv, a, b, _ = o.leaves()
        assert np.array_equal(lv, l2) and np.array_equal(a, i2) and np.array_equal(b, j2)
        for _ in range(K2):
            o.step_frozen(dt)
        return float((o.leaves()[3] * W).sum())

    checked = 0
    for field, tens in (("z_vert", zv), ("n_manning", nf), ("inflow_Q", Q)):
        g = tens.grad.numpy()
        assert np.abs(g).max() > 0, field
        for f in np.argsort(-np.abs(g).ravel())[:3]:
            idx = np.unravel_index(f, g.shape)
            best = None
            for h in (1e-5, 1e-6, 1e-7):
                a = np.array(getattr(p, field), dtype=np.float64)
                b = a.copy()
                a[idx] += h
                b[idx] -= h
                d = (c_loss(replace(p, **{field: a})) - c_loss(replace(p, **{field: b}))) / (2 * h)
                if best is None or abs(d - g[idx]) < abs(best - g[idx]):
                    best = d
            assert abs(best - g[idx]) <= 1e-4 * abs(g[idx]) + 1e-9, (field, idx, g[idx], best)
            checked += 1
    assert checked == 9
