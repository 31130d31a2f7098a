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
