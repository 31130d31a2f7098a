"""Discrete adjoint of the DG2 step on frozen non-uniform grids on the GPU
(mwdg_adj_create_frozen): static graded grids (Sect. 2.2.1) and MWDG2 grids
held fixed over a segment (Sect. 2.3), against the FP64 oracles.

  * the forward sweep is the C oracle's step bit for bit: on static grids
    with the CFL time steps (orc_step), on a frozen MWDG2 grid over given
    steps (orc_step_frozen) and in its first CFL step;
  * its gradients with respect to the leaves' coefficients, the finest bed
    planes, the finest Manning raster and the hydrograph knots agree with
    reverse-mode differentiation of the non-uniform oracle
    (oracle/dg2_adjoint_nonuniform.py) to 1e-9 of each array's largest
    entry;
  * a frozen grid whose leaves are all on the finest level gives the uniform
    context's run and gradients bit for bit;
  * two segments chained by autograd give the one-segment gradients;
  * FP32 tracks the FP64 oracle (steps, depths, gradient correlation);
  * re-freezing at a checkpoint (mwdg_adj_regrid, the MWDG2 adaptation's
    state transfer to the grid the C oracle chose) reproduces the C oracle
    bit for bit, also where refined depth planes need scaling, and its
    transpose and the chain's gradients equal the oracle's to 1e-9;
  * on the benchmark's own MWDG2 grid (1024 x 1024, 10 levels), which the
    oracle cannot run, central differences of the FP64 forward converge to
    the FP64 gradients and FP32 tracks FP64.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import dg2_adjoint_nonuniform as AS
from paper_2107_02750_gb300 import synth as S

from util import oracle_sim

pytestmark = pytest.mark.gpu

TOL = 1e-9


def static_reach(n, Ls, eps):
    p, _ = S.adjoint_reach(n=n)
    return replace(p, mode=S.STATIC, L=Ls, M=n >> Ls, N=n >> Ls, eps=eps)


def adaptive_reach(n, Ls, eps):
    p, _ = S.adjoint_reach(n=n)
    return replace(p, mode=S.ADAPTIVE, L=Ls, M=n >> Ls, N=n >> Ls, eps=eps)


def context(p, lev, ii, jj, K, precision=0):
    from paper_2107_02750_gb300.adjoint import Dg2Adjoint
    return Dg2Adjoint.frozen(p.M, p.N, p.L, p.dx, p.mode, lev, ii, jj, cfl=p.cfl, dt_max=p.dt_max,
                             limiter=p.limiter, bc=tuple(p.bc), inflow_edge=p.inflow_edge, inflow_c0=p.inflow_c0,
                             inflow_c1=p.inflow_c1, rain_rate=p.rain_rate, rain_t_end=p.rain_t_end, max_steps=K,
                             precision=precision)


def grid_of(p, lev, ii, jj):
    mode = "static" if p.mode == S.STATIC else "adaptive"
    return AS.grid_from_leaves(p.M, p.N, p.L, p.dx, lev, ii, jj, mode=mode, bc=p.bc, inflow_edge=p.inflow_edge,
                               inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, rain_rate=p.rain_rate,
                               rain_t_end=p.rain_t_end, knot_t=list(map(float, p.inflow_t)))


def device_inputs(adj, s, p, c0):
    """leaf coefficients (9, n_leaves), the oracle's finest bed planes, the
    finest Manning raster and the knots"""
    import torch
    dev = adj.device
    U0 = torch.tensor(np.ascontiguousarray(c0.T), dtype=adj.dtype, device=dev)
    z = torch.tensor(s.z_level(p.L)[0].reshape(3, p.ny, p.nx), dtype=adj.dtype, device=dev)
    n = torch.tensor(p.n_cell(), dtype=adj.dtype, device=dev)
    kt = torch.tensor(p.inflow_t, dtype=torch.float64, device=dev)
    kQ = torch.tensor(p.inflow_Q, dtype=torch.float64, device=dev)
    return U0, z, n, kt, kQ


def start(p):
    """the oracle at the segment's start: a static grid as built, an MWDG2
    grid after one regridding (with a step of 0.8 times its CFL choice)"""
    s = oracle_sim(p)
    dt = None
    if p.mode == S.ADAPTIVE:
        s.adapt()
        probe = oracle_sim(p)
        dt = probe.step()
    return s, dt


STATIC = [("static_32_L3", static_reach(32, 3, 5e-2)), ("static_64_L5", static_reach(64, 5, 1e-1))]
FROZEN = [("mwdg2_32_L3", adaptive_reach(32, 3, 5e-2)), ("mwdg2_64_L4", adaptive_reach(64, 4, 2e-2))]


@pytest.mark.parametrize("name,p", STATIC, ids=[c[0] for c in STATIC])
def test_static_forward_is_the_c_oracle_bit_for_bit(name, p):
    K = 8
    s, _ = start(p)
    lev, ii, jj, c0 = s.leaves()
    assert len(np.unique(lev)) >= 3
    dts = np.array([s.step() for _ in range(K)])
    _, _, _, cK = s.leaves()
    adj = context(p, lev, ii, jj, K)
    U0, z, n, kt, kQ = device_inputs(adj, s, p, c0)
    UK, d = adj.forward(U0, z, n, kt, kQ, 0.0, K)
    assert np.array_equal(d.cpu().numpy(), dts)
    got = UK.cpu().numpy().T
    assert np.array_equal(got, cK), np.abs(got - cK).max()
    assert (cK[:, 3] != c0[:, 3]).any()


@pytest.mark.parametrize("name,p", FROZEN, ids=[c[0] for c in FROZEN])
def test_frozen_mwdg2_forward_is_the_c_oracle_bit_for_bit(name, p):
    K = 8
    s, dt_cfl = start(p)
    lev, ii, jj, c0 = s.leaves()
    assert len(np.unique(lev)) >= 2
    dts = [0.8 * dt_cfl] * K
    for d in dts:
        s.step_frozen(d)
    l2, _, _, cK = s.leaves()
    assert np.array_equal(l2, lev)
    adj = context(p, lev, ii, jj, K)
    import torch
    U0, z, n, kt, kQ = device_inputs(adj, s, p, c0)
    UK, _ = adj.forward(U0, z, n, kt, kQ, 0.0, K, dts=torch.tensor(dts, dtype=torch.float64, device=adj.device))
    got = UK.cpu().numpy().T
    assert np.array_equal(got, cK), np.abs(got - cK).max()
    # the first step's CFL choice over the frozen grid's leaves
    _, d1 = adj.forward(U0, z, n, kt, kQ, 0.0, 1)
    assert float(d1[0]) == dt_cfl


def oracle_gradients(G, c0, zpl, nf, Q, dts, W):
    """reverse-mode gradients of sum(W * leaves after the steps) from the
    non-uniform oracle, with respect to the leaves' coefficients, the finest
    bed planes, the finest Manning raster and the knots"""
    import torch

    def leaf(a):
        return torch.tensor(np.array(a, dtype=np.float64), requires_grad=True)
    coef, zp, nn, QQ = leaf(c0), leaf(zpl), leaf(nf), leaf(Q)
    U = AS.dense_from_leaves(coef, G)
    zc = AS.pyramid([zp[0], zp[1], zp[2]], G.L)
    nm = AS.manning_levels(nn, G.L)
    t = 0.0
    for dt in dts:
        U = AS.step(U, zc, nm, QQ, float(dt), t, G)
        t = t + float(dt)
    out = AS.leaves_of(U, G)
    (out * torch.as_tensor(W)).sum().backward()
    return out.detach().numpy(), coef.grad.numpy(), zp.grad.numpy(), nn.grad.numpy(), QQ.grad.numpy()


def _close(got, want, what):
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want).max()
    assert err <= TOL * scale, (what, err, scale)


@pytest.mark.parametrize("name,p", STATIC + FROZEN, ids=[c[0] for c in STATIC + FROZEN])
def test_gradients_match_the_oracle(name, p):
    import torch
    K = 6
    s, dt_cfl = start(p)
    lev, ii, jj, c0 = s.leaves()
    dts = [s.step() for _ in range(K)] if p.mode == S.STATIC else [0.8 * dt_cfl] * K
    G = grid_of(p, lev, ii, jj)
    W = np.random.default_rng(13).standard_normal((len(lev), 9))
    zpl = s.z_level(p.L)[0].reshape(3, p.ny, p.nx)
    out, gc, gzo, gno, gQo = oracle_gradients(G, c0, zpl, p.n_cell(), p.inflow_Q, dts, W)
    adj = context(p, lev, ii, jj, K)
    U0, z, n, kt, kQ = device_inputs(adj, s, p, c0)
    d = torch.tensor(dts, dtype=torch.float64, device=adj.device)
    UK, _ = adj.forward(U0, z, n, kt, kQ, 0.0, K, dts=d)
    assert np.array_equal(UK.cpu().numpy().T, out)
    gU0, gz, gn, gQ = adj.backward(U0, z, n, kt, kQ, 0.0, d, torch.tensor(np.ascontiguousarray(W.T),
                                                                            device=adj.device))
    _close(gU0.cpu().numpy().T, gc, "U0")
    _close(gz.cpu().numpy(), gzo, "z")
    _close(gn.cpu().numpy(), gno, "n")
    _close(gQ.cpu().numpy(), gQo, "Q")
    for g in (gc, gzo, gno, gQo):
        assert np.abs(g).max() > 0
    # the tape of the forward call, reused, gives the same gradients
    UK, _ = adj.forward(U0, z, n, kt, kQ, 0.0, K, dts=d)
    gU0r, gzr, gnr, gQr = adj.backward(U0, z, n, kt, kQ, 0.0, d, torch.tensor(np.ascontiguousarray(W.T),
                                                                                device=adj.device),
                                       reuse_tape=True)
    assert torch.equal(gU0r, gU0) and torch.equal(gzr, gz) and torch.equal(gnr, gn) and torch.equal(gQr, gQ)


def test_all_finest_leaves_equal_the_uniform_context_bit_for_bit():
    """A frozen grid whose leaves all sit on the finest level is the uniform
    grid: the same run and the same gradients, bit for bit."""
    import torch
    from paper_2107_02750_gb300.adjoint import Dg2Adjoint
    p0, _ = S.adjoint_reach(n=32)
    p = replace(p0, mode=S.STATIC, M=4, N=4, L=3)
    K = 12
    jj, ii = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    lev = np.full(32 * 32, 3, dtype=np.int32)
    fz = context(p, lev, ii.ravel(), jj.ravel(), K)
    un = Dg2Adjoint(32, 32, p.dx, cfl=p.cfl, dt_max=p.dt_max, limiter=p.limiter, bc=tuple(p.bc),
                    inflow_edge=p.inflow_edge, inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, max_steps=K)
    U0 = torch.cat([un.project(p.h_vert), un.project(p.qx_vert), un.project(p.qy_vert)])
    z = un.project(p.z_vert)
    n = torch.tensor(p.n_cell(), dtype=torch.float64, device=un.device)
    kt = torch.tensor(p.inflow_t, dtype=torch.float64, device=un.device)
    kQ = torch.tensor(p.inflow_Q, dtype=torch.float64, device=un.device)
    UKu, du = un.forward(U0, z, n, kt, kQ, 0.0, K)
    UKf, df = fz.forward(U0.reshape(9, -1), z, n, kt, kQ, 0.0, K)
    assert torch.equal(du, df)
    assert torch.equal(UKu.reshape(9, -1), UKf)
    seed = torch.tensor(np.random.default_rng(5).standard_normal((9, 32, 32)), device=un.device)
    gu = un.backward(U0, z, n, kt, kQ, 0.0, du, seed)
    gf = fz.backward(U0.reshape(9, -1), z, n, kt, kQ, 0.0, df, seed.reshape(9, -1))
    assert torch.equal(gu[0].reshape(9, -1), gf[0])
    for a, b in zip(gu[1:], gf[1:]):
        assert torch.equal(a, b)


def test_chained_segments_equal_one_segment():
    """Two autograd segments of a frozen MWDG2 grid (the second checkpointed
    at the first's end) give the gradients of one segment over both."""
    import torch
    from paper_2107_02750_gb300.adjoint import dg2_run
    p = adaptive_reach(32, 3, 5e-2)
    s, dt_cfl = start(p)
    lev, ii, jj, c0 = s.leaves()
    K1, K2 = 4, 5
    adj1 = context(p, lev, ii, jj, K1 + K2)
    U0, z, n, kt, kQ = device_inputs(adj1, s, p, c0)
    dts = torch.full((K1 + K2,), 0.8 * dt_cfl, dtype=torch.float64, device=adj1.device)
    W = torch.tensor(np.random.default_rng(2).standard_normal((9, len(lev))), device=adj1.device)

    def grads(segments):
        u, zz, nn, Q = (x.clone().requires_grad_(True) for x in (U0, z, n, kQ))
        x, t, k0 = u, 0.0, 0
        for adj, K in segments:
            x, _, t = dg2_run(adj, x, zz, nn, Q, kt, t, K, dts[k0:k0 + K])
            k0 += K
        (x * W).sum().backward()
        return [a.grad for a in (u, zz, nn, Q)]

    one = grads([(adj1, K1 + K2)])
    adj2 = context(p, lev, ii, jj, K2)
    two = grads([(adj1, K1), (adj2, K2)])
    for a, b in zip(one, two):
        scale = float(a.abs().max())
        assert scale > 0 and float((a - b).abs().max()) <= 1e-12 * scale


def test_fp32_tracks_the_fp64_oracle():
    import torch
    p = static_reach(64, 5, 1e-1)
    K = 6
    s, _ = start(p)
    lev, ii, jj, c0 = s.leaves()
    dts = [s.step() for _ in range(K)]
    G = grid_of(p, lev, ii, jj)
    W = np.random.default_rng(21).standard_normal((len(lev), 9))
    zpl = s.z_level(p.L)[0].reshape(3, p.ny, p.nx)
    out, gc, gzo, gno, _ = oracle_gradients(G, c0, zpl, p.n_cell(), p.inflow_Q, dts, W)
    adj = context(p, lev, ii, jj, K, precision=1)
    U0, z, n, kt, kQ = device_inputs(adj, s, p, c0)
    UK, d = adj.forward(U0, z, n, kt, kQ, 0.0, K)
    assert np.allclose(d.cpu().numpy(), dts, rtol=2e-3, atol=0)
    d64 = torch.tensor(dts, dtype=torch.float64, device=adj.device)
    UK, _ = adj.forward(U0, z, n, kt, kQ, 0.0, K, dts=d64)
    assert np.abs(UK.cpu().numpy().T[:, 0] - out[:, 0]).max() <= 1e-4
    gU0, gz, gn, _ = adj.backward(U0, z, n, kt, kQ, 0.0, d64, torch.tensor(np.ascontiguousarray(W.T),
                                                                             dtype=torch.float32,
                                                                             device=adj.device))
    for got, want in ((gU0.cpu().numpy().T, gc), (gz.cpu().numpy(), gzo), (gn.cpu().numpy(), gno)):
        g, w = got.ravel().astype(np.float64), want.ravel()
        assert np.corrcoef(g, w)[0, 1] >= 0.999
        assert np.quantile(np.abs(g - w), 0.99) <= 0.02 * np.abs(w).max()


def _segment(coef, zc, nm, Q, dts, t0, G):
    import torch
    U = AS.dense_from_leaves(coef, G)
    t = t0
    for dt in dts:
        U = AS.step(U, zc, nm, Q, float(dt), t, G)
        t = t + float(dt)
    return AS.leaves_of(U, G)


def test_refrozen_segments_match_the_oracles():
    """Two frozen MWDG2 segments with the grid re-frozen between them
    (mwdg_adj_regrid: the adaptation's state transfer to the grid the C
    oracle chose): the run is the C oracle's bit for bit, and the gradients
    of the chain (dg2_run, regrid, dg2_run through autograd) equal the
    non-uniform oracle's to 1e-9."""
    import torch
    from paper_2107_02750_gb300.adjoint import dg2_run, regrid
    p = adaptive_reach(32, 3, 5e-2)
    s, dt_cfl = start(p)
    dt = 0.8 * dt_cfl
    l1, i1, j1, c0 = s.leaves()
    K1, K2 = 4, 4
    for _ in range(K1):
        s.step_frozen(dt)
    s.adapt()
    l2, i2, j2, cm = s.leaves()
    for _ in range(K2):
        s.step_frozen(dt)
    cK = s.leaves()[3]
    G1, G2 = grid_of(p, l1, i1, j1), grid_of(p, l2, i2, j2)
    assert sum(int((G1.leaf[l] != G2.leaf[l]).sum()) for l in range(p.L + 1)) > 0
    a1, a2 = context(p, l1, i1, j1, K1), context(p, l2, i2, j2, K2)
    U0, z, n, kt, kQ = device_inputs(a1, s, p, c0)
    d1 = torch.full((K1,), dt, dtype=torch.float64, device=a1.device)
    d2 = torch.full((K2,), dt, dtype=torch.float64, device=a1.device)
    W = np.random.default_rng(23).standard_normal((len(l2), 9))
    u, zz, nn, Q = (x.clone().requires_grad_(True) for x in (U0, z, n, kQ))
    x, _, t = dg2_run(a1, u, zz, nn, Q, kt, 0.0, K1, d1)
    xm = regrid(a1, a2, x)
    assert np.array_equal(xm.detach().cpu().numpy().T, cm)
    y, _, _ = dg2_run(a2, xm, zz, nn, Q, kt, t, K2, d2)
    assert np.array_equal(y.detach().cpu().numpy().T, cK)
    (y * torch.tensor(np.ascontiguousarray(W.T), device=a1.device)).sum().backward()

    def leaf(a):
        return torch.tensor(np.array(a, dtype=np.float64), requires_grad=True)
    coef, zp, nf, QQ = leaf(c0), leaf(s.z_level(p.L)[0].reshape(3, p.ny, p.nx)), leaf(p.n_cell()), leaf(p.inflow_Q)
    zc = AS.pyramid([zp[0], zp[1], zp[2]], p.L)
    nm = AS.manning_levels(nf, p.L)
    mid = _segment(coef, zc, nm, QQ, [dt] * K1, 0.0, G1)
    out = _segment(AS.regrid(mid, G1, G2), zc, nm, QQ, [dt] * K2, K1 * dt, G2)
    (out * torch.as_tensor(W)).sum().backward()
    _close(u.grad.cpu().numpy().T, coef.grad.numpy(), "U0")
    _close(zz.grad.cpu().numpy(), zp.grad.numpy(), "z")
    _close(nn.grad.cpu().numpy(), nf.grad.numpy(), "n")
    _close(Q.grad.cpu().numpy(), QQ.grad.numpy(), "Q")


def test_regrid_with_refined_depth_planes_matches_the_oracles():
    """The transfer where the new grid refines coarse, partly wet leaves whose
    depth planes need scaling (a dam break over a steep dry slope): the C
    oracle's adaptation bit for bit, and the transpose equal to the
    oracle's reverse-mode derivative to 1e-9."""
    import torch
    from paper_2107_02750_gb300.adjoint import regrid_forward, regrid_transpose
    from test_oracle_adjoint_nonuniform import steep_slope_adaptive, _refined_below_negative
    p = steep_slope_adaptive()
    s = oracle_sim(p)
    for _ in range(2):
        dt = s.step()
        for _ in range(3):
            s.step_frozen(dt)
        s.adapt()
    s.step()
    for _ in range(3):
        s.step_frozen(dt)
    l1, i1, j1, cb = s.leaves()
    s.adapt()
    l2, i2, j2, ca = s.leaves()
    G1, G2 = grid_of(p, l1, i1, j1), grid_of(p, l2, i2, j2)
    assert _refined_below_negative(cb, G1, G2) > 0
    a1, a2 = context(p, l1, i1, j1, 1), context(p, l2, i2, j2, 1)
    U = torch.tensor(np.ascontiguousarray(cb.T), device=a1.device)
    V = regrid_forward(a1, a2, U)
    assert np.array_equal(V.cpu().numpy().T, ca)
    W = np.random.default_rng(29).standard_normal((len(l2), 9))
    g = regrid_transpose(a1, a2, U, torch.tensor(np.ascontiguousarray(W.T), device=a1.device))
    coef = torch.tensor(cb, requires_grad=True)
    (AS.regrid(coef, G1, G2) * torch.as_tensor(W)).sum().backward()
    _close(g.cpu().numpy().T, coef.grad.numpy(), "U")


def test_full_size_frozen_mwdg2_gradients():
    """The benchmark's own grid: the 1024 x 1024 valley's MWDG2 leaves and
    state after 600 s of the FP64 solver, frozen, one 10-step segment with a
    seeded functional of the leaves.  The oracle cannot run this size, so
    properties that hold at any size stand in: central differences of the
    FP64 forward (steps held, 1e-6 to 1e-8) converge to the FP64 gradients
    at sampled depth coefficients of wet leaves and Manning entries of wet
    finest cells, and the FP32 gradients track the FP64 ones (correlation
    >= 0.999)."""
    import torch
    import paper_2107_02750_gb300 as M
    p = S.valley(n=1024, L=10)
    sol = M.solver_from_problem(p, precision=M.F64)
    sol.run_to_time(600.0)
    t0 = sol.get_time()[0]
    lev, ii, jj, co = sol.read_active()
    del sol
    K = 10
    out = {}
    for precision in (M.F64, M.F32):
        adj = context(p, lev, ii, jj, K, precision=precision)
        dev = adj.device
        U0 = torch.tensor(np.ascontiguousarray(co.T), dtype=adj.dtype, device=dev)
        z = adj.project(p.z_vert)
        n = torch.tensor(p.n_cell(), dtype=adj.dtype, device=dev)
        kt = torch.tensor(p.inflow_t, dtype=torch.float64, device=dev)
        kQ = torch.tensor(p.inflow_Q, dtype=torch.float64, device=dev)
        if precision == M.F64:
            _, d = adj.forward(U0, z, n, kt, kQ, t0, K)
        seed = torch.zeros((9, len(lev)), dtype=adj.dtype, device=dev)
        seed[0] = torch.randn(len(lev), generator=torch.Generator().manual_seed(4)).to(seed)
        out[precision] = (adj, U0, z, n, kt, kQ, seed, adj.backward(U0, z, n, kt, kQ, t0, d, seed))
        del adj
    adj, U0, z, n, kt, kQ, seed, (gU0, gz, gn, gQ) = out[M.F64]

    def J(U0_=U0, n_=n):
        UK, _ = adj.forward(U0_, z, n_, kt, kQ, t0, K, dts=d)
        return float((UK * seed).sum())

    def best(ad, arr, idx, scale, which):
        fs = []
        for rel in (1e-6, 1e-7, 1e-8):
            a, b = arr.clone(), arr.clone()
            a[idx] += rel * scale
            b[idx] -= rel * scale
            fs.append((J(**{which: a}) - J(**{which: b})) / (2.0 * rel * scale))
        return min(fs, key=lambda f: abs(f - ad))

    rng = np.random.default_rng(31)
    gh, gnn = gU0.cpu().numpy()[0], gn.cpu().numpy()
    h0 = co[:, 0]
    checks = []
    cand = np.flatnonzero((np.abs(gh) > 1e-2 * np.abs(gh).max()) & (h0 > 0.05))
    for q in rng.choice(cand, 3, replace=False):
        ad = float(gh[q])
        checks.append(("U0", ad, best(ad, U0, (0, int(q)), 1.0, "U0_")))
    # Manning n: finest cells under wet finest-level leaves
    fine = np.flatnonzero((lev == p.L) & (h0 > 0.05))
    cells = [(int(jj[q]), int(ii[q])) for q in fine]
    gcell = np.array([gnn[j, i] for j, i in cells])
    big = np.flatnonzero(np.abs(gcell) > 1e-2 * np.abs(gnn).max())
    for c in rng.choice(big, 2, replace=False):
        j, i = cells[int(c)]
        ad = float(gnn[j, i])
        checks.append(("n", ad, best(ad, n, (j, i), float(n[j, i]), "n_")))
    for what, ad, f in checks:
        assert abs(ad - f) <= 1e-4 * abs(ad), (what, ad, f)
    g32 = out[M.F32][-1]
    for a, b, what in zip(g32[:3], (gU0, gz, gn), ("U0", "z", "n")):
        x, y = a.double().cpu().numpy().ravel(), b.cpu().numpy().ravel()
        assert np.corrcoef(x, y)[0, 1] >= 0.999, what
