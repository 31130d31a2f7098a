"""Discrete adjoint of the uniform DG2 step on the GPU (include/mwdg_adjoint.h)
against the FP64 oracle (oracle/dg2_adjoint.py, pinned on the CPU).

  * the adjoint's forward sweep is the C oracle's step bit for bit (states
    and CFL time steps), through wet/dry fronts, inflow, an open edge, rain;
  * its gradients with respect to U0, the bed planes, Manning n and the
    hydrograph knots agree with the oracle's to 1e-9 of each array's largest
    entry (same branches, different rounding order in the reverse sweep);
  * the bed's vertex gradient (transpose of Eq. 8) agrees likewise;
  * two checkpointed segments chained by autograd give the one-segment
    gradients;
  * central differences of the GPU forward (time steps held), with steps
    shrinking to 1e-8, converge to the GPU gradients (1e-4 relative);
  * the FP32 adjoint tracks the FP64 oracle: time steps to 2e-3 each,
    depths to 1e-4 m, gradients correlated above 0.999 with 99 % of entries within 2 %
    of the array's largest and none beyond 5 % (wet/dry tests that FP32
    rounding flips move single cells).
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import dg2_adjoint as A
from paper_2107_02750_gb300 import synth as S

from util import oracle_sim

pytestmark = pytest.mark.gpu

TOL = 1e-9


def grid_of(p):
    return A.Grid(nx=p.nx, ny=p.ny, dx=p.dx, limiter=p.limiter, bc=tuple(p.bc), inflow_edge=p.inflow_edge,
                  inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, rain_rate=p.rain_rate,
                  rain_t_end=p.rain_t_end, knot_t=list(map(float, p.inflow_t)))


def state(sim, p):
    _, _, _, co = sim.leaves()
    return co.T.reshape(9, p.ny, p.nx).copy()


def context(p, max_steps, precision=0, tape_views=False):
    from paper_2107_02750_gb300.adjoint import Dg2Adjoint
    return Dg2Adjoint(p.nx, p.ny, p.dx, cfl=p.cfl, dt_max=p.dt_max, limiter=p.limiter, bc=tuple(p.bc),
                      inflow_edge=p.inflow_edge, inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1,
                      rain_rate=p.rain_rate, rain_t_end=p.rain_t_end, max_steps=max_steps, precision=precision,
                      tape_views=tape_views)


def device_inputs(adj, p):
    """the GPU's own projection of the seeded vertex rasters (Eq. 8)"""
    import torch
    U0 = torch.cat([adj.project(p.h_vert), adj.project(p.qx_vert), adj.project(p.qy_vert)])
    z = adj.project(p.z_vert)
    n = torch.tensor(p.n_cell(), dtype=adj.dtype, device=adj.device)
    if p.inflow_edge >= 0:
        kt = torch.tensor(p.inflow_t, dtype=torch.float64, device=adj.device)
        kQ = torch.tensor(p.inflow_Q, dtype=torch.float64, device=adj.device)
    else:
        kt = kQ = None
    return U0, z, n, kt, kQ


def _cases():
    reach, gauges = S.adjoint_reach(n=32)
    rain = replace(reach, rain_rate=5e-3, rain_t_end=8.0)
    dam = S.dam_break_circular(n=32, L=0, radius=6.0, h_out=0.0)
    crop, _ = S.adjoint_reach(n=64, crop_of=1024)
    # rectangular, sides not multiples of the 16 x 16 update tile
    rect = S.crop(S.adjoint_reach(n=64)[0], 0, 18, 40, 28, 0)
    return [("reach", reach, 40), ("reach_rain", rain, 30), ("dam_dry", dam, 40), ("valley_crop64", crop, 40),
            ("rect_40x28", rect, 30)]


CASES = _cases()


@pytest.mark.parametrize("name,p,K", CASES, ids=[c[0] for c in CASES])
def test_forward_sweep_is_the_c_oracle_bit_for_bit(name, p, K):
    s = oracle_sim(p)
    U0o = state(s, p)
    zo = s.z_level(0)[0].reshape(3, p.ny, p.nx)
    dts = np.array([s.step() for _ in range(K)])
    want = state(s, p)
    adj = context(p, K)
    U0, z, n, kt, kQ = device_inputs(adj, p)
    assert np.array_equal(U0.cpu().numpy(), U0o) and np.array_equal(z.cpu().numpy(), zo)
    UK, d = adj.forward(U0, z, n, kt, kQ, 0.0, K)
    assert np.array_equal(d.cpu().numpy(), dts)
    got = UK.cpu().numpy()
    assert np.array_equal(got, want), np.abs(got - want).max()
    # the same run with the steps given
    UK2, _ = adj.forward(U0, z, n, kt, kQ, 0.0, K, dts=d)
    assert np.array_equal(UK2.cpu().numpy(), want)


def _close(got, want, what):
    scale = max(np.abs(want).max(), 1e-300)
    err = np.abs(got - want).max()
    assert err <= TOL * scale, (what, err, scale)


@pytest.mark.parametrize("name,p,K", CASES, ids=[c[0] for c in CASES])
def test_gradients_match_the_oracle(name, p, K):
    import torch
    s = oracle_sim(p)
    U0o = state(s, p)
    zo = s.z_level(0)[0].reshape(3, p.ny, p.nx)
    dts = [s.step() for _ in range(K)]
    rng = np.random.default_rng(11)
    seed = rng.standard_normal((9, p.ny, p.nx))
    Q = p.inflow_Q if p.inflow_edge >= 0 else np.zeros(1)
    G = A.gradients(U0o, zo, p.n_cell(), Q, dts, 0.0, grid_of(p), seed, z_vert=p.z_vert)
    adj = context(p, K)
    U0, z, n, kt, kQ = device_inputs(adj, p)
    d = torch.tensor(dts, dtype=torch.float64, device=adj.device)
    gU0, gz, gn, gQ = adj.backward(U0, z, n, kt, kQ, 0.0, d, torch.tensor(seed, device=adj.device))
    _close(gU0.cpu().numpy(), G["gU0"], "U0")
    _close(gz.cpu().numpy(), G["gz"], "z")
    _close(gn.cpu().numpy(), G["gn"], "n")
    if p.inflow_edge >= 0:
        _close(gQ.cpu().numpy(), G["gQ"], "Q")
    _close(adj.project_transpose(gz).cpu().numpy(), G["gzv"], "z vertices")


def test_checkpointed_segments_chain_to_the_one_segment_gradient():
    """Gauge objective after 40 steps: one segment of 40, or four of 10
    chained by autograd (each backward recomputes its segment from its input
    state)."""
    import torch
    from paper_2107_02750_gb300.adjoint import dg2_run
    p, gauges = S.adjoint_reach(n=32)
    adj = context(p, 40)
    U0, z, n, kt, kQ = device_inputs(adj, p)

    def grads(seg):
        leaves = [x.clone().requires_grad_(True) for x in (U0, z, n, kQ)]
        U, t = leaves[0], 0.0
        for _ in range(40 // seg):
            U, _, t = dg2_run(adj, U, leaves[1], leaves[2], leaves[3], kt, t, seg)
        J = sum(U[0, j, i] for j, i in gauges)
        J.backward()
        return [x.grad.cpu().numpy() for x in leaves], U.detach().cpu().numpy()

    (g1, U1), (g4, U4) = grads(40), grads(10)
    assert np.array_equal(U1, U4)
    for a, b, what in zip(g1, g4, ("U0", "z", "n", "Q")):
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(a).max(), 1e-300), what
    assert np.abs(g1[2]).max() > 0 and np.abs(g1[3]).max() > 0


def test_gpu_gradients_match_central_differences_of_the_gpu_forward():
    """The run is piecewise smooth: a wet/dry test, a minmod pick or the
    inflow ghost's max can switch within 1e-7 (relative) of the base point
    near the inlet, and a difference whose step straddles such a switch
    mixes two branches.  Each check therefore takes steps of 1e-6, 1e-7 and
    1e-8 (relative to the parameter, or metres) and requires the closest
    difference to agree with the gradient to 1e-4: the differences converge
    to it as the step shrinks below the nearest switch."""
    import torch
    p, gauges = S.adjoint_reach(n=32)
    K = 40
    adj = context(p, K)
    U0, z, n, kt, kQ = device_inputs(adj, p)
    _, d = adj.forward(U0, z, n, kt, kQ, 0.0, K)
    seed = torch.zeros((9, p.ny, p.nx), dtype=torch.float64, device=adj.device)
    for j, i in gauges:
        seed[0, j, i] += 1.0
    gU0, gz, gn, gQ = adj.backward(U0, z, n, kt, kQ, 0.0, d, seed)

    def J(U0_=U0, z_=z, n_=n, kQ_=kQ):
        UK, _ = adj.forward(U0_, z_, n_, kt, kQ_, 0.0, K, dts=d)
        return float((UK * seed).sum())

    def fd_best(ad, arr, idx, scale, which):
        best = None
        for rel in (1e-6, 1e-7, 1e-8):
            delta = rel * scale
            a, b = arr.clone(), arr.clone()
            a[idx] += delta
            b[idx] -= delta
            f = (J(**{which: a}) - J(**{which: b})) / (2.0 * delta)
            if best is None or abs(f - ad) < abs(best - ad):
                best = f
        return best

    checks = []
    gnn = gn.cpu().numpy()
    for j, i in np.argwhere(np.abs(gnn) > 1e-2 * np.abs(gnn).max())[::9][:4]:
        checks.append(("n", gnn[j, i], fd_best(gnn[j, i], n, (j, i), float(n[j, i]), "n_")))
    gzz = gz.cpu().numpy()
    for j, i in np.argwhere(np.abs(gzz[0]) > 1e-2 * np.abs(gzz[0]).max())[::13][:4]:
        checks.append(("z0", gzz[0, j, i], fd_best(gzz[0, j, i], z, (0, j, i), 1.0, "z_")))
    for k in (0, 1):
        gq = float(gQ[k])
        checks.append(("Q", gq, fd_best(gq, kQ, (k,), float(kQ[k]), "kQ_")))
    gh = gU0.cpu().numpy()
    for j, i in np.argwhere(np.abs(gh[0]) > 1e-2 * np.abs(gh[0]).max())[::11][:3]:
        checks.append(("h0", gh[0, j, i], fd_best(gh[0, j, i], U0, (0, j, i), 1.0, "U0_")))
    assert len(checks) >= 10
    for what, ad, f in checks:
        assert ad != 0.0, what
        assert abs(ad - f) <= 1e-4 * abs(ad), (what, ad, f)


def test_gauge_misfit_gradient_descends():
    """Squared depth misfit at the 16 gauges after two checkpoint segments
    against observations from a run with a rougher channel (n x 1.3): a
    small step against the Manning gradient lowers the misfit."""
    import torch
    from paper_2107_02750_gb300.adjoint import dg2_run
    p, gauges = S.adjoint_reach(n=64, crop_of=1024)
    adj = context(p, 20)
    U0, z, n, kt, kQ = device_inputs(adj, p)
    gj = torch.tensor(gauges[:, 0], device=adj.device)
    gi = torch.tensor(gauges[:, 1], device=adj.device)

    def run(nn, grad=False):
        nn = nn.clone().requires_grad_(grad)
        U, t, J = U0, 0.0, 0.0
        for s in range(2):
            U, _, t = dg2_run(adj, U, z, nn, kQ, kt, t, 20)
            J = J + ((U[0, gj, gi] - obs[s]) ** 2).sum()
        return J, nn

    obs, U, t = [], U0, 0.0
    for s in range(2):
        U, _, t = dg2_run(adj, U, z, 1.3 * n, kQ, kt, t, 20)
        obs.append(U[0, gj, gi].detach().clone())
    J0, nn = run(n, grad=True)
    J0.backward()
    g = nn.grad
    assert float(g.abs().max()) > 0.0
    step = 1e-3 * float(n.abs().max()) / float(g.abs().max())
    J1, _ = run(n - step * g)
    assert float(J1) < float(J0), (float(J1), float(J0))


@pytest.mark.parametrize("name,p,K", CASES, ids=[c[0] for c in CASES])
def test_f32_adjoint_tracks_the_fp64_oracle(name, p, K):
    import torch
    s = oracle_sim(p)
    U0o = state(s, p)
    zo = s.z_level(0)[0].reshape(3, p.ny, p.nx)
    dts = [s.step() for _ in range(K)]
    want = state(s, p)
    seed = np.random.default_rng(11).standard_normal((9, p.ny, p.nx))
    Q = p.inflow_Q if p.inflow_edge >= 0 else np.zeros(1)
    G = A.gradients(U0o, zo, p.n_cell(), Q, dts, 0.0, grid_of(p), seed)
    adj = context(p, K, precision=1)
    U0, z, n, kt, kQ = device_inputs(adj, p)
    assert U0.dtype == torch.float32
    UK, d = adj.forward(U0, z, n, kt, kQ, 0.0, K)
    # a step set by a thin, fast cell carries FP32's relative error in its speed
    assert np.all(np.abs(d.cpu().numpy() - np.array(dts)) <= 2e-3 * np.array(dts))
    assert np.abs(UK[0].double().cpu().numpy() - want[0]).max() <= 1e-4
    d64 = torch.tensor(dts, dtype=torch.float64, device=adj.device)
    gU0, gz, gn, gQ = adj.backward(U0, z, n, kt, kQ, 0.0, d64, torch.tensor(seed, dtype=torch.float32,
                                                                            device=adj.device))
    pairs = [("U0", gU0, G["gU0"]), ("z", gz, G["gz"]), ("n", gn, G["gn"])]
    if p.inflow_edge >= 0:
        pairs.append(("Q", gQ, G["gQ"]))
    for what, got, ref in pairs:
        a = got.double().cpu().numpy()
        scale = np.abs(ref).max()
        if scale == 0.0:
            assert np.abs(a).max() == 0.0, what
            continue
        err = np.abs(a - ref) / scale
        assert err.max() <= 5e-2, (what, err.max())
        assert np.quantile(err, 0.99) <= 2e-2, (what, np.quantile(err, 0.99))
        assert np.corrcoef(a.ravel(), ref.ravel())[0, 1] >= 0.999, what


def test_tape_reuse_gives_the_recomputed_gradients():
    """The backward may reuse the tape the forward left (reuse_tape), and the
    tape may keep each step's stage inputs and flux views (tape_views); the
    gradients equal those of a backward that recomputes everything from the
    checkpoint, bit for bit, in both precisions.  A tape of another length is
    refused."""
    import torch
    import paper_2107_02750_gb300 as M
    p, _ = S.adjoint_reach(n=32)
    ref = {}
    for precision, views in ((M.F64, False), (M.F32, False), (M.F64, True), (M.F32, True)):
        adj = context(p, 20, precision=precision, tape_views=views)
        U0, z, n, kt, kQ = device_inputs(adj, p)
        seed = torch.randn((9, p.ny, p.nx), generator=torch.Generator().manual_seed(3)).to(U0)
        _, d = adj.forward(U0, z, n, kt, kQ, 0.0, 20)
        a = adj.backward(U0, z, n, kt, kQ, 0.0, d, seed, reuse_tape=False)
        adj.forward(U0, z, n, kt, kQ, 0.0, 20, dts=d)
        b = adj.backward(U0, z, n, kt, kQ, 0.0, d, seed, reuse_tape=True)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        if precision in ref:
            for x, y in zip(ref[precision], a):
                assert torch.equal(x, y)
        ref[precision] = a
        adj.forward(U0, z, n, kt, kQ, 0.0, 10, dts=d[:10])
        with pytest.raises(M.MwdgError):
            adj.backward(U0, z, n, kt, kQ, 0.0, d, seed, reuse_tape=True)


def test_full_size_gradients():
    """The bench's workload, 1024 x 1024 valley with a flowing start, one
    20-step segment, gauge misfit seed.  The oracle cannot run this size, so
    properties that hold at any size stand in: central differences of the
    FP64 forward (steps held, 1e-6 to 1e-8) converge to the FP64 gradients
    at sampled Manning n, bed and depth entries of wet cells (a dry cell at
    h0 = 0 sits on the positivity clip's kink: a negative perturbation is
    clipped, a positive one is not, and a central difference takes half the
    one-sided slope); the FP32 gradients track the FP64 ones (correlation
    >= 0.999 over all cells)."""
    import torch
    import paper_2107_02750_gb300 as M
    p, gauges = S.adjoint_reach(n=1024, crop_of=1024)
    K = 20
    out = {}
    for precision in (M.F64, M.F32):
        adj = context(p, K, precision=precision)
        U0, z, n, kt, kQ = device_inputs(adj, p)
        if precision == M.F64:
            _, d = adj.forward(U0, z, n, kt, kQ, 0.0, K)
        seed = torch.zeros((9, p.ny, p.nx), dtype=adj.dtype, device=adj.device)
        seed[0] = torch.randn((p.ny, p.nx), generator=torch.Generator().manual_seed(9)).to(seed)
        out[precision] = (adj, U0, z, n, kt, kQ, seed, adj.backward(U0, z, n, kt, kQ, 0.0, d, seed))
    adj, U0, z, n, kt, kQ, seed, (gU0, gz, gn, gQ) = out[M.F64]

    def J(U0_=U0, z_=z, n_=n):
        UK, _ = adj.forward(U0_, z_, n_, kt, kQ, 0.0, K, dts=d)
        return float((UK * seed).sum())

    def best(ad, arr, idx, scale, which):
        fs = []
        for rel in (1e-6, 1e-7, 1e-8):
            a, b = arr.clone(), arr.clone()
            a[idx] += rel * scale
            b[idx] -= rel * scale
            fs.append((J(**{which: a}) - J(**{which: b})) / (2.0 * rel * scale))
        return min(fs, key=lambda f: abs(f - ad))

    rng = np.random.default_rng(21)
    gnn, gzz, ghh = gn.cpu().numpy(), gz.cpu().numpy(), gU0.cpu().numpy()
    checks = []
    wet = U0[0].cpu().numpy() > 0.05   # a dry cell at h0 = 0 sits on the clip's kink
    for arr, g, which, scale_of in ((n, gnn, "n_", lambda v: v), (z, gzz[0], "z_", lambda v: 1.0),
                                    (U0, ghh[0], "U0_", lambda v: 1.0)):
        idx = np.argwhere((np.abs(g) > 1e-2 * np.abs(g).max()) & wet)
        for j, i in idx[rng.choice(len(idx), 2, replace=False)]:
            full = (j, i) if which == "n_" else (0, j, i)
            ad = float(g[j, i])
            checks.append((which, ad, best(ad, arr, full, scale_of(float(arr[full])), which)))
    for what, ad, f in checks:
        assert abs(ad - f) <= 1e-4 * abs(ad), (what, ad, f)
    g32 = out[M.F32][-1]
    for a, b, what in zip(g32[:3], (gU0, gz, gn), ("U0", "z", "n")):
        x, y = a.double().cpu().numpy().ravel(), b.cpu().numpy().ravel()
        assert np.corrcoef(x, y)[0, 1] >= 0.999, what


def _strip(along_x):
    """a one-cell-wide dam break on a sloping, rough bed, along x or along y"""
    p = S.dam_break_strip(nx=64, ny=1, dx=0.5, h_left=1.0, h_right=0.1)
    z = np.tile(np.linspace(0.4, 0.0, 65), (2, 1))
    p = replace(p, z_vert=z, n_manning=0.03)
    if along_x:
        return p
    return replace(p, M=1, N=64, z_vert=np.ascontiguousarray(p.z_vert.T),
                   h_vert=np.ascontiguousarray(p.h_vert.T), qx_vert=np.ascontiguousarray(p.qy_vert.T),
                   qy_vert=np.ascontiguousarray(p.qx_vert.T))


@pytest.mark.parametrize("along_x", [True, False], ids=["strip_x", "strip_y"])
def test_one_cell_wide_strips(along_x):
    """64 x 1 and 1 x 64: one-sided limiting, a single row of update tiles;
    the forward sweep is the C oracle's bit for bit and the gradients are
    the oracle's (1e-9)."""
    import torch
    p = _strip(along_x)
    K = 30
    s = oracle_sim(p)
    U0o = state(s, p)
    zo = s.z_level(0)[0].reshape(3, p.ny, p.nx)
    dts = [s.step() for _ in range(K)]
    want = state(s, p)
    seed = np.random.default_rng(2).standard_normal((9, p.ny, p.nx))
    G = A.gradients(U0o, zo, p.n_cell(), np.zeros(1), dts, 0.0, grid_of(p), seed)
    adj = context(p, K)
    U0, z, n, kt, kQ = device_inputs(adj, p)
    UK, d = adj.forward(U0, z, n, kt, kQ, 0.0, K)
    assert np.array_equal(d.cpu().numpy(), np.array(dts))
    assert np.array_equal(UK.cpu().numpy(), want)
    gU0, gz, gn, _ = adj.backward(U0, z, n, kt, kQ, 0.0, d, torch.tensor(seed, device=adj.device))
    _close(gU0.cpu().numpy(), G["gU0"], "U0")
    _close(gz.cpu().numpy(), G["gz"], "z")
    _close(gn.cpu().numpy(), G["gn"], "n")


def test_degenerate_runs():
    """Zero steps: U_K = U0 and the cotangent passes through unchanged, with
    no bed, roughness or knot sensitivity.  An all-dry domain: nothing moves,
    the depth average's cotangent passes through (a dry cell keeps its
    average), everything else is zero."""
    import torch
    p, _ = S.adjoint_reach(n=32)
    adj = context(p, 10)
    U0, z, n, kt, kQ = device_inputs(adj, p)
    seed = torch.randn((9, p.ny, p.nx), generator=torch.Generator().manual_seed(4)).to(U0)
    UK, d = adj.forward(U0, z, n, kt, kQ, 0.0, 0)
    assert torch.equal(UK, U0) and d.numel() == 0
    gU0, gz, gn, gQ = adj.backward(U0, z, n, kt, kQ, 0.0, d, seed)
    assert torch.equal(gU0, seed)
    assert float(gz.abs().max()) == 0.0 and float(gn.abs().max()) == 0.0 and float(gQ.abs().max()) == 0.0
    dry = replace(p, h_vert=np.zeros_like(p.h_vert), qx_vert=np.zeros_like(p.h_vert),
                  qy_vert=np.zeros_like(p.h_vert), inflow_edge=-1)
    adj = context(dry, 10)
    U0, z, n, kt, kQ = device_inputs(adj, dry)
    UK, d = adj.forward(U0, z, n, kt, kQ, 0.0, 10)
    assert float(UK.abs().max()) == 0.0
    assert np.all(d.cpu().numpy() == dry.dt_max)
    gU0, gz, gn, _ = adj.backward(U0, z, n, kt, kQ, 0.0, d, seed)
    assert torch.equal(gU0[0], seed[0])
    assert float(gU0[1:].abs().max()) == 0.0
    assert float(gz.abs().max()) == 0.0 and float(gn.abs().max()) == 0.0
