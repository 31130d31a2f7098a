"""FP64 oracle of the discrete adjoint of the DG2 step on a frozen
non-uniform grid: a static graded grid, or an adaptive (MWDG2) grid held
fixed over a checkpoint segment.

TEST INFRASTRUCTURE ONLY.  Like the rest of ``oracle/``, this module is the
plain, slow reference that the CUDA library is checked against; only the tests
may import it, and the product package never imports or falls back to it.

What it computes.  The DG2 step of Sect. 2.1.1 (Eq. 1-4) on the active leaves
of a non-uniform grid, with the paper's rule on non-homogeneous interfaces:
every leaf evaluates its four faces from its own limits and its neighbour's
view at the leaf's own level.  That view is the neighbour leaf's limits; for
a neighbour below a coarser leaf, the prolongation of that leaf's planes down
to it (Eq. 10 with zero details); for a refined neighbour, on static grids
(Sect. 2.2.1, graded) the mean of the interface-centre limits of its two
children on the face, and on MWDG2 grids (Sect. 2.3) the local encoding of
its finer leaves' views (Eq. 9).  Friction, limiting (same-level leaf
neighbours only), revision, HLL, the RK2 stages and the positivity clip are
those of the uniform restatement in ``dg2_adjoint.py``, applied level by
level, in the C oracle's operation order, so that a run over given time
steps reproduces the C oracle bit for bit (its `orc_step_dt` on static grids,
`orc_step_frozen` on a frozen MWDG2 grid).  The bed pyramid, the Manning
means and (static grids) the initial state come from the inputs the C oracle
takes: DEM vertices (Eq. 8, then Eq. 9 up the levels), the finest Manning
raster (each coarser node the mean of its children), the initial vertex
rasters.  Each level is a dense array; positions that are not leaves carry
still water and are reset to it after every stage, so they never reach a
leaf.  The discrete adjoint is the derivative of this map by PyTorch's
reverse-mode automatic differentiation, with the readings of
``dg2_adjoint.py`` (time steps held at the recorded values, branches as
taken, the interface bed max split at ties, zero derivative of the Manning
speed at rest).  The static reflux rule is not restated (the paper rule
only).

`regrid` restates the state transfer of the MWDG2 adaptation between two
such grids (the C oracle's orc_adapt with the new grid it chose), so that a
run of frozen segments re-frozen at each checkpoint is differentiable.

Pinned by the tests against: the C oracle's steps over recorded time steps,
bit for bit; central differences of the C oracle's fixed-dt steps with
respect to DEM vertices, the Manning raster, initial depth vertices (static)
and hydrograph knots; the C oracle's adaptation (regrid) bit for bit, and
central differences of two frozen segments with the C oracle's regridding
between them; the refinement's invariants (children's depths non-negative,
the parent's average kept, planes with non-negative children unchanged).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .dg2_adjoint import (F64, S3, WALL, OPEN, _Cbrt, _TieMax, _safe, _shift, _w, drain_limit, face_lim, friction,
                          hll, inflow_Q, limit, post, project, revise)

HALF_S3 = 0.5 * S3


@dataclass
class LeafGrid:
    """A frozen non-uniform grid: M x N roots, L levels below them, finest
    cell size R; `leaf[l]` marks the active leaves of level l (row j south to
    north, column i west to east); mode "static" (graded, the static
    interface rule) or "adaptive" (MWDG2 views).  Physical parameters as in
    Grid."""
    M: int
    N: int
    L: int
    R: float
    leaf: list
    mode: str = "static"
    g: float = 9.80665
    hd: float = 1e-3
    limiter: int = 1
    bc: tuple = (WALL, WALL, WALL, WALL)
    inflow_edge: int = -1
    inflow_c0: int = 0
    inflow_c1: int = -1
    rain_rate: float = 0.0
    rain_t_end: float = 0.0
    knot_t: list = field(default_factory=list)

    def __post_init__(self):
        L = self.L
        self.leaf = [torch.as_tensor(np.asarray(a, dtype=bool)) for a in self.leaf]
        # refined: an ancestor of a leaf; below: covered by a coarser leaf
        sig = [None] * (L + 1)
        sig[L] = torch.zeros_like(self.leaf[L])
        for l in range(L - 1, -1, -1):
            d = self.leaf[l + 1] | sig[l + 1]
            ny, nx = d.shape
            sig[l] = d.reshape(ny // 2, 2, nx // 2, 2).any(dim=3).any(dim=1)
        self.sig = sig
        self.below = [~(self.leaf[l] | sig[l]) for l in range(L + 1)]

    def nx(self, l):
        return self.M << l

    def ny(self, l):
        return self.N << l

    def dx(self, l):
        return self.R * float(1 << (self.L - l))


def grid_from_leaves(M, N, L, R, lev, ii, jj, **kw) -> LeafGrid:
    leaf = [np.zeros((N << l, M << l), dtype=bool) for l in range(L + 1)]
    for l, a, b in zip(lev, ii, jj):
        leaf[int(l)][int(b), int(a)] = True
    return LeafGrid(M, N, L, R, leaf, **kw)


# ---------------------------------------------------------------------------
# the pyramid: Eq. 9 encode, the mean of the Manning raster, Eq. 10 prolongation
# ---------------------------------------------------------------------------
def _lowpass(c):
    """A_c as the C oracle forms it (rows k, columns m)"""
    sx = 1.0 if c & 1 else -1.0
    sy = 1.0 if c & 2 else -1.0
    return [[1.0, 0.0, 0.0], [HALF_S3 * sx, 0.5, 0.0], [HALF_S3 * sy, 0.0, 0.5]]


_A = [_lowpass(c) for c in range(4)]


def _children(a):
    """the four children (c = cx + 2 cy) of every node of the coarser level"""
    return [a[(c >> 1)::2, (c & 1)::2] for c in range(4)]


def encode_planes(p):
    """Eq. 9 (scale coefficients only) of one variable's planes p = (c0, c1x,
    c1y) one level up, summed in the C oracle's order"""
    ch = [_children(q) for q in p]
    out = []
    for k in range(3):
        acc = None
        for c in range(4):
            for m in range(3):
                term = _A[c][k][m] * ch[m][c]
                acc = term if acc is None else acc + term
        out.append(0.25 * acc)
    return out


def pyramid(finest, L):
    """planes of one variable at every level, finest (level L) first given"""
    levels = [None] * (L + 1)
    levels[L] = list(finest)
    for l in range(L - 1, -1, -1):
        levels[l] = encode_planes(levels[l + 1])
    return levels


def manning_levels(n_finest, L):
    levels = [None] * (L + 1)
    levels[L] = n_finest
    for l in range(L - 1, -1, -1):
        ch = _children(levels[l + 1])
        levels[l] = 0.25 * (((ch[0] + ch[1]) + ch[2]) + ch[3])
    return levels


def _upsample(a):
    return a.repeat_interleave(2, dim=0).repeat_interleave(2, dim=1)


def prolong_planes(p, ny, nx):
    """Eq. 10 with zero details: every node of a level from its parent's
    planes p (one level up), in the C oracle's order"""
    sp = [_upsample(q) for q in p]
    jj = torch.arange(ny).view(ny, 1).expand(ny, nx)
    ii = torch.arange(nx).view(1, nx).expand(ny, nx)
    sx = torch.where((ii & 1) == 1, 1.0, -1.0).to(F64)
    sy = torch.where((jj & 1) == 1, 1.0, -1.0).to(F64)
    c0 = (sp[0] + (HALF_S3 * sx) * sp[1]) + (HALF_S3 * sy) * sp[2]
    return [c0, 0.5 * sp[1], 0.5 * sp[2]]


# ---------------------------------------------------------------------------
# the operator on a graded grid
# ---------------------------------------------------------------------------
_PAIR = {0: (0, 2), 1: (1, 3), 2: (0, 1), 3: (2, 3)}   # the neighbour's children on face f
_EDGE = {0: 1, 1: 0, 2: 3, 3: 2}                        # the domain edge of face f
_STEP = {0: (1, 1), 1: (1, -1), 2: (0, 1), 3: (0, -1)}  # (axis, step) to the neighbour


def _inside(G, l, f):
    ny, nx = G.ny(l), G.nx(l)
    jj = torch.arange(ny).view(ny, 1).expand(ny, nx)
    ii = torch.arange(nx).view(1, nx).expand(ny, nx)
    return {0: ii < nx - 1, 1: ii > 0, 2: jj < ny - 1, 3: jj > 0}[f]


def _limits(w, ze, f):
    """interface-centre limits (h, qx, qy, z) of flux-view planes on face f"""
    return [face_lim(w[3 * v], w[3 * v + 1], w[3 * v + 2], f) for v in range(3)] + \
        [face_lim(ze[0], ze[1], ze[2], f)]


def _ghost(own, f, l, Q, t, G):
    """boundary ghost of face f (wall mirror, open copy, or the inflow at
    critical depth with the unit discharge of the leaf's overlap with the
    inflow cells), over the whole level"""
    h, qx, qy, zz = own
    e = _EDGE[f]
    out_h, out_x, out_y = h, qx, qy
    if G.bc[e] == WALL:
        if e < 2:
            out_x = -qx
        else:
            out_y = -qy
    if G.inflow_edge == e and len(G.knot_t) > 0:
        ny, nx = h.shape
        sh = G.L - l
        nk = ny if e < 2 else nx
        k = torch.arange(nk)
        lo = torch.clamp(k << sh, min=G.inflow_c0)
        hi = torch.clamp((k + 1) << sh, max=G.inflow_c1 + 1)
        ov = (hi - lo).clamp(min=0).to(F64)
        nin = float(G.inflow_c1 - G.inflow_c0 + 1)
        q1 = inflow_Q(Q, t, G.knot_t) * ov / (nin * G.dx(l))
        q = q1.view(ny, 1).expand(ny, nx) if e < 2 else q1.view(1, nx).expand(ny, nx)
        has = (ov > 0).view(-1, 1).expand(ny, nx) if e < 2 else (ov > 0).view(1, -1).expand(ny, nx)
        has = has & (q > 0.0)
        qs = _safe(has, q)
        hc = _Cbrt.apply(qs * qs / G.g)
        qn = qs if e in (0, 2) else -qs
        zero = torch.zeros_like(h)
        out_h = _w(has, _w(h >= hc, h, hc), out_h)
        if e < 2:
            out_x = _w(has, qn, out_x)
            out_y = _w(has, zero, out_y)
        else:
            out_x = _w(has, zero, out_x)
            out_y = _w(has, qn, out_y)
    return [out_h, out_x, out_y, zz]


def build_views(Wf, Zf, G: LeafGrid):
    """the same-level view (9 flow and 3 bed coefficients) of every node of
    every level, as the C oracle builds it: leaves their flux views, refined
    nodes the encoding of their children's views (Eq. 9, bottom-up), nodes
    below a coarser leaf the prolongation of their parent's view (Eq. 10 with
    zero details, top-down)"""
    L = G.L
    VS = [None] * (L + 1)
    for l in range(L, -1, -1):
        own = list(Wf[l]) + list(Zf[l])
        if l < L:
            enc = []
            for g0 in range(0, 12, 3):
                enc += encode_planes(VS[l + 1][g0:g0 + 3])
            own = [_w(G.sig[l], enc[m], own[m]) for m in range(12)]
        VS[l] = own
    V = [None] * (L + 1)
    V[0] = VS[0]
    for l in range(1, L + 1):
        pro = []
        for g0 in range(0, 12, 3):
            pro += prolong_planes(V[l - 1][g0:g0 + 3], G.ny(l), G.nx(l))
        V[l] = [_w(G.below[l], pro[m], VS[l][m]) for m in range(12)]
    return V


def operator(Wf, Zf, t, Q, G: LeafGrid, dt=0.0):
    """DG2 operator of every leaf (Eq. 4) from the flux views Wf[l] (9) and
    beds Zf[l] (3) of every level; returns the nine components per level.
    With dt > 0 each side's interface flux carries the outflow limit of a
    forward-Euler stage of that length (the donor is the own leaf or the
    neighbour's view, whose averages are those of the view's planes or, on a
    static grid's coarse side, the mean of the two finer leaves')."""
    g, hd = G.g, G.hd
    V = build_views(Wf, Zf, G)
    Lout = [None] * (G.L + 1)
    for l in range(G.L + 1):
        if not bool(G.leaf[l].any()):
            continue
        ny, nx, dxl = G.ny(l), G.nx(l), G.dx(l)
        own = [_limits(Wf[l], Zf[l], f) for f in range(4)]
        Fh, hs, us, vs, zr = [None] * 4, [None] * 4, [None] * 4, [None] * 4, [None] * 4
        for f in range(4):
            fo = f ^ 1
            axis, step = _STEP[f]
            # the same-level view of every node of this level across its face
            # fo: leaves, encodings of refined nodes, prolongations below
            # coarser leaves; on static grids a refined node's is the mean of
            # its two children on the face
            view = _limits(V[l][:9], V[l][9:], fo)
            vavg = [V[l][3 * v] for v in range(3)]
            if G.mode == "static" and l + 1 <= G.L:
                c1, c2 = _PAIR[f]
                fine = _limits(V[l + 1][:9], V[l + 1][9:], fo)
                avg = [0.5 * (_children(q)[c1] + _children(q)[c2]) for q in fine]
                view = [_w(G.sig[l], avg[q], view[q]) for q in range(4)]
                favg = [0.5 * (_children(V[l + 1][3 * v])[c1] + _children(V[l + 1][3 * v])[c2])
                        for v in range(3)]
                vavg = [_w(G.sig[l], favg[v], vavg[v]) for v in range(3)]
            nb = [_shift(q, axis, step) for q in view]
            nbavg = [_shift(q, axis, step) for q in vavg]
            gh = _ghost(own[f], f, l, Q, t, G)
            ins = _inside(G, l, f)
            nb = [_w(ins, nb[q], gh[q]) for q in range(4)]
            zf = _TieMax.apply(own[f][3], nb[3])
            ro = revise(own[f][0], own[f][1], own[f][2], own[f][3], zf, hd)
            rn = revise(nb[0], nb[1], nb[2], nb[3], zf, hd)
            if f == 0:
                Fh[f] = hll(ro[0], ro[1], ro[2], rn[0], rn[1], rn[2], g, hd)
            elif f == 1:
                Fh[f] = hll(rn[0], rn[1], rn[2], ro[0], ro[1], ro[2], g, hd)
            elif f == 2:
                H = hll(ro[0], ro[2], ro[1], rn[0], rn[2], rn[1], g, hd)
                Fh[f] = [H[0], H[2], H[1]]
            else:
                H = hll(rn[0], rn[2], rn[1], ro[0], ro[2], ro[1], g, hd)
                Fh[f] = [H[0], H[2], H[1]]
            if dt > 0.0:
                own_first = f in (0, 2)
                from_own = (Fh[f][0] > 0.0) if own_first else (Fh[f][0] < 0.0)
                mn, mt = (3, 6) if f < 2 else (6, 3)
                d_own = [Wf[l][0], Wf[l][mn], Wf[l][mt]]
                d_nb = [nbavg[0], nbavg[mn // 3], nbavg[mt // 3]]
                don = [_w(from_own, d_own[q], d_nb[q]) for q in range(3)]
                act = (Fh[f][0] != 0.0) & (from_own | ins)
                Fh[f] = drain_limit(Fh[f], don, act, dt, dxl, g, hd)
            hs[f], us[f], vs[f], zr[f] = ro
        Fxp, Gyp = [], []
        for a in range(2):
            f = a
            q = hs[f] * us[f]
            Fxp.append([q, q * us[f] + 0.5 * g * hs[f] * hs[f], q * vs[f]])
            f = 2 + a
            r = hs[f] * vs[f]
            Gyp.append([r, r * us[f], r * vs[f] + 0.5 * g * hs[f] * hs[f]])
        w, ze = Wf[l], Zf[l]
        Lo = [None] * 9
        for v in range(3):
            L0 = -(Fh[0][v] - Fh[1][v]) / dxl - (Fh[2][v] - Fh[3][v]) / dxl
            if v == 1:
                L0 = L0 + -g * 0.5 * (hs[0] + hs[1]) * (zr[0] - zr[1]) / dxl
            if v == 2:
                L0 = L0 + -g * 0.5 * (hs[2] + hs[3]) * (zr[2] - zr[3]) / dxl
            L1x = -(S3 / dxl) * (Fh[0][v] + Fh[1][v] - Fxp[0][v] - Fxp[1][v])
            L1y = -(S3 / dxl) * (Fh[2][v] + Fh[3][v] - Gyp[0][v] - Gyp[1][v])
            if v == 1:
                L1x = L1x + -(2.0 * S3 * g / dxl) * w[1] * (w[1] + ze[1])
            if v == 2:
                L1y = L1y + -(2.0 * S3 * g / dxl) * w[2] * (w[2] + ze[2])
            Lo[3 * v], Lo[3 * v + 1], Lo[3 * v + 2] = L0, L1x, L1y
        Lout[l] = Lo
    return Lout


# ---------------------------------------------------------------------------
# step and run
# ---------------------------------------------------------------------------
def _still(ref):
    one, zero = torch.ones_like(ref), torch.zeros_like(ref)
    return [one] + [zero] * 8


def _mask(U, G):
    """non-leaf positions back to still water (they never reach a leaf)"""
    out = []
    for l in range(G.L + 1):
        still = _still(U[l][0])
        out.append([_w(G.leaf[l], U[l][m], still[m]) for m in range(9)])
    return out


def step(U, z, nman, Q, dt, t, G: LeafGrid):
    """One DG2 step of size dt from time t on the frozen grid (Eq. 4a, 4b)."""
    rain = G.rain_rate if t < G.rain_t_end else 0.0
    levels = range(G.L + 1)
    Un = [friction(U[l], nman[l], dt, rain, G) for l in levels]
    s1 = [limit(Un[l], z[l], G, nbmask=G.leaf[l]) for l in levels]
    L1 = operator([s[1] for s in s1], [s[2] for s in s1], t, Q, G, dt)
    Ui = _mask([post([s1[l][0][m] + dt * L1[l][m] for m in range(9)], G.hd) if L1[l] is not None
                else s1[l][0] for l in levels], G)
    s2 = [limit(Ui[l], z[l], G, nbmask=G.leaf[l]) for l in levels]
    L2 = operator([s[1] for s in s2], [s[2] for s in s2], t + dt, Q, G, dt)
    return _mask([post([0.5 * (s1[l][0][m] + s2[l][0][m] + dt * L2[l][m]) for m in range(9)], G.hd)
                  if L2[l] is not None else s1[l][0] for l in levels], G)


def inputs(z_vert, n_finest, h_vert, qx_vert, qy_vert, G: LeafGrid):
    """per-level beds, Manning n and initial state from the C oracle's inputs
    (vertex rasters and the finest Manning raster), as the C oracle forms them"""
    zc = pyramid(project(z_vert), G.L)
    nm = manning_levels(n_finest, G.L)
    flow = [pyramid(project(v), G.L) for v in (h_vert, qx_vert, qy_vert)]
    U = [[flow[v][l][m] for v in range(3) for m in range(3)] for l in range(G.L + 1)]
    return _mask(U, G), zc, nm


def leaves_of(U, G: LeafGrid):
    """(n_leaves, 9) coefficients in the C oracle's leaf order (level, then
    row-major)"""
    rows = []
    for l in range(G.L + 1):
        idx = torch.nonzero(G.leaf[l], as_tuple=False)
        if idx.numel() == 0:
            continue
        jj, ii = idx[:, 0], idx[:, 1]
        rows.append(torch.stack([U[l][m][jj, ii] for m in range(9)], dim=1))
    return torch.cat(rows, dim=0)


def dense_from_leaves(coef, G: LeafGrid):
    """per-level state from (n_leaves, 9) coefficients in the C oracle's
    leaf order (non-leaf positions still water)"""
    U = []
    k0 = 0
    for l in range(G.L + 1):
        idx = torch.nonzero(G.leaf[l], as_tuple=False)
        still = _still(torch.zeros(G.ny(l), G.nx(l), dtype=F64))
        n = idx.shape[0]
        lvl = []
        for m in range(9):
            a = still[m].clone()
            if n:
                a = a.index_put((idx[:, 0], idx[:, 1]), coef[k0:k0 + n, m])
            lvl.append(a)
        U.append(lvl)
        k0 += n
    return U


def run_from(coef0, z_vert, n_finest, Q, dts, t0, G: LeafGrid):
    """the run from given leaf coefficients (an MWDG2 grid frozen after its
    adaptation, whose leaves hold the decoded state)"""
    U = dense_from_leaves(coef0, G)
    zc = pyramid(project(z_vert), G.L)
    nm = manning_levels(n_finest, G.L)
    t = t0
    for dt in dts:
        U = step(U, zc, nm, Q, float(dt), t, G)
        t = t + float(dt)
    return leaves_of(U, G)


def run(z_vert, n_finest, h_vert, qx_vert, qy_vert, Q, dts, t0, G: LeafGrid):
    U, zc, nm = inputs(z_vert, n_finest, h_vert, qx_vert, qy_vert, G)
    t = t0
    for dt in dts:
        U = step(U, zc, nm, Q, float(dt), t, G)
        t = t + float(dt)
    return leaves_of(U, G)


# ---------------------------------------------------------------------------
# regridding at a checkpoint: the MWDG2 adaptation's state transfer from one
# frozen grid to the next, with its decisions (the new grid) held
# ---------------------------------------------------------------------------
def depth_plane_for_children(sp):
    """The depth plane (c0, c1x, c1y) that a refinement prolongs: where one of
    its four children's averages (Eq. 10 with zero details) would be
    negative, its slopes are scaled about its average so that the smallest
    becomes zero (the scaling limiter of Zhang & Shu 2010 at the children's
    centres), or dropped when the plane has no content.  The smallest
    child is taken as the first of them in child order (c = cx + 2 cy)."""
    c0s = []
    for c in range(4):
        sx = 1.0 if c & 1 else -1.0
        sy = 1.0 if c & 2 else -1.0
        c0s.append((sp[0] + (HALF_S3 * sx) * sp[1]) + (HALF_S3 * sy) * sp[2])
    stack = torch.stack(c0s)
    idx = torch.argmin(stack.detach(), dim=0, keepdim=True)
    m = torch.gather(stack, 0, idx)[0]
    neg = m < 0.0
    pos = sp[0] > 0.0
    th = sp[0] / _safe(neg & pos, sp[0] - m)
    zero = torch.zeros_like(sp[0])
    s1 = _w(neg, _w(pos, sp[1] * th, zero), sp[1])
    s2 = _w(neg, _w(pos, sp[2] * th, zero), sp[2])
    return [sp[0], s1, s2]


def regrid(coef, G1: LeafGrid, G2: LeafGrid):
    """The leaves' coefficients on grid G2 from those on G1 (same roots and
    levels), as the MWDG2 adaptation transfers them (Sect. 2.3): the state is
    prolonged below G1's leaves down to the finest level (Eq. 10 with zero
    details; depth planes kept non-negative for the children, a child's
    rounding residue below zero depth set to zero), encoded up G1's refined
    nodes (Eq. 9), and read at G2's leaves: a leaf of both grids keeps its
    coefficients, a coarsened one takes its encoding, a refined one the
    prolongation of its old leaf.  Summed in the C oracle's order."""
    L = G1.L
    U = dense_from_leaves(coef, G1)
    for l in range(1, L + 1):
        ny, nx = G1.ny(l), G1.nx(l)
        par = U[l - 1]
        pro = prolong_planes(depth_plane_for_children(par[0:3]), ny, nx)
        pro += prolong_planes(par[3:6], ny, nx) + prolong_planes(par[6:9], ny, nx)
        pro[0] = _w(pro[0] < 0.0, torch.zeros_like(pro[0]), pro[0])
        U[l] = [_w(G1.below[l], pro[m], U[l][m]) for m in range(9)]
    for l in range(L - 1, -1, -1):
        enc = []
        for g0 in (0, 3, 6):
            enc += encode_planes(U[l + 1][g0:g0 + 3])
        U[l] = [_w(G1.sig[l], enc[m], U[l][m]) for m in range(9)]
    return leaves_of(U, G2)


# ---------------------------------------------------------------------------
# the reverse of the views: who reads each leaf's flux-view planes
# ---------------------------------------------------------------------------
def _face_row(f):
    """face_lim on face f as a row vector on (c0, c1x, c1y)"""
    return {0: np.array([1.0, S3, 0.0]), 1: np.array([1.0, -S3, 0.0]), 2: np.array([1.0, 0.0, S3]),
            3: np.array([1.0, 0.0, -S3])}[f]


def view_reverse_table(G: LeafGrid):
    """The neighbour-side limits of every leaf face, written as a linear
    function of the owner leaves' flux-view planes: entries (reader leaf,
    face f, owner leaf, w) with nb_q(reader, f) = sum over its entries of
    w . planes_q(owner), the same 3-vector w for each variable q (h, qx, qy,
    bed).  Leaves are numbered in the C oracle's order (level, then
    row-major); domain-edge faces (ghosts) have no entries.  Same-level leaf:
    w = the face-limit row of face f^1.  Static refined neighbour: half of it
    on each of the two children on the face.  MWDG2 refined neighbour: the
    transpose of the encode down its subtree (1/4 row A_c per level).  Below
    a coarser leaf: the transpose of the prolongation up to that leaf (row
    A_c^T per level).  The reverse of the views is then g_owner += w
    cot(reader, f, q), which is what reverse kernels gather by owner."""
    L = G.L
    index = {}
    for l in range(L + 1):
        for j, i in torch.nonzero(G.leaf[l], as_tuple=False).tolist():
            index[(l, i, j)] = len(index)

    def kind(l, i, j):
        return 'leaf' if bool(G.leaf[l][j, i]) else ('sig' if bool(G.sig[l][j, i]) else 'below')

    def down(l, a, b, row):
        out = []
        for c in range(4):
            ca, cb = 2 * a + (c & 1), 2 * b + (c >> 1)
            r = 0.25 * row @ np.array(_A[c])
            out += [(index[(l + 1, ca, cb)], r)] if kind(l + 1, ca, cb) == 'leaf' else down(l + 1, ca, cb, r)
        return out

    def up(l, a, b, row):
        r = row @ np.array(_A[(a & 1) + 2 * (b & 1)]).T
        pa, pb = a >> 1, b >> 1
        return [(index[(l - 1, pa, pb)], r)] if kind(l - 1, pa, pb) == 'leaf' else up(l - 1, pa, pb, r)

    table = []
    for (l, i, j), k in index.items():
        for f in range(4):
            a = i + (f == 0) - (f == 1)
            b = j + (f == 2) - (f == 3)
            if not (0 <= a < G.nx(l) and 0 <= b < G.ny(l)):
                continue
            row = _face_row(f ^ 1)
            kd = kind(l, a, b)
            if kd == 'leaf':
                ents = [(index[(l, a, b)], row)]
            elif kd == 'sig' and G.mode == 'static':
                ents = [(index[(l + 1, 2 * a + (c & 1), 2 * b + (c >> 1))], 0.5 * row) for c in _PAIR[f]]
            elif kd == 'sig':
                ents = down(l, a, b, row)
            else:
                ents = up(l, a, b, row)
            table += [(k, f, owner, w) for owner, w in ents]
    return table
