"""FP64 oracle of the discrete adjoint of the DG2 step on a uniform grid.

TEST INFRASTRUCTURE ONLY.  Like the rest of ``oracle/``, this module is the
plain, slow reference that the CUDA library is checked against; only the tests
may import it, and the product package never imports or falls back to it.

What it computes.  The uniform-grid DG2 step of Sect. 2.1.1 (Eq. 1-4: the
planar scaled-Legendre basis, split implicit Manning friction at the start of
a step, slope limiting with partial-wet reduction, hydrostatic face revision,
HLL fluxes, the two-stage Runge-Kutta update with positivity clip), restated
with plain PyTorch CPU tensor operations in FP64, element by element in the
same operation order as ``mwdg2_oracle.c`` so that a run over a given time-step
sequence reproduces the C oracle bit for bit (checked by the tests).  The
discrete adjoint is then the derivative of that map, taken by PyTorch's
reverse-mode automatic differentiation: a library primitive applied to the
plain definition, not a hand-derived reverse sweep.

Readings (the paper gives no adjoint; it is the gradient capability that the
hot path's users ask of the step):
  * The time steps are the recorded ones, held fixed: the map differentiated
    is U_K = S_{dt_K} o ... o S_{dt_1}(U_0; z, n, Q), with each dt the value the
    CFL condition chose on the unperturbed run.
  * Branches (wet/dry tests, partial-wet reduction, minmod selection, HLL wave
    regions, positivity clip) are taken as the forward run took them; the
    derivative is that of the branch taken.  Where minmod's selected value is
    met by two arguments, the earlier argument (the slope, then the forward
    difference, then the backward difference) is the one differentiated.
  * The interface bed max(z_L, z_R): when the two limits agree to within
    1e-10 max(1, |z_L|, |z_R|) (a continuous DEM gives equal limits from both
    sides up to rounding) each side takes half of the cotangent, the mean of
    the two one-sided derivatives, which is what a central difference of the
    step measures there.  Otherwise the larger side takes all of it.
  * The Manning speed |u| at rest: derivative zero (the apex of the cone).

Pinned by the tests against: the C oracle's forward bit for bit; central
finite differences of the C oracle's fixed-dt step with respect to Manning n,
DEM vertex heights, hydrograph knots and initial depth and discharge
vertices; still water (no sensitivity to n or to the knots).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

S3 = math.sqrt(3.0)
TIE_REL = 1e-10
F64 = torch.float64

WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
WALL, OPEN = 0, 1


@dataclass
class Grid:
    """Uniform grid and physical parameters (SI units); edges 0 W, 1 E, 2 S, 3 N."""
    nx: int
    ny: int
    dx: float
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


# ---------------------------------------------------------------------------
# primitives with stated derivatives
# ---------------------------------------------------------------------------
def _cbrt_newton(x: torch.Tensor) -> torch.Tensor:
    """Cube root as the C oracle computes it (Kahan's exponent seed, six Newton
    steps); x >= 0, zero maps to zero."""
    pos = x > 0.0
    xs = torch.where(pos, x, torch.ones_like(x))
    small = xs < 1e-290
    xs = torch.where(small, xs * 2.0 ** 300, xs)
    scale = torch.where(small, torch.full_like(xs, 2.0 ** -100), torch.ones_like(xs))
    b = xs.contiguous().view(torch.int64)
    b = torch.div(b, 3, rounding_mode="floor") + (682 << 52)
    y = b.view(F64)
    for _ in range(6):
        y = y - (y * y * y - xs) / (3.0 * y * y)
    return torch.where(pos, scale * y, x)


class _Cbrt(torch.autograd.Function):
    """x^(1/3) with derivative 1 / (3 y^2) (zero at x = 0, never used there)."""

    @staticmethod
    def forward(ctx, x):
        y = _cbrt_newton(x)
        ctx.save_for_backward(y)
        return y

    @staticmethod
    def backward(ctx, g):
        (y,) = ctx.saved_tensors
        d = torch.where(y > 0.0, 1.0 / (3.0 * torch.where(y > 0.0, y, torch.ones_like(y)) ** 2),
                        torch.zeros_like(y))
        return g * d


def _sqrt_rn(x: torch.Tensor) -> torch.Tensor:
    """correctly rounded square root (numpy's IEEE sqrt; the vectorised CPU
    kernel behind torch.sqrt may differ from it in the last place)"""
    return torch.from_numpy(np.sqrt(x.detach().contiguous().numpy()))


class _Sqrt(torch.autograd.Function):
    """sqrt(x), x > 0, with derivative 1 / (2 sqrt(x))."""

    @staticmethod
    def forward(ctx, x):
        y = _sqrt_rn(x)
        ctx.save_for_backward(y)
        return y

    @staticmethod
    def backward(ctx, g):
        (y,) = ctx.saved_tensors
        return g * 0.5 / y


class _Speed(torch.autograd.Function):
    """sqrt(u^2 + v^2); derivative (u, v) / |.|, zero at the origin."""

    @staticmethod
    def forward(ctx, u, v):
        s = _sqrt_rn(u * u + v * v)
        ctx.save_for_backward(u, v, s)
        return s

    @staticmethod
    def backward(ctx, g):
        u, v, s = ctx.saved_tensors
        nz = s > 0.0
        ss = torch.where(nz, s, torch.ones_like(s))
        z = torch.zeros_like(s)
        return torch.where(nz, g * u / ss, z), torch.where(nz, g * v / ss, z)


class _TieMax(torch.autograd.Function):
    """max(a, b) for the interface bed; a tie within TIE_REL splits the
    cotangent in halves."""

    @staticmethod
    def forward(ctx, a, b):
        ctx.save_for_backward(a, b)
        return torch.maximum(a, b)

    @staticmethod
    def backward(ctx, g):
        a, b = ctx.saved_tensors
        scale = torch.maximum(torch.ones_like(a), torch.maximum(a.abs(), b.abs()))
        tie = (a - b).abs() <= TIE_REL * scale
        ga = torch.where(tie, 0.5 * g, torch.where(a > b, g, torch.zeros_like(g)))
        gb = torch.where(tie, 0.5 * g, torch.where(a > b, torch.zeros_like(g), g))
        return ga, gb


def _w(c, a, b):
    """select with a condition that carries no derivative"""
    return torch.where(c.detach() if isinstance(c, torch.Tensor) else c, a, b)


def _safe(c, x):
    """x where c holds, 1 elsewhere (keeps untaken branches finite)"""
    return torch.where(c, x, torch.ones_like(x))


def face_lim(c0, c1x, c1y, f):
    """limit of a plane at the centre of face f (0 E, 1 W, 2 N, 3 S)"""
    if f == 0:
        return c0 + S3 * c1x
    if f == 1:
        return c0 - S3 * c1x
    if f == 2:
        return c0 + S3 * c1y
    return c0 - S3 * c1y


# ---------------------------------------------------------------------------
# the pieces of one step
# ---------------------------------------------------------------------------
def friction(U, nman, dt, rain, P: Grid):
    """rain depth of the step, then split implicit Manning friction (Sect. 2.1.1)"""
    w0 = U[0]
    if rain > 0.0:
        w0 = w0 + rain * dt
    wet = w0 > P.hd
    h = _safe(wet, w0)
    u = U[3] / h
    v = U[6] / h
    sp = _Speed.apply(u, v)
    den = 1.0 + (dt * P.g) * nman * nman * sp / (h * _Cbrt.apply(h))
    f = 1.0 / den
    out = [w0, U[1], U[2]]
    for m in range(3, 9):
        out.append(_w(wet, U[m] * f, torch.zeros_like(U[m])))
    return out


def _shift(a, axis, step):
    """value of the neighbour at +step along axis (own value past the edge)"""
    out = a.clone()
    if axis == 1:  # x
        if step > 0:
            out[:, :-1] = a[:, 1:]
        else:
            out[:, 1:] = a[:, :-1]
    else:
        if step > 0:
            out[:-1, :] = a[1:, :]
        else:
            out[1:, :] = a[:-1, :]
    return out


def limit(X, z, P: Grid, nbmask=None):
    """Stage-input limiting: (stored view w_st, flux view w_fx, flux-view bed ze).
    nbmask (non-uniform grids): which cells of the level are leaves; only
    those count as neighbours (same-level leaf neighbours, Sect. 2.2.1)."""
    hd = P.hd
    ny, nx = X[0].shape
    h0 = X[0]
    eta0 = h0 + z[0]
    red = ~(h0 > hd)
    for f in range(4):
        red = red | ~(face_lim(X[0], X[1], X[2], f) > hd)
        red = red | ~(eta0 - face_lim(z[0], z[1], z[2], f) > hd)
    ws = list(X)
    if P.limiter:
        ii = torch.arange(nx).view(1, nx).expand(ny, nx)
        jj = torch.arange(ny).view(ny, 1).expand(ny, nx)
        for d in range(2):
            axis = 1 if d == 0 else 0
            if d == 0:
                hasA, hasB = ii < nx - 1, ii > 0
            else:
                hasA, hasB = jj < ny - 1, jj > 0
            if nbmask is not None:
                hasA = hasA & _shift(nbmask, axis, 1)
                hasB = hasB & _shift(nbmask, axis, -1)
            cs = 1 + d
            hC, hA, hB = X[0], _shift(X[0], axis, 1), _shift(X[0], axis, -1)
            wet = (hC > hd) & (~hasA | (hA > hd)) & (~hasB | (hB > hd))
            for v in range(3):
                if v == 0:
                    aC = hC + z[0]
                    a0 = hA + _shift(z[0], axis, 1)
                    aB = hB + _shift(z[0], axis, -1)
                    slope = X[cs] + z[cs]
                    coef = cs
                else:
                    aC = X[3 * v]
                    a0 = _shift(X[3 * v], axis, 1)
                    aB = _shift(X[3 * v], axis, -1)
                    slope = X[3 * v + cs]
                    coef = 3 * v + cs
                a = S3 * slope
                d1 = a0 - aC
                d2 = aC - aB
                ad, d1d, d2d = a.detach(), d1.detach(), d2.detach()
                both = hasA & hasB
                pos3 = (ad > 0) & (d1d > 0) & (d2d > 0)
                neg3 = (ad < 0) & (d1d < 0) & (d2d < 0)
                mm3 = torch.where(pos3, torch.minimum(ad, torch.minimum(d1d, d2d)),
                                  torch.where(neg3, torch.maximum(ad, torch.maximum(d1d, d2d)),
                                              torch.zeros_like(ad)))
                oth = torch.where(hasA, d1d, d2d)
                pos2 = (ad > 0) & (oth > 0)
                neg2 = (ad < 0) & (oth < 0)
                mm2 = torch.where(pos2, torch.minimum(ad, oth),
                                  torch.where(neg2, torch.maximum(ad, oth), torch.zeros_like(ad)))
                mm = torch.where(both, mm3, mm2)
                same = torch.where(both, pos3 | neg3, pos2 | neg2)
                # which argument the replaced value is
                take1 = same & torch.where(both, mm == d1d, hasA)
                take2 = same & ~take1
                val = torch.where(take1, d1, torch.where(take2, d2, torch.zeros_like(d1)))
                new = val / S3
                if v == 0:
                    new = new - z[cs]
                active = ~red & (hasA | hasB) & (wet if v == 0 else torch.ones_like(wet))
                repl = active & (mm != ad)
                ws[coef] = _w(repl, new, ws[coef])
    zero = torch.zeros_like(X[0])
    w_st, w_fx = [], []
    for m in range(9):
        if m in (1, 2):
            red_st = -z[m]
        elif m in (4, 5, 7, 8):
            red_st = zero
        else:
            red_st = X[m]
        w_st.append(_w(red, red_st, ws[m]))
        w_fx.append(_w(red, zero if m in (1, 2) else red_st, ws[m]))
    ze = [z[0], _w(red, zero, z[1]), _w(red, zero, z[2])]
    return w_st, w_fx, ze


def inflow_Q(Q, t, knot_t):
    """piecewise-linear hydrograph, constant outside the knots"""
    n = len(knot_t)
    if t <= knot_t[0]:
        return Q[0]
    if t >= knot_t[n - 1]:
        return Q[n - 1]
    k = 0
    while k + 1 < n and not (t < knot_t[k + 1]):
        k += 1
    return Q[k] + (Q[k + 1] - Q[k]) * (t - knot_t[k]) / (knot_t[k + 1] - knot_t[k])


def ghost(own, e, Q, t, P: Grid):
    """ghost limit at a boundary face on edge e: inflow (critical depth carrying
    the hydrograph), open (copy) or wall (mirror).  own = (h, qx, qy, z),
    tensors along the edge."""
    h, qx, qy, zz = own
    nedge = h.shape[0]
    out_h, out_x, out_y = h, qx, qy
    if P.bc[e] == WALL:
        if e < 2:
            out_x = -qx
        else:
            out_y = -qy
    if P.inflow_edge == e and len(P.knot_t) > 0:
        nin = P.inflow_c1 - P.inflow_c0 + 1
        k = torch.arange(nedge)
        inr = (k >= P.inflow_c0) & (k <= P.inflow_c1)
        q = inflow_Q(Q, t, P.knot_t) * 1.0 / (float(nin) * P.dx) * torch.ones(nedge, dtype=F64)
        has = inr & (q > 0.0)
        qs = _safe(has, q)
        hc = _Cbrt.apply(qs * qs / P.g)
        qn = qs if e in (0, 2) else -qs
        zero = torch.zeros_like(h)
        out_h = _w(has, _w(h >= hc, h, hc), out_h)
        if e < 2:
            out_x = _w(has, qn, out_x)
            out_y = _w(has, zero, out_y)
        else:
            out_x = _w(has, zero, out_x)
            out_y = _w(has, qn, out_y)
    return out_h, out_x, out_y, zz


def revise(h, qx, qy, z, zf, hd):
    eta = h + z
    d = eta - zf
    wetf = d > hd
    hs = _w(wetf, d, torch.zeros_like(d))
    zr = _w(wetf, zf, eta)
    wet = h > hd
    hh = _safe(wet, h)
    u = _w(wet, qx / hh, torch.zeros_like(h))
    v = _w(wet, qy / hh, torch.zeros_like(h))
    return hs, u, v, zr


def hll(hL, unL, utL, hR, unR, utR, g, hd):
    dryL, dryR = ~(hL > hd), ~(hR > hd)
    cL = _Sqrt.apply(g * _safe(~dryL, hL))
    cR = _Sqrt.apply(g * _safe(~dryR, hR))
    us = 0.5 * (unL + unR) + cL - cR
    cs = 0.5 * (cL + cR) + 0.25 * (unL - unR)
    a1, a2 = unL - cL, us - cs
    b1, b2 = unR + cR, us + cs
    sLw = _w(a1 <= a2, a1, a2)
    sRw = _w(b1 >= b2, b1, b2)
    sL = _w(dryL, unR - 2.0 * cR, _w(dryR, unL - cL, sLw))
    sR = _w(dryL, unR + cR, _w(dryR, unL + 2.0 * cL, sRw))
    qL, qR = hL * unL, hR * unR
    FL = [qL, qL * unL + 0.5 * g * hL * hL, qL * utL]
    FR = [qR, qR * unR + 0.5 * g * hR * hR, qR * utR]
    UL = [hL, qL, hL * utL]
    UR = [hR, qR, hR * utR]
    left = sL >= 0.0
    right = ~left & (sR <= 0.0)
    mid = ~left & ~right
    den = _safe(mid, sR - sL)
    both_dry = dryL & dryR
    F = []
    for k in range(3):
        Fm = (sR * FL[k] - sL * FR[k] + sL * sR * (UR[k] - UL[k])) / den
        Fk = _w(left, FL[k], _w(right, FR[k], Fm))
        F.append(_w(both_dry, torch.zeros_like(Fk), Fk))
    return F


def drain_limit(F, don, act, dt, dx, g, hd):
    """Outflow limited by content (the C oracle's drain_limit): where act (the
    donor, the side the mass leaves, is a leaf and F[0] != 0) the mass flux is
    limited to |F[0]| dt <= s_f h0 dx with the donor's share
    s_f = e_f / (e_E + e_W + e_N + e_S), e_f = max(0, outward average
    velocity) + sqrt(g h0), and the momentum components are scaled by the
    same factor; a donor without content passes nothing.  F in (h, qx, qy)
    order along +x or +y; don = the donor's flux-view averages (h0, q_n0,
    q_t0)."""
    h0 = don[0]
    zero = torch.zeros_like(h0)
    pos = h0 > 0.0
    wet = h0 > hd
    hh = _safe(wet, h0)
    un = _w(wet, don[1] / hh, zero)
    ut = _w(wet, don[2] / hh, zero)
    c = _Sqrt.apply(g * _safe(pos, h0))
    out = _w(F[0] > 0.0, un, -un)
    e = _w(out > 0.0, out, zero) + c
    S = (un.abs() + ut.abs()) + 4.0 * c
    cap = (h0 * dx / dt) * (e / S)
    a = F[0].abs()
    kill = act & ~pos
    bite = act & pos & (a > cap)
    th = cap / _safe(bite, a)
    F0 = _w(bite, _w(F[0] > 0.0, cap, -cap), F[0])
    out_F = [F0, _w(bite, F[1] * th, F[1]), _w(bite, F[2] * th, F[2])]
    return [_w(kill, zero, q) for q in out_F]


def operator(w, ze, t, Q, P: Grid, dt=0.0):
    """DG2 spatial operator of every cell (Eq. 4) from the flux view w (9) and
    its beds ze (3); returns the nine operator components.  With dt > 0 the
    interface fluxes carry the outflow limit of a forward-Euler stage of that
    length."""
    g, hd, dx = P.g, P.hd, P.dx
    lim = [[face_lim(w[3 * v], w[3 * v + 1], w[3 * v + 2], f) for v in range(3)] +
           [face_lim(ze[0], ze[1], ze[2], f)] for f in range(4)]
    # x faces: (ny, nx + 1); left side = cell i-1's E limit, right = cell i's W limit
    gW = ghost([lim[1][q][:, 0] for q in range(4)], WEST, Q, t, P)
    gE = ghost([lim[0][q][:, -1] for q in range(4)], EAST, Q, t, P)
    Lx = [torch.cat([gW[q][:, None], lim[0][q]], dim=1) for q in range(4)]
    Rx = [torch.cat([lim[1][q], gE[q][:, None]], dim=1) for q in range(4)]
    gS = ghost([lim[3][q][0, :] for q in range(4)], SOUTH, Q, t, P)
    gN = ghost([lim[2][q][-1, :] for q in range(4)], NORTH, Q, t, P)
    By = [torch.cat([gS[q][None, :], lim[2][q]], dim=0) for q in range(4)]
    Ty = [torch.cat([lim[3][q], gN[q][None, :]], dim=0) for q in range(4)]

    zfx = _TieMax.apply(Lx[3], Rx[3])
    rL = revise(Lx[0], Lx[1], Lx[2], Lx[3], zfx, hd)
    rR = revise(Rx[0], Rx[1], Rx[2], Rx[3], zfx, hd)
    Fx = hll(rL[0], rL[1], rL[2], rR[0], rR[1], rR[2], g, hd)
    zfy = _TieMax.apply(By[3], Ty[3])
    rB = revise(By[0], By[1], By[2], By[3], zfy, hd)
    rT = revise(Ty[0], Ty[1], Ty[2], Ty[3], zfy, hd)
    H = hll(rB[0], rB[2], rB[1], rT[0], rT[2], rT[1], g, hd)
    Fy = [H[0], H[2], H[1]]

    if dt > 0.0:
        # x interfaces (ny, nx + 1): left cell i - 1, right cell i; y
        # interfaces (ny + 1, nx): below j - 1, above j; boundary ghosts are
        # never limited donors
        ny, nx = w[0].shape
        col = torch.arange(nx + 1).view(1, nx + 1).expand(ny, nx + 1)
        row = torch.arange(ny + 1).view(ny + 1, 1).expand(ny + 1, nx)
        for xdir in (True, False):
            Fi = Fx if xdir else Fy
            mn, mt = (3, 6) if xdir else (6, 3)
            if xdir:
                lo = [torch.cat([w[m][:, :1], w[m]], dim=1) for m in (0, mn, mt)]
                hi = [torch.cat([w[m], w[m][:, -1:]], dim=1) for m in (0, mn, mt)]
                lo_ok, hi_ok = col >= 1, col <= nx - 1
            else:
                lo = [torch.cat([w[m][:1, :], w[m]], dim=0) for m in (0, mn, mt)]
                hi = [torch.cat([w[m], w[m][-1:, :]], dim=0) for m in (0, mn, mt)]
                lo_ok, hi_ok = row >= 1, row <= ny - 1
            fwd = Fi[0] > 0.0
            don = [_w(fwd, lo[q], hi[q]) for q in range(3)]
            act = (Fi[0] != 0.0) & torch.where(fwd, lo_ok, hi_ok)
            Fl = drain_limit(Fi, don, act, dt, dx, g, hd)
            if xdir:
                Fx = Fl
            else:
                Fy = Fl
    Fh = [[Fx[v][:, 1:] for v in range(3)], [Fx[v][:, :-1] for v in range(3)],
          [Fy[v][1:, :] for v in range(3)], [Fy[v][:-1, :] for v in range(3)]]
    own = [[r[:, 1:] for r in rL], [r[:, :-1] for r in rR], [r[1:, :] for r in rB], [r[:-1, :] for r in rT]]
    hs = [own[f][0] for f in range(4)]
    us = [own[f][1] for f in range(4)]
    vs = [own[f][2] for f in range(4)]
    zr = [own[f][3] for f in range(4)]
    Fxp, Gyp = [], []
    for a in range(2):
        f = a
        q = hs[f] * us[f]
        Fxp.append([q, q * us[f] + 0.5 * g * hs[f] * hs[f], q * vs[f]])
        f = 2 + a
        r = hs[f] * vs[f]
        Gyp.append([r, r * us[f], r * vs[f] + 0.5 * g * hs[f] * hs[f]])
    Lo = [None] * 9
    for v in range(3):
        L0 = -(Fh[0][v] - Fh[1][v]) / dx - (Fh[2][v] - Fh[3][v]) / dx
        if v == 1:
            L0 = L0 + -g * 0.5 * (hs[0] + hs[1]) * (zr[0] - zr[1]) / dx
        if v == 2:
            L0 = L0 + -g * 0.5 * (hs[2] + hs[3]) * (zr[2] - zr[3]) / dx
        L1x = -(S3 / dx) * (Fh[0][v] + Fh[1][v] - Fxp[0][v] - Fxp[1][v])
        L1y = -(S3 / dx) * (Fh[2][v] + Fh[3][v] - Gyp[0][v] - Gyp[1][v])
        if v == 1:
            L1x = L1x + -(2.0 * S3 * g / dx) * w[1] * (w[1] + ze[1])
        if v == 2:
            L1y = L1y + -(2.0 * S3 * g / dx) * w[2] * (w[2] + ze[2])
        Lo[3 * v], Lo[3 * v + 1], Lo[3 * v + 2] = L0, L1x, L1y
    return Lo


def post(o, hd):
    """positivity clip and dry reset after a stage"""
    h = _w(o[0] < 0.0, torch.zeros_like(o[0]), o[0])
    dry = ~(h > hd)
    out = [h]
    for m in range(1, 9):
        out.append(_w(dry, torch.zeros_like(o[m]), o[m]))
    return out


def step(U, z, nman, Q, dt, t, P: Grid):
    """One DG2 step of size dt from time t (Eq. 4a, 4b)."""
    rain = P.rain_rate if t < P.rain_t_end else 0.0
    Un = friction(U, nman, dt, rain, P)
    w1, f1, z1 = limit(Un, z, P)
    L1 = operator(f1, z1, t, Q, P, dt)
    Ui = post([w1[m] + dt * L1[m] for m in range(9)], P.hd)
    w2, f2, z2 = limit(Ui, z, P)
    L2 = operator(f2, z2, t + dt, Q, P, dt)
    return post([0.5 * (w1[m] + w2[m] + dt * L2[m]) for m in range(9)], P.hd)


def project(vert):
    """Eq. 8 in tensor form (same operation order as the C oracle)"""
    sw, se = vert[:-1, :-1], vert[:-1, 1:]
    nw, ne = vert[1:, :-1], vert[1:, 1:]
    zn, zs = 0.5 * (nw + ne), 0.5 * (sw + se)
    ze, zw = 0.5 * (ne + se), 0.5 * (nw + sw)
    return [0.5 * (ze + zw), (ze - zw) / (2.0 * S3), (zn - zs) / (2.0 * S3)]


# ---------------------------------------------------------------------------
# drivers
# ---------------------------------------------------------------------------
def run(U0, z, nman, Q, dts, t0, P: Grid):
    """U_K after the steps dts from time t0; U0 (9, ny, nx), z (3, ny, nx),
    nman (ny, nx), Q (knots,) as tensors."""
    U = [U0[m] for m in range(9)]
    zl = [z[m] for m in range(3)]
    t = t0
    for dt in dts:
        U = step(U, zl, nman, Q, float(dt), t, P)
        t = t + float(dt)
    return torch.stack(U)


def _t(a):
    return torch.tensor(a, dtype=F64)


def forward(U0, z, nman, Q, dts, t0, P: Grid):
    """numpy in, numpy out"""
    with torch.no_grad():
        return run(_t(U0), _t(z), _t(nman), _t(Q), dts, t0, P).numpy()


def gradients(U0, z, nman, Q, dts, t0, P: Grid, seed, z_vert=None):
    """Cotangents of J = sum(seed * U_K) with respect to U0 (9, ny, nx), the bed
    planes z (3, ny, nx), Manning n (ny, nx) and the knots Q; with z_vert
    given, the bed comes from that vertex raster by Eq. 8 and its gradient is
    returned too."""
    U0t = _t(U0).requires_grad_(True)
    nt = _t(nman).requires_grad_(True)
    Qt = _t(Q).requires_grad_(True)
    if z_vert is not None:
        vt = _t(z_vert).requires_grad_(True)
        zt = torch.stack(project(vt))
        zt.retain_grad()
    else:
        zt = _t(z).requires_grad_(True)
    UK = run(U0t, zt, nt, Qt, dts, t0, P)
    J = (UK * _t(seed)).sum()
    J.backward()
    out = dict(U=UK.detach().numpy(), gU0=U0t.grad.numpy(), gz=zt.grad.numpy(), gn=nt.grad.numpy(),
               gQ=Qt.grad.numpy() if Qt.grad is not None else torch.zeros_like(Qt).numpy())
    if z_vert is not None:
        out["gzv"] = vt.grad.numpy()
    return out
