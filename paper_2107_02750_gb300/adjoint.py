"""Binding of the DG2 adjoint (include/mwdg_adjoint.h) and its autograd form.

Argument marshalling only: the forward and reverse sweeps run in the
library's CUDA kernels.  Tensors are on the CUDA device, contiguous, FP64 for
an F64 context and FP32 for an F32 one (time steps and knots FP64 in both):
U (9, ny, nx) in the component order (h0, h1x, h1y, qx0, qx1x, qx1y, qy0,
qy1x, qy1y), bed planes z (3, ny, nx), Manning n (ny, nx), hydrograph knots
(k,).  Work is queued on torch's current CUDA stream.

On a frozen non-uniform grid (``Dg2Adjoint.frozen``: a static graded grid or
an MWDG2 grid held fixed over the segment) U is (9, n_leaves), the leaves in
the order given; z and n stay on the finest level.

``Dg2Run`` is a ``torch.autograd.Function`` over one segment of K steps: its
forward records the CFL time steps (or takes given ones), its backward
recomputes the segment from its input state (the checkpoint) and returns the
gradients with respect to U0, z, n and the knots.  Chaining segments through
autograd checkpoints every K steps.
"""
from __future__ import annotations

import ctypes as C

from .binding import MwdgError, lib as _lib, WALL, F64, F32, STATIC, ADAPTIVE

ADJ_EXPORTS = (
    "mwdg_adj_params_default", "mwdg_adj_create", "mwdg_adj_create_frozen", "mwdg_adj_destroy", "mwdg_adj_project",
    "mwdg_adj_project_transpose", "mwdg_adj_forward", "mwdg_adj_backward", "mwdg_adj_last_error",
    "mwdg_adj_profile", "mwdg_adj_kernel_times", "mwdg_adj_regrid", "mwdg_adj_regrid_transpose",
)
# kernel classes of mwdg_adj_kernel_times, in order
ADJ_CLASSES = ("cfl", "friction", "limit", "update", "rev_face", "rev_knots", "rev_limit", "rev_gather",
               "rev_friction")


class AdjParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double), ("g", C.c_double), ("h_dry", C.c_double),
        ("cfl", C.c_double), ("dt_max", C.c_double), ("limiter", C.c_int32), ("bc", C.c_int32 * 4),
        ("inflow_edge", C.c_int32), ("inflow_c0", C.c_int32), ("inflow_c1", C.c_int32),
        ("rain_rate", C.c_double), ("rain_t_end", C.c_double), ("max_steps", C.c_int32),
        ("precision", C.c_int32), ("tape_views", C.c_int32),
    ]


def lib():
    L = _lib()
    if not getattr(L, "_adj_ready", False):
        vp, dp, i32 = C.c_void_p, C.c_double, C.c_int32
        L.mwdg_adj_params_default.argtypes = [C.POINTER(AdjParams)]
        L.mwdg_adj_create.argtypes = [C.POINTER(AdjParams), C.POINTER(vp)]
        L.mwdg_adj_create_frozen.argtypes = [C.POINTER(AdjParams), i32, i32, i32, i32, C.c_int64, vp, vp, vp,
                                             C.POINTER(vp)]
        L.mwdg_adj_destroy.argtypes = [vp]
        L.mwdg_adj_destroy.restype = None
        L.mwdg_adj_project.argtypes = [vp, vp, vp, vp]
        L.mwdg_adj_project_transpose.argtypes = [vp, vp, vp, vp]
        L.mwdg_adj_forward.argtypes = [vp, vp, vp, vp, i32, vp, vp, dp, i32, i32, vp, vp, vp]
        L.mwdg_adj_backward.argtypes = [vp, vp, vp, vp, i32, vp, vp, dp, i32, vp, vp, vp, vp, vp, vp, i32, vp]
        L.mwdg_adj_regrid.argtypes = [vp, vp, vp, vp, vp]
        L.mwdg_adj_regrid_transpose.argtypes = [vp, vp, vp, vp, vp, vp]
        L.mwdg_adj_last_error.argtypes = [vp]
        L.mwdg_adj_last_error.restype = C.c_char_p
        L.mwdg_adj_profile.argtypes = [vp, i32]
        L.mwdg_adj_kernel_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        for name in ("mwdg_adj_params_default", "mwdg_adj_create", "mwdg_adj_create_frozen", "mwdg_adj_project",
                     "mwdg_adj_project_transpose", "mwdg_adj_forward", "mwdg_adj_backward",
                     "mwdg_adj_profile", "mwdg_adj_kernel_times", "mwdg_adj_regrid",
                     "mwdg_adj_regrid_transpose"):
            getattr(L, name).restype = C.c_int
        L._adj_ready = True
    return L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Dg2Adjoint:
    """One adjoint context (include/mwdg_adjoint.h) on the current device."""

    def __init__(self, nx, ny, dx, *, g=9.80665, h_dry=1e-3, cfl=0.33, dt_max=1.0, limiter=1,
                 bc=(WALL, WALL, WALL, WALL), inflow_edge=-1, inflow_c0=0, inflow_c1=-1, rain_rate=0.0,
                 rain_t_end=0.0, max_steps=200, precision=F64, tape_views=False, _frozen=None):
        import numpy as np
        import torch
        if not torch.cuda.is_available():
            raise MwdgError(-3, "Dg2Adjoint", "no CUDA device")
        L = lib()
        p = AdjParams()
        L.mwdg_adj_params_default(C.byref(p))
        p.nx, p.ny, p.dx, p.g, p.h_dry, p.cfl, p.dt_max, p.limiter = nx, ny, dx, g, h_dry, cfl, dt_max, limiter
        for e in range(4):
            p.bc[e] = bc[e]
        p.inflow_edge, p.inflow_c0, p.inflow_c1 = inflow_edge, inflow_c0, inflow_c1
        p.rain_rate, p.rain_t_end, p.max_steps = rain_rate, rain_t_end, max_steps
        p.precision = precision
        p.tape_views = int(bool(tape_views))
        h = C.c_void_p()
        self.n_leaves = None
        if _frozen is None:
            st = L.mwdg_adj_create(C.byref(p), C.byref(h))
        else:
            M, N, Lv, mode, lev, ii, jj = _frozen
            lev, ii, jj = (np.ascontiguousarray(a, dtype=np.int32) for a in (lev, ii, jj))
            if not (lev.shape == ii.shape == jj.shape and lev.ndim == 1):
                raise MwdgError(-1, "Dg2Adjoint.frozen", "level, i, j differ in shape")
            st = L.mwdg_adj_create_frozen(C.byref(p), int(M), int(N), int(Lv), int(mode), int(lev.size),
                                          lev.ctypes.data_as(C.c_void_p), ii.ctypes.data_as(C.c_void_p),
                                          jj.ctypes.data_as(C.c_void_p), C.byref(h))
            self.n_leaves = int(lev.size)
        if st != 0:
            raise MwdgError(st, "mwdg_adj_create" if _frozen is None else "mwdg_adj_create_frozen")
        self._h = h
        self.p = p
        self.nx, self.ny, self.dx, self.max_steps = nx, ny, dx, max_steps
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.float32 if precision == F32 else torch.float64

    @classmethod
    def frozen(cls, M, N, L, dx, mode, level, i, j, **kw):
        """A context on a frozen non-uniform grid: M x N roots, L levels, finest
        cell size dx; mode STATIC (graded grid, Sect. 2.2.1) or ADAPTIVE (an
        MWDG2 grid held fixed, Sect. 2.3); the active leaves (level, i, j)."""
        if mode not in (STATIC, ADAPTIVE):
            raise MwdgError(-1, "Dg2Adjoint.frozen", "mode must be STATIC or ADAPTIVE")
        return cls(M << L, N << L, dx, _frozen=(M, N, L, mode, level, i, j), **kw)

    def _state_shape(self):
        return (9, self.n_leaves) if self.n_leaves is not None else (9, self.ny, self.nx)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().mwdg_adj_destroy(h)
            self._h = None

    def _check(self, st, where):
        if st != 0:
            raise MwdgError(st, where, lib().mwdg_adj_last_error(self._h).decode())

    def _t(self, a, shape=None, dtype=None):
        import torch
        t = torch.as_tensor(a, dtype=dtype or self.dtype, device=self.device).contiguous()
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise MwdgError(-1, "Dg2Adjoint", f"shape {tuple(t.shape)}, expected {tuple(shape)}")
        return t

    def profile(self, max_launches: int):
        """time the next `max_launches` launch groups with CUDA events (0: stop)"""
        self._check(lib().mwdg_adj_profile(self._h, int(max_launches)), "mwdg_adj_profile")

    def kernel_times(self):
        """{class: (milliseconds, launch groups)} since the last call"""
        n = len(ADJ_CLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        self._check(lib().mwdg_adj_kernel_times(self._h, ms, cnt), "mwdg_adj_kernel_times")
        return {c: (ms[k], cnt[k]) for k, c in enumerate(ADJ_CLASSES)}

    def project(self, vert):
        """Eq. 8: (ny+1, nx+1) vertex raster -> planes (3, ny, nx)."""
        import torch
        v = self._t(vert, (self.ny + 1, self.nx + 1), torch.float64)
        out = torch.empty((3, self.ny, self.nx), dtype=self.dtype, device=self.device)
        self._check(lib().mwdg_adj_project(self._h, _ptr(v), _ptr(out), _stream()), "mwdg_adj_project")
        return out

    def project_transpose(self, g_planes):
        """cotangents of the planes (3, ny, nx) -> of the vertex raster"""
        import torch
        gp = self._t(g_planes, (3, self.ny, self.nx))
        out = torch.empty((self.ny + 1, self.nx + 1), dtype=self.dtype, device=self.device)
        self._check(lib().mwdg_adj_project_transpose(self._h, _ptr(gp), _ptr(out), _stream()),
                    "mwdg_adj_project_transpose")
        return out

    def _common(self, U0, z, n, knot_t, knot_Q):
        import torch
        U0 = self._t(U0, self._state_shape())
        z = self._t(z, (3, self.ny, self.nx))
        n = self._t(n, (self.ny, self.nx))
        kt = self._t(knot_t, dtype=torch.float64) if knot_t is not None else None
        kQ = self._t(knot_Q, dtype=torch.float64) if knot_Q is not None else None
        nk = 0 if kt is None else int(kt.numel())
        if kQ is not None and int(kQ.numel()) != nk:
            raise MwdgError(-1, "Dg2Adjoint", "knot_t and knot_Q differ in length")
        return U0, z, n, kt, kQ, nk

    def forward(self, U0, z, n, knot_t, knot_Q, t0, steps, dts=None):
        """U_K after `steps` steps from U0 at t0, and the time steps (the CFL
        ones, or `dts` when given)."""
        import torch
        self._tape_token = None
        U0, z, n, kt, kQ, nk = self._common(U0, z, n, knot_t, knot_Q)
        fixed = dts is not None
        d = self._t(dts, (steps,), torch.float64) if fixed else torch.empty(max(1, steps), dtype=torch.float64,
                                                                             device=self.device)
        out = torch.empty_like(U0)
        st = lib().mwdg_adj_forward(self._h, _ptr(U0), _ptr(z), _ptr(n), nk, _ptr(kt), _ptr(kQ), float(t0),
                                    int(steps), int(fixed), _ptr(d), _ptr(out), _stream())
        self._check(st, "mwdg_adj_forward")
        return out, d[:steps]

    def backward(self, U0, z, n, knot_t, knot_Q, t0, dts, gUK, reuse_tape=False):
        """(gU0, gz, gn, gQ): the cotangents of U0, z, n and the knots, given
        that of U_K, over the steps dts from U0 at t0.  reuse_tape: the last
        forward call ran exactly this segment and nothing changed since."""
        import torch
        self._tape_token = None
        U0, z, n, kt, kQ, nk = self._common(U0, z, n, knot_t, knot_Q)
        d = self._t(dts, dtype=torch.float64)
        g = self._t(gUK, self._state_shape())
        gU0 = torch.empty_like(U0)
        gz = torch.zeros_like(z)
        gn = torch.zeros_like(n)
        gQ = torch.zeros(max(1, nk), dtype=torch.float64, device=self.device)
        st = lib().mwdg_adj_backward(self._h, _ptr(U0), _ptr(z), _ptr(n), nk, _ptr(kt), _ptr(kQ), float(t0),
                                     int(d.numel()), _ptr(d), _ptr(g), _ptr(gU0), _ptr(gz), _ptr(gn), _ptr(gQ),
                                     int(bool(reuse_tape)), _stream())
        self._check(st, "mwdg_adj_backward")
        return gU0, gz, gn, gQ[:nk]


def regrid_forward(src: "Dg2Adjoint", dst: "Dg2Adjoint", U):
    """the leaves' coefficients on dst's grid from those on src's (the
    MWDG2 adaptation's state transfer, mwdg_adj_regrid)"""
    import torch
    U = src._t(U, src._state_shape())
    out = torch.empty((9, dst.n_leaves), dtype=src.dtype, device=src.device)
    src._check(lib().mwdg_adj_regrid(src._h, dst._h, _ptr(U), _ptr(out), _stream()), "mwdg_adj_regrid")
    return out


def regrid_transpose(src: "Dg2Adjoint", dst: "Dg2Adjoint", U, gV):
    """cotangent of U (on src's grid) given gV, that of its regridding"""
    import torch
    U = src._t(U, src._state_shape())
    gV = dst._t(gV, dst._state_shape())
    out = torch.empty_like(U)
    src._check(lib().mwdg_adj_regrid_transpose(src._h, dst._h, _ptr(U), _ptr(gV), _ptr(out), _stream()),
               "mwdg_adj_regrid_transpose")
    return out


def _autograd_function():
    import torch

    class Dg2Run(torch.autograd.Function):
        """U_K = run(U0, z, n, Q) over one segment; gradients by the adjoint."""

        @staticmethod
        def forward(ctx, U0, z, n, Q, adj, knot_t, t0, steps, dts):
            UK, d = adj.forward(U0, z, n, knot_t, Q, t0, steps, dts)
            ctx.save_for_backward(U0, z, n, Q, d)
            ctx.adj, ctx.knot_t, ctx.t0 = adj, knot_t, t0
            # the context's tape holds this segment until another call
            # writes it; saved tensors cannot change (autograd's version
            # check), so the tape is valid while this token is the last
            adj._tape_token = ctx.token = object()
            ctx.mark_non_differentiable(d)
            return UK, d

        @staticmethod
        def backward(ctx, gUK, _gd):
            U0, z, n, Q, d = ctx.saved_tensors
            reuse = getattr(ctx.adj, "_tape_token", None) is ctx.token
            gU0, gz, gn, gQ = ctx.adj.backward(U0, z, n, ctx.knot_t, Q, ctx.t0, d, gUK.contiguous(),
                                               reuse_tape=reuse)
            ctx.adj._tape_token = ctx.token   # the tape holds this segment's run either way
            return gU0, gz, gn, (gQ if Q is not None and Q.numel() else None), None, None, None, None, None

    return Dg2Run


_DG2RUN = None
_REGRID = None


def _regrid_function():
    import torch

    class Regrid(torch.autograd.Function):
        """U on dst's grid from U on src's (a checkpoint's re-freezing)"""

        @staticmethod
        def forward(ctx, U, src, dst):
            ctx.save_for_backward(U)
            ctx.src, ctx.dst = src, dst
            return regrid_forward(src, dst, U)

        @staticmethod
        def backward(ctx, gV):
            (U,) = ctx.saved_tensors
            return regrid_transpose(ctx.src, ctx.dst, U, gV.contiguous()), None, None

    return Regrid


def regrid(src: Dg2Adjoint, dst: Dg2Adjoint, U):
    """Differentiable state transfer from src's frozen MWDG2 grid to dst's at
    a checkpoint: chain dg2_run(src) -> regrid -> dg2_run(dst) to
    differentiate a run whose grid is re-frozen at each checkpoint."""
    global _REGRID
    if _REGRID is None:
        _REGRID = _regrid_function()
    return _REGRID.apply(U, src, dst)


def dg2_run(adj: Dg2Adjoint, U0, z, n, Q, knot_t, t0: float, steps: int, dts=None):
    """One differentiable segment: returns (U_K, dts, t_K) with t_K the time
    after the segment (the steps summed in order, as the device does)."""
    global _DG2RUN
    if _DG2RUN is None:
        _DG2RUN = _autograd_function()
    UK, d = _DG2RUN.apply(U0, z, n, Q, adj, knot_t, float(t0), int(steps), dts)
    t = float(t0)
    for v in d.detach().cpu().tolist():
        t = t + v
    return UK, d, t
