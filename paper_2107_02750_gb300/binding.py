"""ctypes binding of libmwdg (include/mwdg.h).  Argument marshalling only:
every step of the solver runs in the library's CUDA kernels.  The method
names follow the C entry points (``mwdg_load_dem`` -> ``Solver.load_dem``)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

UNIFORM, STATIC, ADAPTIVE = 0, 1, 2
F64, F32 = 0, 1
DG2, FV1, ACC = 0, 1, 2
WALL, OPEN = 0, 1
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3

EXPORTS = (
    "mwdg_params_default", "mwdg_create", "mwdg_destroy", "mwdg_load_dem", "mwdg_load_roughness",
    "mwdg_load_dem_dev", "mwdg_load_roughness_dev", "mwdg_load_initial_dev",
    "mwdg_set_roughness_scalar", "mwdg_load_initial", "mwdg_set_inflow", "mwdg_set_rain",
    "mwdg_mra_encode", "mwdg_mra_adapt", "mwdg_dg2_step", "mwdg_dg2_step_dt", "mwdg_run_steps", "mwdg_run_to_time",
    "mwdg_read_fields", "mwdg_read_fields_dev", "mwdg_read_active", "mwdg_get_time",
    "mwdg_get_volume", "mwdg_profile", "mwdg_kernel_times", "mwdg_launch_count",
    "mwdg_last_error", "mwdg_status_string", "mwdg_state_bytes", "mwdg_save_state",
    "mwdg_load_state", "mwdg_volume_noalloc", "mwdg_fma_rate", "mwdg_get_counters", "mwdg_read_gauges",
    "mwdg_set_launch_shape", "mwdg_get_launch_shape", "mwdg_ensemble_create", "mwdg_ensemble_destroy",
    "mwdg_ensemble_step", "mwdg_ensemble_run_to_time", "mwdg_ensemble_tune", "mwdg_ensemble_set_batched",
    "mwdg_ensemble_last_error",
)


class Params(C.Structure):
    _fields_ = [
        ("M", C.c_int32), ("N", C.c_int32), ("L", C.c_int32), ("mode", C.c_int32),
        ("precision", C.c_int32), ("limiter", C.c_int32), ("bc", C.c_int32 * 4),
        ("iface_rule", C.c_int32), ("scheme", C.c_int32), ("dx", C.c_double), ("eps", C.c_double), ("cfl", C.c_double), ("g", C.c_double),
        ("h_dry", C.c_double), ("dt_max", C.c_double), ("cuda_stream", C.c_void_p),
    ]


class MwdgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where} failed with status {status}"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_lib = None


def lib(build: bool = True):
    """Load libmwdg (compiling it in-tree first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.lib_path()
    if not path.exists():
        raise RuntimeError(f"libmwdg is not built ({path}); call __graft_entry__.build()")
    L = C.CDLL(str(path))
    vp, dp, ip, lp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    sig = {
        "mwdg_params_default": [C.POINTER(Params)],
        "mwdg_create": [C.POINTER(Params), C.POINTER(C.c_void_p)],
        "mwdg_load_dem": [vp, dp, C.c_int64],
        "mwdg_load_dem_dev": [vp, vp, C.c_int64],
        "mwdg_load_roughness": [vp, dp, C.c_int64],
        "mwdg_load_roughness_dev": [vp, vp, C.c_int64],
        "mwdg_load_initial_dev": [vp, vp, vp, vp, C.c_int64, C.c_int32],
        "mwdg_set_roughness_scalar": [vp, C.c_double],
        "mwdg_load_initial": [vp, dp, dp, dp, C.c_int32],
        "mwdg_set_inflow": [vp, C.c_int32, C.c_int32, C.c_int32, dp, dp, C.c_int32],
        "mwdg_set_rain": [vp, C.c_double, C.c_double],
        "mwdg_mra_encode": [vp],
        "mwdg_mra_adapt": [vp, C.c_double, lp],
        "mwdg_dg2_step": [vp, dp],
        "mwdg_dg2_step_dt": [vp, C.c_double],
        "mwdg_fma_rate": [C.c_int32, vp, dp],
        "mwdg_run_steps": [vp, C.c_int64],
        "mwdg_run_to_time": [vp, C.c_double, lp],
        "mwdg_read_fields": [vp, dp, dp, dp, C.c_int64],
        "mwdg_read_fields_dev": [vp, vp, vp, vp, C.c_int64],
        "mwdg_read_gauges": [vp, ip, C.c_int32, dp, dp, dp],
        "mwdg_set_launch_shape": [vp, C.c_int32, C.c_int64],
        "mwdg_get_launch_shape": [vp, ip, lp],
        "mwdg_ensemble_create": [C.POINTER(C.c_void_p), C.c_int32, vp, C.POINTER(C.c_void_p)],
        "mwdg_ensemble_step": [vp, C.c_int64],
        "mwdg_ensemble_run_to_time": [vp, C.c_double, lp],
        "mwdg_ensemble_tune": [vp, C.c_int32, lp],
        "mwdg_ensemble_set_batched": [vp, C.c_int32],
        "mwdg_read_active": [vp, ip, ip, ip, dp, C.c_int64, lp],
        "mwdg_get_time": [vp, dp, lp],
        "mwdg_get_counters": [vp, lp, lp],
        "mwdg_get_volume": [vp, dp, dp, dp, dp, dp, lp],
        "mwdg_profile": [vp, C.c_int32],
        "mwdg_kernel_times": [vp, C.POINTER(C.c_char_p), dp, lp, C.c_int32, ip],
        "mwdg_launch_count": [vp, lp],
        "mwdg_state_bytes": [vp, lp],
        "mwdg_save_state": [vp, vp, C.c_int64],
        "mwdg_load_state": [vp, vp, C.c_int64],
        "mwdg_volume_noalloc": [vp, vp, C.c_int64, C.c_double, C.c_int32, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.mwdg_destroy.argtypes = [vp]
    L.mwdg_destroy.restype = None
    L.mwdg_ensemble_destroy.argtypes = [vp]
    L.mwdg_ensemble_destroy.restype = None
    L.mwdg_ensemble_last_error.argtypes = [vp]
    L.mwdg_ensemble_last_error.restype = C.c_char_p
    L.mwdg_last_error.argtypes = [vp]
    L.mwdg_last_error.restype = C.c_char_p
    L.mwdg_status_string.argtypes = [C.c_int]
    L.mwdg_status_string.restype = C.c_char_p
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Solver:
    """One simulation context (mwdg_ctx) on the current CUDA device."""

    def __init__(self, *, M, N, L, dx, mode=UNIFORM, precision=F64, eps=1e-3, cfl=0.33,
                 g=9.80665, h_dry=1e-3, dt_max=1.0, limiter=1, bc=(WALL,) * 4, iface_rule=0, scheme=0,
                 stream=None):
        self._lib = lib()
        p = Params()
        self._lib.mwdg_params_default(C.byref(p))
        p.M, p.N, p.L, p.mode, p.precision, p.limiter = M, N, L, mode, precision, limiter
        p.iface_rule = iface_rule
        p.scheme = scheme
        for k in range(4):
            p.bc[k] = bc[k]
        p.dx, p.eps, p.cfl, p.g, p.h_dry, p.dt_max = dx, eps, cfl, g, h_dry, dt_max
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        p.cuda_stream = stream
        self.p = p
        self.nx, self.ny = M << L, N << L
        # finest level of the reported active leaves (a uniform grid is one level)
        self.levels = 0 if mode == UNIFORM else L
        h = C.c_void_p()
        st = self._lib.mwdg_create(C.byref(p), C.byref(h))
        if st != 0:
            raise MwdgError(st, "mwdg_create", self._lib.mwdg_status_string(st).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mwdg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st, where):
        if st != 0:
            raise MwdgError(st, where, self._lib.mwdg_last_error(self._h).decode())

    # --- inputs --------------------------------------------------------------
    def load_dem(self, z_vert):
        z = _f64(z_vert)
        assert z.shape == (self.ny + 1, self.nx + 1)
        self._ck(self._lib.mwdg_load_dem(self._h, _dp(z), 0), "mwdg_load_dem")

    def load_roughness(self, n_cell):
        a = _f64(np.broadcast_to(np.asarray(n_cell, np.float64), (self.ny, self.nx)))
        self._ck(self._lib.mwdg_load_roughness(self._h, _dp(a), 0), "mwdg_load_roughness")

    @staticmethod
    def _dev2d(t, rows, cols, what):
        """a CUDA FP64 tensor of rows x cols whose rows are contiguous: its
        pointer and row stride"""
        if t.dtype != __import__("torch").float64 or not t.is_cuda or t.dim() != 2 or tuple(t.shape) != (rows, cols) \
                or t.stride(1) != 1:
            raise ValueError(f"{what}: expected a CUDA float64 tensor of shape ({rows}, {cols}) with unit column "
                             "stride")
        return C.c_void_p(t.data_ptr()), t.stride(0)

    def load_dem_dev(self, z_vert):
        """the DEM from a CUDA tensor (ny+1, nx+1), rows possibly strided"""
        zp, ld = self._dev2d(z_vert, self.ny + 1, self.nx + 1, "z_vert")
        self._ck(self._lib.mwdg_load_dem_dev(self._h, zp, ld), "mwdg_load_dem_dev")

    def load_roughness_dev(self, n_cell):
        """Manning n from a CUDA tensor (ny, nx), rows possibly strided"""
        np_, ld = self._dev2d(n_cell, self.ny, self.nx, "n_cell")
        self._ck(self._lib.mwdg_load_roughness_dev(self._h, np_, ld), "mwdg_load_roughness_dev")

    def load_initial_dev(self, h_vert, qx_vert, qy_vert, is_eta=False):
        """the initial state from three CUDA tensors (ny+1, nx+1) with one row stride"""
        ptrs = [self._dev2d(t, self.ny + 1, self.nx + 1, "initial raster") for t in (h_vert, qx_vert, qy_vert)]
        if len({ld for _, ld in ptrs}) != 1:
            raise ValueError("the three initial rasters must share one row stride")
        self._ck(self._lib.mwdg_load_initial_dev(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[0][1],
                                                 int(is_eta)), "mwdg_load_initial_dev")

    def set_roughness_scalar(self, n):
        self._ck(self._lib.mwdg_set_roughness_scalar(self._h, float(n)), "mwdg_set_roughness_scalar")

    def load_initial(self, h_vert, qx_vert=None, qy_vert=None, is_eta=False):
        shape = (self.ny + 1, self.nx + 1)
        h = _f64(h_vert)
        qx = _f64(np.zeros(shape) if qx_vert is None else qx_vert)
        qy = _f64(np.zeros(shape) if qy_vert is None else qy_vert)
        self._ck(self._lib.mwdg_load_initial(self._h, _dp(h), _dp(qx), _dp(qy), int(is_eta)),
                 "mwdg_load_initial")

    def set_inflow(self, edge, c0, c1, t, Q):
        t, Q = _f64(t), _f64(Q)
        self._ck(self._lib.mwdg_set_inflow(self._h, edge, c0, c1, _dp(t), _dp(Q), len(t)),
                 "mwdg_set_inflow")

    def set_rain(self, rate, t_stop):
        self._ck(self._lib.mwdg_set_rain(self._h, float(rate), float(t_stop)), "mwdg_set_rain")

    # --- MRA and stepping ----------------------------------------------------
    def mra_encode(self):
        self._ck(self._lib.mwdg_mra_encode(self._h), "mwdg_mra_encode")

    def mra_adapt(self, eps) -> int:
        n = C.c_int64()
        self._ck(self._lib.mwdg_mra_adapt(self._h, float(eps), C.byref(n)), "mwdg_mra_adapt")
        return n.value

    def dg2_step(self) -> float:
        dt = C.c_double()
        self._ck(self._lib.mwdg_dg2_step(self._h, C.byref(dt)), "mwdg_dg2_step")
        return dt.value

    def dg2_step_dt(self, dt):
        """one step of the prescribed length dt (no CFL condition)"""
        self._ck(self._lib.mwdg_dg2_step_dt(self._h, float(dt)), "mwdg_dg2_step_dt")

    def run_steps(self, n):
        self._ck(self._lib.mwdg_run_steps(self._h, int(n)), "mwdg_run_steps")

    def run_to_time(self, t_end) -> int:
        n = C.c_int64()
        self._ck(self._lib.mwdg_run_to_time(self._h, float(t_end), C.byref(n)), "mwdg_run_to_time")
        return n.value

    # --- outputs -------------------------------------------------------------
    def read_fields(self):
        h, u, v = (np.empty((self.ny, self.nx)) for _ in range(3))
        self._ck(self._lib.mwdg_read_fields(self._h, _dp(h), _dp(u), _dp(v), 0), "mwdg_read_fields")
        return h, u, v

    def read_fields_dev(self, h=None, u=None, v=None):
        """fill FP64 CUDA tensors of shape (ny, nx) (any may be None; rows
        possibly strided, one row stride for all)"""
        given = [x for x in (h, u, v) if x is not None]
        lds = {self._dev2d(x, self.ny, self.nx, "field")[1] for x in given}
        if len(lds) > 1:
            raise ValueError("the field tensors must share one row stride")
        ld = lds.pop() if lds else 0
        ptr = lambda x: None if x is None else C.c_void_p(x.data_ptr())
        self._ck(self._lib.mwdg_read_fields_dev(self._h, ptr(h), ptr(u), ptr(v), ld), "mwdg_read_fields_dev")

    def read_gauges(self, cells):
        """h, u, v at finest cells given as an (n, 2) array of (i, j)"""
        ij = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 2))
        n = ij.shape[0]
        h, u, v = (np.empty(n) for _ in range(3))
        self._ck(self._lib.mwdg_read_gauges(self._h, _ip(ij), n, _dp(h), _dp(u), _dp(v)), "mwdg_read_gauges")
        return h, u, v

    def read_active(self):
        n = C.c_int64()
        self._ck(self._lib.mwdg_read_active(self._h, None, None, None, None, 0, C.byref(n)),
                 "mwdg_read_active")
        cnt = n.value
        lev = np.empty(cnt, np.int32)
        ii = np.empty(cnt, np.int32)
        jj = np.empty(cnt, np.int32)
        co = np.empty((cnt, 9))
        self._ck(self._lib.mwdg_read_active(self._h, _ip(lev), _ip(ii), _ip(jj), _dp(co), cnt,
                                            C.byref(n)), "mwdg_read_active")
        return lev, ii, jj, co

    def n_active(self) -> int:
        n = C.c_int64()
        self._ck(self._lib.mwdg_read_active(self._h, None, None, None, None, 0, C.byref(n)),
                 "mwdg_read_active")
        return n.value

    def get_time(self):
        t, s = C.c_double(), C.c_int64()
        self._ck(self._lib.mwdg_get_time(self._h, C.byref(t), C.byref(s)), "mwdg_get_time")
        return t.value, s.value

    def get_counters(self):
        """(steps, active-leaf updates) since the initial state"""
        s, u = C.c_int64(), C.c_int64()
        self._ck(self._lib.mwdg_get_counters(self._h, C.byref(s), C.byref(u)), "mwdg_get_counters")
        return s.value, u.value

    def get_volume(self) -> dict:
        v = [C.c_double() for _ in range(5)]
        n = C.c_int64()
        self._ck(self._lib.mwdg_get_volume(self._h, *(C.byref(x) for x in v), C.byref(n)),
                 "mwdg_get_volume")
        return dict(volume=v[0].value, v_in=v[1].value, v_out=v[2].value, v_rain=v[3].value,
                    v_clip=v[4].value, n_clip=n.value)

    def profile(self, enable: bool):
        self._ck(self._lib.mwdg_profile(self._h, int(enable)), "mwdg_profile")

    def kernel_times(self) -> dict:
        cap = 32
        names = (C.c_char_p * cap)()
        ms = np.zeros(cap)
        cnt = np.zeros(cap, np.int64)
        n = C.c_int32()
        self._ck(self._lib.mwdg_kernel_times(self._h, names, _dp(ms),
                                             cnt.ctypes.data_as(C.POINTER(C.c_int64)), cap,
                                             C.byref(n)), "mwdg_kernel_times")
        return {names[k].decode(): (float(ms[k]), int(cnt[k])) for k in range(n.value)}

    def state_bytes(self) -> int:
        n = C.c_int64()
        self._ck(self._lib.mwdg_state_bytes(self._h, C.byref(n)), "mwdg_state_bytes")
        return n.value

    def save_state(self, buf=None):
        """checkpoint into a host buffer (numpy uint8, or a pinned torch uint8
        tensor); returns the buffer"""
        n = self.state_bytes()
        if buf is None:
            buf = np.empty(n, np.uint8)
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else buf.data_ptr()
        self._ck(self._lib.mwdg_save_state(self._h, C.c_void_p(ptr), n), "mwdg_save_state")
        return buf

    def load_state(self, buf):
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else buf.data_ptr()
        n = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel()
        self._ck(self._lib.mwdg_load_state(self._h, C.c_void_p(ptr), n), "mwdg_load_state")

    def launch_count(self) -> int:
        n = C.c_int64()
        self._ck(self._lib.mwdg_launch_count(self._h, C.byref(n)), "mwdg_launch_count")
        return n.value

    def set_launch_shape(self, grid_leaves=0, coarse_nodes=0):
        self._ck(self._lib.mwdg_set_launch_shape(self._h, int(grid_leaves), int(coarse_nodes)),
                 "mwdg_set_launch_shape")

    def launch_shape(self):
        g, c = C.c_int32(), C.c_int64()
        self._ck(self._lib.mwdg_get_launch_shape(self._h, C.byref(g), C.byref(c)), "mwdg_get_launch_shape")
        return g.value, c.value


class Ensemble:
    """Members (Solver objects on one device) stepped together, one CUDA graph
    per ensemble step: each member's step a parallel branch, or with batch = g
    >= 2 the adaptive DG2 members of one precision in groups of g, each group's
    step one launch per kernel over its members' blocks."""

    def __init__(self, members, stream=None, batch=0):
        self._lib = lib()
        self.members = list(members)  # keeps them alive
        n = len(self.members)
        arr = (C.c_void_p * n)(*[m._h.value for m in self.members])
        h = C.c_void_p()
        st = self._lib.mwdg_ensemble_create(arr, n, None if stream is None else C.c_void_p(stream), C.byref(h))
        if st != 0:
            raise MwdgError(st, "mwdg_ensemble_create", self._lib.mwdg_status_string(st).decode())
        self._h = h
        if batch:
            self.set_batch(batch)

    def set_batch(self, group: int):
        """members per batched group (0: one graph branch per member)"""
        self._ck(self._lib.mwdg_ensemble_set_batched(self._h, int(group)), "mwdg_ensemble_set_batched")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mwdg_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st, where):
        if st != 0:
            raise MwdgError(st, where, self._lib.mwdg_ensemble_last_error(self._h).decode())

    def step(self, n=1):
        self._ck(self._lib.mwdg_ensemble_step(self._h, int(n)), "mwdg_ensemble_step")

    def run_to_time(self, t_end) -> int:
        n = C.c_int64()
        self._ck(self._lib.mwdg_ensemble_run_to_time(self._h, float(t_end), C.byref(n)),
                 "mwdg_ensemble_run_to_time")
        return n.value

    def tune(self, steps=8):
        """autotune every member's launch shape; returns (n, 2) (grid_leaves, coarse_nodes)"""
        out = np.zeros(2 * len(self.members), np.int64)
        self._ck(self._lib.mwdg_ensemble_tune(self._h, int(steps), out.ctypes.data_as(C.POINTER(C.c_int64))),
                 "mwdg_ensemble_tune")
        return out.reshape(-1, 2)


def fma_rate(precision=F64, stream=None) -> float:
    """measured FMA rate of the current device's FP64 or FP32 pipes (flop/s)"""
    L = lib()
    out = C.c_double()
    st = L.mwdg_fma_rate(int(precision), C.c_void_p(stream or 0), C.byref(out))
    if st != 0:
        raise MwdgError(st, "mwdg_fma_rate")
    return out.value


def solver_from_problem(p, precision=F64, stream=None, **over) -> Solver:
    """A Solver loaded with a synthetic problem (paper_2107_02750_gb300.synth)."""
    kw = dict(M=p.M, N=p.N, L=p.L, dx=p.dx, mode=p.mode, precision=precision, eps=p.eps,
              limiter=p.limiter, bc=p.bc, dt_max=p.dt_max, iface_rule=p.iface_rule, scheme=p.scheme,
              cfl=p.cfl, stream=stream)
    kw.update(over)
    s = Solver(**kw)
    s.load_dem(p.z_vert)
    nm = np.asarray(p.n_manning)
    if nm.ndim == 0:
        s.set_roughness_scalar(float(nm))
    else:
        s.load_roughness(p.n_cell())
    if len(p.inflow_t):
        s.set_inflow(p.inflow_edge, p.inflow_c0, p.inflow_c1, p.inflow_t, p.inflow_Q)
    if p.rain_rate > 0:
        s.set_rain(p.rain_rate, p.rain_t_end)
    s.load_initial(p.h_vert, p.qx_vert, p.qy_vert, p.is_eta)
    return s
