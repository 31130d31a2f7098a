"""FP64 CPU oracle for the DG2 / multiwavelet-MRA flood solvers (arXiv 2107.02750).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, per-element reference
that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The product package never imports it and has no CPU fallback.

The C source (``mwdg2_oracle.c``) is compiled here with ``gcc -O2
-ffp-contract=off`` (no FMA contraction) into ``oracle/_build``; this module is
argument marshalling over ctypes plus the flood-extent metrics of Sect. 2
(Eq. 11 and the H/F/C scores).

Parity status of the oracle's functions (what pins each one is listed in the
tests):
  project (Eq. 8)                 pinned: L2 projection of the bilinear vertex
                                  interpolant by quadrature, planar DEMs exact
  lowpass/highpass filters        pinned: orthogonality, closed-form entries,
                                  quadrature projection, Parseval
  encode / decode (Eq. 9-10)      pinned: lossless round trip, planar fields
                                  give zero details
  threshold / closure / grading   pinned: brute force from quadrature details
                                  on tiny grids, tiling and 2:1 invariants;
                                  MWDG2 regridding (normalisation, prediction,
                                  closure) by brute force on a tiny grid
  DG2 step (Eq. 4, HLL, revisions) pinned: lake at rest (wet and with
                                  islands), Ritter and Stoker dam breaks,
                                  volume conservation, D4 symmetry
  outflow limit (non-negative      pinned: no clipped depth and the mass budget
  depths at wet/dry fronts)       closed without clipped volume on the valley
                                  window through the inflow and on a dam
                                  break over a steep dry slope; a mound drained
                                  in one stage ends at zero; a scratch copy
                                  without the limit fails each of these
  friction                        pinned: exact decay of a uniform flow; the
                                  Manning normal depth of a sloped channel
  limiter                         pinned: hand-evaluated minmod cases (through
                                  the bit-exact restatement in dg2_adjoint.py)
  non-homogeneous interface rule  pinned on planar data: one stage on a
                                  non-uniform grid equals, leaf by leaf, the
                                  stage on the uniform grid of each leaf's
                                  level (static and adaptive); elsewhere by
                                  the invariants above
  discrete adjoint of the uniform DG2 step (dg2_adjoint.py, PyTorch CPU
  autograd over a restatement of the step):
                                  pinned: bit-for-bit forward against the C
                                  step, central differences of the C step
  the same on frozen non-uniform grids (dg2_adjoint_nonuniform.py, static
  graded and MWDG2 grids held over a segment):
                                  pinned the same way
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "mwdg2_oracle.c"
_BUILD = _HERE / "_build"

UNIFORM, STATIC, ADAPTIVE = 0, 1, 2
WALL, OPEN = 0, 1
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3


def _lib_path() -> Path:
    return _BUILD / f"liborc_{platform.machine()}.so"


def build(force: bool = False) -> Path:
    """Compile the oracle (idempotent)."""
    out = _lib_path()
    if not force and out.exists() and out.stat().st_mtime >= _SRC.stat().st_mtime:
        return out
    _BUILD.mkdir(exist_ok=True)
    tmp = out.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-shared", "-fPIC",
           str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Params(C.Structure):
    _fields_ = [
        ("M", C.c_int32), ("N", C.c_int32), ("L", C.c_int32), ("mode", C.c_int32),
        ("R", C.c_double), ("eps", C.c_double), ("cfl", C.c_double), ("g", C.c_double),
        ("h_dry", C.c_double), ("dt_max", C.c_double),
        ("limiter", C.c_int32), ("bc", C.c_int32 * 4),
        ("inflow_edge", C.c_int32), ("inflow_c0", C.c_int32), ("inflow_c1", C.c_int32),
        ("rain_rate", C.c_double), ("rain_t_end", C.c_double),
        ("iface_rule", C.c_int32), ("scheme", C.c_int32),
    ]


_lib = None


def load(path) -> C.CDLL:
    """The oracle's entry points from a compiled copy at path, typed."""
    L = C.CDLL(str(path))
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(Params)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_levels.restype = C.c_int
    L.orc_levels.argtypes = [C.c_void_p]
    for name in ("orc_load_dem", "orc_load_roughness"):
        getattr(L, name).argtypes = [C.c_void_p, dp]
    L.orc_load_initial.argtypes = [C.c_void_p, dp, dp, dp, C.c_int]
    L.orc_set_inflow.argtypes = [C.c_void_p, C.c_int, dp, dp]
    L.orc_init_grid.argtypes = [C.c_void_p]
    L.orc_adapt.argtypes = [C.c_void_p]
    L.orc_step.restype = C.c_double
    L.orc_step.argtypes = [C.c_void_p, C.c_double]
    L.orc_stage.argtypes = [C.c_void_p, C.c_double]
    L.orc_step_frozen.restype = C.c_double
    L.orc_step_frozen.argtypes = [C.c_void_p, C.c_double]
    L.orc_step_dt.restype = C.c_double
    L.orc_step_dt.argtypes = [C.c_void_p, C.c_double]
    L.orc_run_to.restype = C.c_int64
    L.orc_run_to.argtypes = [C.c_void_p, C.c_double, C.c_int64]
    L.orc_time.restype = C.c_double
    L.orc_time.argtypes = [C.c_void_p]
    L.orc_steps.restype = C.c_int64
    L.orc_steps.argtypes = [C.c_void_p]
    L.orc_last_dt.restype = C.c_double
    L.orc_last_dt.argtypes = [C.c_void_p]
    L.orc_diag.argtypes = [C.c_void_p, dp]
    L.orc_n_leaves.restype = C.c_int64
    L.orc_n_leaves.argtypes = [C.c_void_p]
    L.orc_get_leaves.argtypes = [C.c_void_p, ip, ip, ip, dp]
    L.orc_read_fields.argtypes = [C.c_void_p, dp, dp, dp]
    L.orc_get_z.argtypes = [C.c_void_p, C.c_int, dp, dp]
    L.orc_project.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp]
    L.orc_filters.argtypes = [dp, dp]
    L.orc_encode_node.argtypes = [dp, dp, dp]
    L.orc_decode_node.argtypes = [dp, dp, dp]
    L.orc_haar_encode.argtypes = [dp, dp, dp]
    L.orc_haar_decode.argtypes = [C.c_double, dp, dp]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Stateless pieces
# ---------------------------------------------------------------------------
def project(vert: np.ndarray):
    """Eq. 8: (ny+1, nx+1) vertex raster -> (c0, c1x, c1y), each (ny, nx)."""
    v = _f64(vert)
    ny, nx = v.shape[0] - 1, v.shape[1] - 1
    out = [np.empty((ny, nx)) for _ in range(3)]
    lib().orc_project(_dp(v), nx, ny, *(_dp(o) for o in out))
    return tuple(out)


def filters():
    """(A, G): A[c] the 3x3 low-pass, G[c] the 9x3 high-pass of child c."""
    A = np.empty((4, 3, 3))
    G = np.empty((4, 9, 3))
    lib().orc_filters(_dp(A), _dp(G))
    return A, G


def encode_node(children: np.ndarray):
    """Eq. 9 for one variable: children (4, 3) -> (parent (3,), details (9,))."""
    ch = _f64(children).reshape(12)
    sp, d = np.empty(3), np.empty(9)
    lib().orc_encode_node(_dp(ch), _dp(sp), _dp(d))
    return sp, d


def haar_encode(children: np.ndarray):
    """Haar wavelets (HWFV1): four child averages -> (parent average, 3 details)."""
    sc = _f64(children).reshape(4)
    p, d = np.empty(1), np.empty(3)
    lib().orc_haar_encode(_dp(sc), _dp(p), _dp(d))
    return float(p[0]), d


def haar_decode(parent: float, details: np.ndarray):
    d = _f64(details)
    out = np.empty(4)
    lib().orc_haar_decode(float(parent), _dp(d), _dp(out))
    return out


def decode_node(parent: np.ndarray, details: np.ndarray):
    """Eq. 10 for one variable: -> children (4, 3)."""
    sp, d = _f64(parent), _f64(details)
    out = np.empty(12)
    lib().orc_decode_node(_dp(sp), _dp(d), _dp(out))
    return out.reshape(4, 3)


# ---------------------------------------------------------------------------
# Simulation
# ---------------------------------------------------------------------------
class Sim:
    """One oracle simulation.  Arrays follow the raster convention: row j runs
    south to north, column i west to east."""

    def __init__(self, *, M, N, L, R, mode=UNIFORM, eps=1e-3, cfl=0.33, g=9.80665,
                 h_dry=1e-3, dt_max=1.0, limiter=1, bc=(WALL, WALL, WALL, WALL),
                 inflow_edge=-1, inflow_c0=0, inflow_c1=-1, rain_rate=0.0, rain_t_end=0.0,
                 iface_rule=0, scheme=0, library=None):
        self._L = library if library is not None else lib()
        p = Params()
        p.M, p.N, p.L, p.mode = M, N, L, mode
        p.R, p.eps, p.cfl, p.g, p.h_dry, p.dt_max = R, eps, cfl, g, h_dry, dt_max
        p.limiter = limiter
        for k in range(4):
            p.bc[k] = bc[k]
        p.inflow_edge, p.inflow_c0, p.inflow_c1 = inflow_edge, inflow_c0, inflow_c1
        p.rain_rate, p.rain_t_end = rain_rate, rain_t_end
        p.iface_rule = iface_rule
        p.scheme = scheme
        self.p = p
        self.nx, self.ny = M << L, N << L
        self._h = self._L.orc_create(C.byref(p))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    def load_dem(self, z_vert):
        z = _f64(z_vert)
        assert z.shape == (self.ny + 1, self.nx + 1)
        self._L.orc_load_dem(self._h, _dp(z))

    def load_roughness(self, n):
        a = np.broadcast_to(np.asarray(n, dtype=np.float64), (self.ny, self.nx))
        a = _f64(a)
        self._L.orc_load_roughness(self._h, _dp(a))

    def load_initial(self, h_vert, qx_vert=None, qy_vert=None, is_eta=False):
        shape = (self.ny + 1, self.nx + 1)
        h = _f64(h_vert)
        qx = _f64(np.zeros(shape) if qx_vert is None else qx_vert)
        qy = _f64(np.zeros(shape) if qy_vert is None else qy_vert)
        assert h.shape == shape and qx.shape == shape and qy.shape == shape
        self._L.orc_load_initial(self._h, _dp(h), _dp(qx), _dp(qy), int(is_eta))

    def set_inflow(self, t, Q):
        t, Q = _f64(t), _f64(Q)
        self._L.orc_set_inflow(self._h, len(t), _dp(t), _dp(Q))

    def init_grid(self):
        self._L.orc_init_grid(self._h)

    def adapt(self):
        self._L.orc_adapt(self._h)

    def step(self, t_end=float("inf")) -> float:
        return self._L.orc_step(self._h, t_end)

    def step_dt(self, dt) -> float:
        """one step with the given dt (the CFL condition is not applied)"""
        return self._L.orc_step_dt(self._h, dt)

    def step_frozen(self, dt) -> float:
        """one step with the given dt on the current active set (no MWDG2
        regridding at its start)"""
        return self._L.orc_step_frozen(self._h, dt)

    def stage(self, dt):
        """one forward-Euler stage of Eq. 4a on the current leaves (no
        adaptation, rain, friction or clock advance)"""
        self._L.orc_stage(self._h, dt)

    def run_to(self, t_end, max_steps=1 << 40) -> int:
        return self._L.orc_run_to(self._h, t_end, max_steps)

    @property
    def t(self) -> float:
        return self._L.orc_time(self._h)

    @property
    def steps(self) -> int:
        return self._L.orc_steps(self._h)

    @property
    def last_dt(self) -> float:
        return self._L.orc_last_dt(self._h)

    def diag(self) -> dict:
        out = np.empty(6)
        self._L.orc_diag(self._h, _dp(out))
        return dict(volume=out[0], v_in=out[1], v_out=out[2], v_rain=out[3], v_clip=out[4],
                    n_clip=int(out[5]))

    def leaves(self):
        """(level, i, j, coeffs (n, 9)) ordered by level then row-major."""
        n = self._L.orc_n_leaves(self._h)
        lev = np.empty(n, np.int32)
        ii = np.empty(n, np.int32)
        jj = np.empty(n, np.int32)
        co = np.empty((n, 9))
        self._L.orc_get_leaves(self._h, _ip(lev), _ip(ii), _ip(jj), _dp(co))
        return lev, ii, jj, co

    def fields(self):
        """finest-resolution (h, u, v), each (ny, nx)."""
        h, u, v = (np.empty((self.ny, self.nx)) for _ in range(3))
        self._L.orc_read_fields(self._h, _dp(h), _dp(u), _dp(v))
        return h, u, v

    def z_level(self, level):
        """static topography pyramid at a stored level: (coeffs (3, n), dz (n,))."""
        Ls = self._L.orc_levels(self._h)
        nl = (self.p.M << level) * (self.p.N << level) if Ls > 0 else self.nx * self.ny
        z = np.empty(3 * nl)
        dz = np.empty(nl)
        self._L.orc_get_z(self._h, level, _dp(z), _dp(dz))
        return z.reshape(3, nl), dz


# ---------------------------------------------------------------------------
# Evaluation metrics (Sect. 2, Eq. 11 and the flood-extent scores)
# ---------------------------------------------------------------------------
def rmse(p, p_ref) -> float:
    """Eq. 11 over the N_s samples of a time series (the printed summation
    index is garbled; the sum runs over the same N_s samples as the divisor)."""
    p, p_ref = np.asarray(p, np.float64), np.asarray(p_ref, np.float64)
    return float(np.sqrt(np.sum((p - p_ref) ** 2) / p.size))


def extent_scores(h, h_ref, wet=0.01):
    """Hit rate H = A/(A+C), false alarm F = B/(A+B), critical success index
    C = A/(A+B+C) of the wet extents (depth > `wet` metres; the paper gives
    no threshold)."""
    m = np.asarray(h) > wet
    r = np.asarray(h_ref) > wet
    A = int(np.sum(m & r))
    B = int(np.sum(m & ~r))
    Cc = int(np.sum(~m & r))
    H = A / (A + Cc) if A + Cc else 1.0
    F = B / (A + B) if A + B else 0.0
    CSI = A / (A + B + Cc) if A + B + Cc else 1.0
    return H, F, CSI
