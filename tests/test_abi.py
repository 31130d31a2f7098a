"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/*.h declares (no compute calls: no GPU needed)."""
import re
from pathlib import Path

import pytest

from paper_2107_02750_gb300 import adjoint, binding, build

INCLUDE = Path(__file__).resolve().parents[1] / "include"


def declared():
    text = "".join(h.read_text() for h in sorted(INCLUDE.glob("*.h")))
    return sorted(set(re.findall(r"MWDG_API[^;(]*?\b(mwdg_\w+)\s*\(", text, flags=re.S)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("mwdg_create", "mwdg_load_dem", "mwdg_load_roughness", "mwdg_set_inflow",
                 "mwdg_mra_encode", "mwdg_mra_adapt", "mwdg_dg2_step", "mwdg_run_to_time",
                 "mwdg_read_fields", "mwdg_read_active", "mwdg_get_volume", "mwdg_adj_forward",
                 "mwdg_adj_backward"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = binding.lib()
    assert Path(L._name).name == build.lib_path().name
    for name in declared():
        assert hasattr(L, name), name
    assert set(binding.EXPORTS) <= set(declared())
    assert set(adjoint.ADJ_EXPORTS) <= set(declared())


def test_status_strings_and_defaults_without_device():
    import ctypes as C
    L = binding.lib()
    assert L.mwdg_status_string(0) == b"ok"
    p = binding.Params()
    assert L.mwdg_params_default(C.byref(p)) == 0
    assert (p.M, p.N, p.L, p.mode, p.precision) == (1, 1, 0, 0, 0)
    assert abs(p.cfl - 0.33) < 1e-15 and p.dx == 1.0
    # argument validation happens before any device work
    bad = binding.Params()
    L.mwdg_params_default(C.byref(bad))
    bad.L = 99
    h = C.c_void_p()
    assert L.mwdg_create(C.byref(bad), C.byref(h)) == -2
    bad.L, bad.M = 0, 0
    assert L.mwdg_create(C.byref(bad), C.byref(h)) == -2
    assert L.mwdg_create(None, C.byref(h)) == -1


def test_adjoint_parameters_are_validated_without_device():
    """mwdg_adj_create rejects bad sizes and parameters before any device
    work (no GPU needed for these answers)."""
    import ctypes as C
    L = adjoint.lib()
    h = C.c_void_p()
    assert L.mwdg_adj_create(None, C.byref(h)) == -1

    def create(**kw):
        p = adjoint.AdjParams()
        assert L.mwdg_adj_params_default(C.byref(p)) == 0
        p.nx, p.ny, p.dx = 8, 8, 1.0
        for k, v in kw.items():
            setattr(p, k, v)
        return L.mwdg_adj_create(C.byref(p), C.byref(h))

    p = adjoint.AdjParams()
    L.mwdg_adj_params_default(C.byref(p))
    assert (p.max_steps, p.precision, p.tape_views, p.inflow_edge, p.limiter) == (200, 0, 0, -1, 1)
    assert abs(p.cfl - 0.33) < 1e-15 and abs(p.g - 9.80665) < 1e-15
    assert create(nx=0) == -2
    assert create(dx=0.0) == -2
    assert create(max_steps=0) == -2
    assert create(precision=7) == -1
    assert create(cfl=-1.0) == -1
    assert create(inflow_edge=4) == -1
    assert create(inflow_edge=0, inflow_c0=3, inflow_c1=2) == -1
    assert create(inflow_edge=0, inflow_c0=0, inflow_c1=8) == -1     # beyond the 8 cells of the edge


@pytest.mark.parametrize("field,value,status", [
    ("L", -1, -2), ("M", 0, -2), ("N", -3, -2), ("dx", 0.0, -2), ("dx", float("nan"), -2),
    ("mode", 3, -1), ("mode", -1, -1), ("precision", 2, -1), ("cfl", 0.0, -1), ("cfl", float("nan"), -1),
    ("g", -9.8, -1), ("h_dry", -1e-3, -1), ("dt_max", 0.0, -1), ("eps", -1e-3, -1),
    ("eps", float("inf"), -1), ("eps", float("nan"), -1), ("iface_rule", 2, -1), ("scheme", 3, -1),
])
def test_create_rejects_each_bad_parameter_without_device(field, value, status):
    """mwdg_create answers every invalid parameter with its status before any
    device work (MWDG_ERR_DIMS for sizes, MWDG_ERR_ARG otherwise), and
    leaves the handle NULL."""
    import ctypes as C
    L = binding.lib()
    p = binding.Params()
    assert L.mwdg_params_default(C.byref(p)) == 0
    p.M = p.N = 4
    p.L = 3
    setattr(p, field, value)
    h = C.c_void_p(12345)
    assert L.mwdg_create(C.byref(p), C.byref(h)) == status
    assert not h.value


@pytest.mark.parametrize("combo", ["reflux_adaptive", "acc_adaptive", "too_wide", "too_tall"])
def test_create_rejects_bad_combinations_without_device(combo):
    """the reflux rule and the ACC solver are static-grid options (not on
    adaptive grids), and a finest level wider or taller than 2^20 cells is
    refused"""
    import ctypes as C
    L = binding.lib()
    p = binding.Params()
    L.mwdg_params_default(C.byref(p))
    if combo == "reflux_adaptive":
        p.L, p.mode, p.iface_rule = 3, 2, 1
        want = -1
    elif combo == "acc_adaptive":
        p.L, p.mode, p.scheme = 3, 2, 2
        want = -1
    elif combo == "too_wide":
        p.M, p.L = 3, 19  # 3 * 2^19 > 2^20
        want = -2
    else:
        p.N, p.L = 2049, 10
        want = -2
    h = C.c_void_p(1)
    assert L.mwdg_create(C.byref(p), C.byref(h)) == want
    assert not h.value


def test_frozen_adjoint_grid_is_validated_without_device():
    """mwdg_adj_create_frozen checks the sizes against M, N, L and that the
    leaves tile the domain (no gap, no overlap, none listed twice or out of
    range) before any device work"""
    import ctypes as C
    import numpy as np
    L = adjoint.lib()

    def create(lev, ii, jj, M=1, N=1, Lv=2, mode=1, nx=4, ny=4):
        p = adjoint.AdjParams()
        L.mwdg_adj_params_default(C.byref(p))
        p.nx, p.ny, p.dx = nx, ny, 1.0
        a = [np.ascontiguousarray(x, dtype=np.int32) for x in (lev, ii, jj)]
        h = C.c_void_p(7)
        st = L.mwdg_adj_create_frozen(C.byref(p), M, N, Lv, mode, len(a[0]), *(x.ctypes.data_as(C.c_void_p)
                                                                               for x in a), C.byref(h))
        assert st == 0 or not h.value
        return st

    # one level-1 quadrant refined into four level-2 leaves, three level-1 leaves
    lev = [1, 1, 1, 2, 2, 2, 2]
    ii = [1, 0, 1, 0, 1, 0, 1]
    jj = [0, 1, 1, 0, 0, 1, 1]
    assert create(lev, ii, jj, nx=8) == -2            # nx is not M 2^L
    assert create(lev, ii, jj, mode=0) == -1          # uniform is not a frozen grid's mode
    assert create(lev[:-1], ii[:-1], jj[:-1]) == -1   # a gap
    assert create(lev + [2], ii + [1], jj + [1]) == -1     # listed twice
    assert create(lev + [0], ii + [0], jj + [0]) == -1     # a leaf over other leaves
    assert create(lev[:-1] + [2], ii[:-1] + [4], jj[:-1] + [0]) == -1   # out of range
    assert create([1, 1, 1, 1], [0, 1, 0, 1], [0, 0, 1, 1], Lv=16) == -2
