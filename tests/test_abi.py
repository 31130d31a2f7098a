"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/*.h declares (no compute calls: no GPU needed)."""
import re
from pathlib import Path

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
