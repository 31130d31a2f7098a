"""mwdg_volume_noalloc: the allocation-free volume sum.

Some callers cannot allocate device memory while they run (a host that gives
all device memory to its own pool at start-up, a real-time flood-warning loop
that must not risk an allocation failure mid-run, a plug-in that only
receives buffers).  mwdg_volume_noalloc serves them: it takes the caller's
device arrays and writes the volume to the caller's device pointer, keeping
its partial sums in a fixed device array of the library.  This test calls it
through the C ABI twice in a row and checks each result against
mwdg_get_volume on the same state.  It runs last (file name) and also passes
alone in a fresh process, where its first call performs the per-device
set-up."""
import ctypes as C

import numpy as np
import pytest

from paper_2107_02750_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-12   # relative, as the FP64 volume checks of the parity tests


def _call(lib, h0, lev, n, dx, L, out, stream):
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    return lib.mwdg_volume_noalloc(ptr(h0), ptr(lev), n, dx, L, ptr(out), C.c_void_p(stream))


def test_noalloc_volume_matches_get_volume():
    import torch
    import paper_2107_02750_gb300 as M
    lib = M.lib()
    p = S.valley(n=128, L=7, mode=S.ADAPTIVE, eps=1e-2, peak_Q=200.0, t_peak=100.0)
    s = M.solver_from_problem(p, precision=M.F64)
    s.run_to_time(80.0)
    ref = s.get_volume()["volume"]
    lev, _, _, co = s.read_active()
    assert len(np.unique(lev)) > 1 and ref > 0.0
    dev = torch.device("cuda", torch.cuda.current_device())
    h0 = torch.tensor(co[:, 0], dtype=torch.float64, device=dev)
    lv = torch.tensor(lev, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):   # two calls in a row share the scratch array
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        st = _call(lib, h0, lv, len(lev), p.dx, p.L, out, stream)
        assert st == 0, lib.mwdg_status_string(st)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= TOL * ref, (got, ref)


def test_noalloc_volume_limits():
    import torch
    import paper_2107_02750_gb300 as M
    lib = M.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    # no leaves: zero volume
    assert _call(lib, None, None, 0, 1.0, 0, out, stream) == 0
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
    # beyond the stated maximum: rejected before any device work
    dummy = torch.zeros(1, dtype=torch.float64, device=dev)
    lv = torch.zeros(1, dtype=torch.int32, device=dev)
    assert _call(lib, dummy, lv, 67108864 + 1, 1.0, 0, out, stream) == -7
    assert _call(lib, dummy, lv, 1, 0.0, 0, out, stream) == -1
    # a level outside 0..L is refused (not clamped): the volume reads NaN
    for bad in (3, -1):
        lvb = torch.tensor([0, bad], dtype=torch.int32, device=dev)
        h2 = torch.ones(2, dtype=torch.float64, device=dev)
        assert _call(lib, h2, lvb, 2, 1.0, 2, out, stream) == -1
        torch.cuda.synchronize()
        assert np.isnan(float(out.item()))
    # and a valid call after it succeeds again
    lvg = torch.tensor([0, 2], dtype=torch.int32, device=dev)
    assert _call(lib, h2, lvg, 2, 1.0, 2, out, stream) == 0
    torch.cuda.synchronize()
    assert float(out.item()) == 16.0 + 1.0
