"""The raster entry points of the C ABI: host rasters with a row stride,
device rasters (torch tensors, rows possibly strided) for the DEM, the
roughness and the initial state, and strided read-back to host and device
(include/mwdg.h).  A problem loaded either way steps to the same state bit
for bit; non-finite device values and short row strides are refused."""
import ctypes as C

import numpy as np
import pytest

from paper_2107_02750_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _padded(a, pad=7):
    """a CUDA float64 view of a whose rows lie pad elements apart beyond their length"""
    import torch
    t = torch.full((a.shape[0], a.shape[1] + pad), float("nan"), dtype=torch.float64, device="cuda")
    t[:, :a.shape[1]] = torch.as_tensor(np.array(a, dtype=np.float64))
    return t[:, :a.shape[1]]


def _device_loaded(p, precision):
    import paper_2107_02750_gb300 as M
    s = M.Solver(M=p.M, N=p.N, L=p.L, dx=p.dx, mode=p.mode, precision=precision, eps=p.eps, limiter=p.limiter,
                 bc=p.bc, dt_max=p.dt_max, iface_rule=p.iface_rule, scheme=p.scheme, cfl=p.cfl)
    s.load_dem_dev(_padded(p.z_vert))
    s.load_roughness_dev(_padded(p.n_cell(), pad=3))
    s.set_inflow(p.inflow_edge, p.inflow_c0, p.inflow_c1, p.inflow_t, p.inflow_Q)
    pad = 5
    s.load_initial_dev(_padded(p.h_vert, pad), _padded(p.qx_vert, pad), _padded(p.qy_vert, pad), p.is_eta)
    return s


@pytest.mark.parametrize("precision", [0, 1])
def test_device_rasters_step_like_host_rasters(precision):
    import paper_2107_02750_gb300 as M
    p = S.valley(n=128, L=7, mode=S.ADAPTIVE, eps=1e-2, peak_Q=200.0, t_peak=60.0)
    p.n_manning = 0.03 + 0.01 * S.fractal_surface(p.nx, 3, 3.0)[:p.ny, :p.nx] ** 2
    ref = M.solver_from_problem(p, precision=precision)
    dev = _device_loaded(p, precision)
    for _ in range(30):
        assert ref.dg2_step() == dev.dg2_step()
    la, ia, ja, ca = ref.read_active()
    lb, ib, jb, cb = dev.read_active()
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(ca, cb)


def test_strided_read_back_host_and_device():
    import torch
    import paper_2107_02750_gb300 as M
    p = S.valley(n=128, L=7, mode=S.ADAPTIVE, eps=1e-2, peak_Q=200.0, t_peak=60.0)
    s = M.solver_from_problem(p)
    s.run_steps(40)
    h, u, v = s.read_fields()
    ld = p.nx + 9
    buf = np.full((3, p.ny, ld), np.nan)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    assert s._lib.mwdg_read_fields(s._h, dp(buf[0]), dp(buf[1]), dp(buf[2]), ld) == 0
    for q, ref in enumerate((h, u, v)):
        np.testing.assert_array_equal(buf[q, :, :p.nx], ref)
    assert np.isnan(buf[:, :, p.nx:]).all()   # the padding is not written
    t = torch.full((3, p.ny, ld), float("nan"), dtype=torch.float64, device="cuda")
    s.read_fields_dev(t[0, :, :p.nx], t[1, :, :p.nx], t[2, :, :p.nx])
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    for q, ref in enumerate((h, u, v)):
        np.testing.assert_array_equal(got[q, :, :p.nx], ref)
    assert np.isnan(got[:, :, p.nx:]).all()
    # a row stride below the row length is refused
    assert s._lib.mwdg_read_fields(s._h, dp(buf[0]), None, None, p.nx - 1) == -1


def test_device_rasters_are_checked():
    import torch
    import paper_2107_02750_gb300 as M
    p = S.valley(n=64, L=6, mode=S.UNIFORM, peak_Q=50.0, t_peak=60.0)
    s = M.Solver(M=p.M, N=p.N, L=p.L, dx=p.dx, mode=p.mode)
    z = _padded(p.z_vert)
    z[3, 4] = float("inf")
    with pytest.raises(M.MwdgError) as e:
        s.load_dem_dev(z)
    assert e.value.status == -4
    # a refused input leaves the context in its error state (MWDG_ERR_STATE after)
    with pytest.raises(M.MwdgError) as e:
        s.load_dem_dev(_padded(p.z_vert))
    assert e.value.status == -6
    s = M.Solver(M=p.M, N=p.N, L=p.L, dx=p.dx, mode=p.mode)
    s.load_dem_dev(_padded(p.z_vert))
    h = _padded(p.h_vert)
    q = _padded(p.qx_vert)
    q[1, 1] = float("nan")
    with pytest.raises(M.MwdgError) as e:
        s.load_initial_dev(h, q, _padded(p.qy_vert), False)
    assert e.value.status == -4
    # host rasters with a row stride below the row length are refused
    s = M.Solver(M=p.M, N=p.N, L=p.L, dx=p.dx, mode=p.mode)
    zz = np.ascontiguousarray(p.z_vert)
    assert s._lib.mwdg_load_dem(s._h, zz.ctypes.data_as(C.POINTER(C.c_double)), p.nx) == -1
