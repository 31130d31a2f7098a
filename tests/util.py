"""Helpers shared by the tests: build an oracle simulation from a synthetic
problem, analytic dam-break profiles."""
import numpy as np

import oracle as O


def oracle_sim(p, **over):
    kw = dict(M=p.M, N=p.N, L=p.L, R=p.dx, mode=p.mode, eps=p.eps, bc=p.bc,
              inflow_edge=p.inflow_edge, inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1,
              rain_rate=p.rain_rate, rain_t_end=p.rain_t_end, limiter=p.limiter,
              dt_max=p.dt_max, iface_rule=p.iface_rule, scheme=p.scheme, cfl=p.cfl)
    kw.update(over)
    s = O.Sim(**kw)
    s.load_dem(p.z_vert)
    s.load_roughness(p.n_cell())
    s.load_initial(p.h_vert, p.qx_vert, p.qy_vert, p.is_eta)
    if len(p.inflow_t):
        s.set_inflow(p.inflow_t, p.inflow_Q)
    s.init_grid()
    return s


def average_raster(sim):
    """Finest-resolution raster of the active leaves' average depths (each
    finest cell takes the average of the leaf covering it)."""
    lev, ii, jj, co = sim.read_active()
    L = sim.levels
    nx, ny = sim.nx, sim.ny
    out = np.zeros((ny, nx))
    for l in np.unique(lev):
        m = lev == l
        w = 1 << (L - l)
        for a, b, h in zip(ii[m], jj[m], co[m, 0]):
            out[b * w:(b + 1) * w, a * w:(a + 1) * w] = h
    return out


def ritter_depth(x, t, x0, hL, g):
    """Dry-bed dam break (Ritter): depth at positions x and time t > 0."""
    cL = np.sqrt(g * hL)
    xi = (x - x0) / t
    h = np.where(xi <= -cL, hL, (2.0 * cL - xi) ** 2 / (9.0 * g))
    return np.where(xi >= 2.0 * cL, 0.0, h)


def stoker_depth(x, t, x0, hL, hR, g):
    """Wet-bed dam break (Stoker): rarefaction, constant middle state, shock."""
    cL, cR = np.sqrt(g * hL), np.sqrt(g * hR)
    # middle celerity: -8 g hR cm^2 (cL - cm)^2 + (cm^2 - g hR)^2 (cm^2 + g hR) = 0
    f = lambda c: -8.0 * g * hR * c * c * (cL - c) ** 2 + (c * c - g * hR) ** 2 * (c * c + g * hR)
    lo, hi = cR, cL
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.sign(f(mid)) == np.sign(f(lo)):
            lo = mid
        else:
            hi = mid
    cm = 0.5 * (lo + hi)
    hm = cm * cm / g
    S = 2.0 * cm * cm * (cL - cm) / (cm * cm - g * hR)
    xi = (x - x0) / t
    h = np.where(xi <= -cL, hL, (2.0 * cL - xi) ** 2 / (9.0 * g))
    h = np.where(xi >= 2.0 * cL - 3.0 * cm, hm, h)
    return np.where(xi >= S, hR, h)


def oracle_variant(tmp_path, edits):
    """A scratch copy of the oracle with text edits applied (a planted change
    whose effect a test checks), compiled like the oracle and typed by
    ``oracle.load``; every edit must match the source exactly once or more."""
    import subprocess
    from pathlib import Path
    src = (Path(O.__file__).resolve().parent / "mwdg2_oracle.c").read_text()
    for old, new in edits:
        assert old in src, old
        src = src.replace(old, new)
    c = tmp_path / "variant.c"
    c.write_text(src)
    so = tmp_path / "libvariant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-shared", "-fPIC",
                    str(c), "-o", str(so), "-lm"], check=True)
    return O.load(so)
