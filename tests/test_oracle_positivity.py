"""Pins of the oracle's wet/dry treatment: depths stay non-negative (Sect.
2.1.1: the revisions keep depths non-negative at wet/dry fronts) through the
outflow limit of the interface fluxes, and the mass budget closes without
any clipped volume.

What fixes the limit other than itself:
  * a mound drained by one stage of any length stays non-negative with its
    volume conserved; at rest its centre ends at exactly zero depth (the
    shares of its content add up to one) and its four neighbours receive
    equal volumes, and with an eastward velocity the east one receives more
    than the west one;
  * the rapid-flow valley (a 256 x 256 window through the inflow, 10 min) and
    a dam break over a steep dry slope keep every depth non-negative with the
    mass budget closed to round-off, uniform and adaptive;
  * the same runs of a scratch copy of the oracle with the limit removed
    clip depths (several per cent of the inflowed volume on the valley; on
    the slope the time step collapses), so the pins see the limit;
  * where the limit is not reached it changes nothing: the closed-form dam
    breaks, lake at rest, Manning normal depth and volume pins of the other
    oracle tests hold unchanged."""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2107_02750_gb300 import synth as S
from util import oracle_sim, oracle_variant

NO_LIMIT = [("drain_limit(F, don, g, hd, s->dx[l], dt);", ";")]


def _mound(u=0.0, library=None):
    """5 x 5 cells of 1 m: a centre cell 1 m deep on a flat bed at 0, its
    four neighbours 0.4 m deep and the diagonal ones 0.1 m on beds rising to
    0.5 m, the rest dry; the centre's discharge vertices carry u m^2/s along
    +x."""
    n = 5
    z = np.full((n + 1, n + 1), 0.5)
    z[2:4, 2:4] = 0.0
    eta = np.full((n + 1, n + 1), 0.3)
    eta[2:4, 2:4] = 1.0
    qx = np.zeros((n + 1, n + 1))
    qx[2:4, 2:4] = u
    s = O.Sim(M=n, N=n, L=0, R=1.0, mode=S.UNIFORM, limiter=1, library=library)
    s.load_dem(z)
    s.load_initial(eta, qx, None, True)
    s.init_grid()
    return s


def _depths(s):
    _, _, _, c = s.leaves()
    return c[:, 0].reshape(5, 5)


@pytest.mark.parametrize("u", [0.0, 1.0])
def test_mound_drained_by_one_long_stage(u):
    s = _mound(u)
    h0 = _depths(s)
    s.stage(1.0e3)  # far beyond any Courant number: every interface of the centre is limited
    h = _depths(s)
    if u == 0.0:
        assert h[2, 2] == pytest.approx(0.0, abs=1e-15)
    assert (h >= 0.0).all() and s.diag()["n_clip"] == 0
    assert abs(h.sum() - h0.sum()) <= 1e-14 * h0.sum()
    east, west, north, south = h[2, 3] - h0[2, 3], h[2, 1] - h0[2, 1], h[3, 2] - h0[3, 2], h[1, 2] - h0[1, 2]
    if u == 0.0:
        assert east == pytest.approx(west, abs=1e-15)
        assert east == pytest.approx(north, abs=1e-15) and east == pytest.approx(south, abs=1e-15)
    else:
        assert east > west and north == pytest.approx(south, abs=1e-15)


def test_mound_without_the_limit_goes_negative(tmp_path):
    s = _mound(0.0, library=oracle_variant(tmp_path, NO_LIMIT))
    s.stage(1.0e3)
    assert s.diag()["n_clip"] >= 1


def _valley_window(mode):
    full = S.valley(n=1024)
    L = 8 if mode == S.ADAPTIVE else 0
    return replace(S.crop(full, 0, 1024 // 2 - 128, 256, 256, L=L), mode=mode)


@pytest.mark.parametrize("mode", [S.UNIFORM, S.ADAPTIVE])
def test_valley_window_through_the_inflow(mode):
    """The rapid-flow valley's window through the inflow for 10 min, uniform
    and MWDG2: no depth is clipped, and the budget closes with no clipped
    volume in it."""
    p = _valley_window(mode)
    s = oracle_sim(p)
    v0 = s.diag()["volume"]
    s.run_to(600.0)
    d = s.diag()
    assert d["n_clip"] == 0 and d["v_clip"] == 0.0
    budget = v0 + d["v_in"] - d["v_out"] + d["v_rain"]
    assert abs(d["volume"] - budget) <= 1e-12 * d["volume"]
    assert d["v_in"] > 4.0e4


def test_valley_window_without_the_limit_clips(tmp_path):
    p = _valley_window(S.UNIFORM)
    s = oracle_sim(p, library=oracle_variant(tmp_path, NO_LIMIT))
    s.run_to(120.0)
    d = s.diag()
    assert d["v_clip"] > 0.02 * d["v_in"]


def _steep_slope():
    """Dam break over a steep dry slope: 48 x 48 cells of 2 m, the bed falling
    30 % to the east and rising 15 % to the north, with 0.5 m of seeded
    fractal roughness; a reservoir of 2 m over the highest point behind
    x = 19.2 m; Manning n = 0.02, open east edge, walls elsewhere."""
    n, dx, slope = 48, 2.0, 0.3
    x = np.arange(n + 1) * dx
    X, Y = np.meshgrid(x, x)
    z = slope * (n * dx - X) + 0.5 * slope * Y + 0.5 * S.fractal_surface(n + 1, 7, 4.0)
    eta = np.where(X <= 0.2 * n * dx, z.max() + 2.0 - 0.3 * slope * X, z)
    zeros = np.zeros_like(z)
    return S.Problem("steep_slope", n, n, 0, dx, z, eta, zeros, zeros.copy(), is_eta=True, n_manning=0.02,
                     bc=(S.WALL, S.OPEN, S.WALL, S.WALL), mode=S.UNIFORM)


def test_steep_dry_slope_dam_break():
    p = _steep_slope()
    s = oracle_sim(p)
    v0 = s.diag()["volume"]
    s.run_to(30.0, max_steps=5000)
    d = s.diag()
    assert s.t == 30.0 and s.last_dt > 1e-3
    assert d["n_clip"] == 0 and d["v_clip"] == 0.0
    assert abs(d["volume"] - (v0 - d["v_out"])) <= 1e-12 * v0
    assert d["v_out"] > 0.0


def test_steep_dry_slope_without_the_limit_fails(tmp_path):
    s = oracle_sim(_steep_slope(), library=oracle_variant(tmp_path, NO_LIMIT))
    s.run_to(30.0, max_steps=3000)
    d = s.diag()
    assert d["n_clip"] > 0 or s.t < 30.0
