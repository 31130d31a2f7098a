"""Oracle pins for the ACC (local inertial) solver (Sect. 2.1.3): lake at rest
over rough terrain with islands on uniform and static graded grids (no
interface discharge at all), volume conservation and the mass budget with
inflow and rain (also across coarse/fine faces, whose half-face discharges
are aggregated), and the Manning normal depth of a steady uniform channel
flow, which the semi-implicit resistance term reaches exactly."""
import numpy as np
import pytest

from paper_2107_02750_gb300 import synth as S
from util import oracle_sim


@pytest.mark.parametrize("mode", [S.UNIFORM, S.STATIC])
def test_acc_lake_at_rest(mode):
    kw = dict(n=32, islands=True)
    if mode == S.STATIC:
        kw.update(L=3, mode=mode, eps=1e-2)
    p = S.acc(S.lake_at_rest(**kw))
    s = oracle_sim(p)
    _, _, _, c0 = s.leaves()
    for _ in range(300):
        s.step()
    lev, _, _, c = s.leaves()
    assert np.abs(c[:, 3:]).max() == 0.0
    np.testing.assert_array_equal(c[:, 0], c0[:, 0])
    if mode == S.STATIC:
        assert len(np.unique(lev)) > 1


def test_acc_volume_and_budget():
    # a gentle (subcritical) circular release: ACC's domain, no clipping
    p = S.acc(S.dam_break_circular(h_in=0.6, h_out=0.5))
    s = oracle_sim(p)
    v0 = s.diag()["volume"]
    s.run_to(5.0)
    d = s.diag()
    assert abs(d["volume"] - v0) <= 1e-12 * v0 and s.steps > 10 and d["n_clip"] == 0
    h, _, _ = s.fields()
    assert np.abs(h - h.T).max() <= 1e-12 and np.abs(h - h[::-1, :]).max() <= 1e-12
    for mode in (S.UNIFORM, S.STATIC):
        q = S.acc(S.valley(n=64, L=6, mode=mode, eps=1e-2, dx=10.0, peak_Q=50.0, t_peak=60.0))
        q.rain_rate, q.rain_t_end = 1e-4, 40.0
        s = oracle_sim(q)
        if mode == S.STATIC:
            assert len(np.unique(s.leaves()[0])) > 1
        v0 = s.diag()["volume"]
        s.run_to(150.0)
        d = s.diag()
        budget = v0 + d["v_in"] - d["v_out"] + d["v_rain"] + d["v_clip"]
        assert abs(d["volume"] - budget) <= 1e-12 * max(1.0, d["volume"]), mode
        assert d["v_in"] > 0 and d["v_rain"] > 0


def test_acc_manning_normal_depth():
    """Steady uniform flow down a constant slope: q = h^(5/3) S^(1/2) / n, so
    the depth away from the ends tends to h_n = (q n / S^(1/2))^(3/5)."""
    q_in, S_, n_m = 2.0, 1e-3, 0.03
    # 4 km of subcritical channel: the reach away from the inlet and from the
    # drawdown to the free outlet (length scale h_n / S ~ 1.5 km) is uniform
    p = S.acc(S.sloped_channel(nx=400, ny=4, dx=10.0, slope=S_, q_in=q_in, n_manning=n_m))
    s = oracle_sim(p, dt_max=5.0)
    s.run_to(4 * 3600.0)
    h, u, _ = s.fields()
    hn = (q_in * n_m / np.sqrt(S_)) ** 0.6
    reach = slice(20, 150)
    assert np.abs(h[:, reach] / hn - 1.0).max() < 0.01, (h[:, reach].min(), h[:, reach].max(), hn)
    assert np.abs(h[:, reach] * u[:, reach] / q_in - 1.0).max() < 1e-6  # steady: q = q_in
