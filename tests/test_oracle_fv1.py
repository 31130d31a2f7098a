"""Oracle pins for the FV1 solver (Sect. 2.1.2, Eq. 5-7) and the Haar-wavelet
adaptive HWFV1 (Sect. 2.3): Haar transform identities, lake at rest over
rough terrain on uniform, static and adaptive grids, the Ritter and Stoker
dam breaks with an error that falls with dx at first order, volume
conservation and the mass budget, and HWFV1 at epsilon = 0 against uniform
FV1."""
import numpy as np
import pytest

import oracle as O
from paper_2107_02750_gb300 import synth as S
from util import oracle_sim, ritter_depth, stoker_depth

G = 9.80665


def test_haar_transform_identities():
    rng = np.random.default_rng(11)
    for _ in range(20):
        sc = rng.normal(size=4)
        p, d = O.haar_encode(sc)
        # parent = mean, lossless, Parseval of the orthonormal transform
        assert abs(p - sc.mean()) <= 1e-15
        np.testing.assert_allclose(O.haar_decode(p, d), sc, atol=1e-15)
        assert abs(0.25 * np.sum(sc ** 2) - (p * p + 0.25 * np.sum(d ** 2))) <= 1e-14
    # a west-east step gives only the x detail; constants give none
    p, d = O.haar_encode(np.array([0.0, 2.0, 0.0, 2.0]))
    assert p == 1.0 and d[0] == 2.0 and d[1] == 0.0 and d[2] == 0.0
    _, d = O.haar_encode(np.full(4, 3.5))
    assert np.all(d == 0.0)


@pytest.mark.parametrize("mode,islands", [(S.UNIFORM, False), (S.UNIFORM, True), (S.STATIC, True),
                                          (S.ADAPTIVE, True)])
def test_fv1_lake_at_rest(mode, islands):
    kw = dict(n=32, islands=islands)
    if mode != S.UNIFORM:
        kw.update(L=3, mode=mode, eps=1e-2)
    p = S.fv1(S.lake_at_rest(**kw))
    s = oracle_sim(p)
    _, _, _, c0 = s.leaves()
    for _ in range(400):
        s.step()
    lev, _, _, c = s.leaves()
    assert np.abs(c[:, 3:]).max() <= 1e-12
    assert np.abs(c[:, [1, 2]]).max() == 0.0  # piecewise constant
    if mode == S.STATIC:
        assert len(np.unique(lev)) > 1


@pytest.mark.parametrize("kind", ["ritter", "stoker"])
def test_fv1_dam_break_closed_forms(kind):
    hR = 0.0 if kind == "ritter" else 0.1
    errs = []
    for nx, dx in ((100, 1.0), (200, 0.5)):
        p = S.fv1(S.dam_break_strip(nx=nx, ny=4, dx=dx, h_left=1.0, h_right=hR))
        s = oracle_sim(p, dt_max=1.0)
        s.run_to(6.0)
        x = (np.arange(nx) + 0.5) * dx
        h, _, _ = s.fields()
        prof = h.mean(axis=0)
        exact = ritter_depth(x, 6.0, 50.0, 1.0, G) if kind == "ritter" else stoker_depth(x, 6.0, 50.0, 1.0, hR, G)
        errs.append(np.mean(np.abs(prof - exact)))
        assert np.abs(h - h[0:1, :]).max() < 1e-12
    assert errs[1] < 0.8 * errs[0]
    assert errs[1] < (0.01 if kind == "ritter" else 0.008)


def test_fv1_volume_and_mass_budget():
    p = S.fv1(S.dam_break_circular())
    s = oracle_sim(p)
    v0 = s.diag()["volume"]
    s.run_to(5.0)
    d = s.diag()
    assert abs(d["volume"] - v0) <= 1e-12 * v0 and d["n_clip"] == 0
    h, _, _ = s.fields()
    assert np.abs(h - h.T).max() <= 1e-12
    q = S.fv1(S.valley(n=64, L=6, mode=S.UNIFORM, dx=10.0, peak_Q=50.0, t_peak=60.0))
    q.rain_rate, q.rain_t_end = 1e-4, 40.0
    s = oracle_sim(q)
    v0 = s.diag()["volume"]
    s.run_to(120.0)
    d = s.diag()
    assert d["n_clip"] == 0 and d["v_clip"] == 0.0
    budget = v0 + d["v_in"] - d["v_out"] + d["v_rain"]
    assert abs(d["volume"] - budget) <= 1e-12 * max(1.0, d["volume"])
    assert d["v_in"] > 0 and d["v_rain"] > 0


def test_hwfv1_at_zero_epsilon_equals_uniform_fv1():
    pu = S.fv1(S.dam_break_circular(n=64, radius=6.0, L=6, mode=S.UNIFORM))
    pa = S.fv1(S.dam_break_circular(n=64, radius=6.0, L=6, mode=S.ADAPTIVE, eps=0.0))
    su, sa = oracle_sim(pu), oracle_sim(pa)
    for _ in range(20):
        assert abs(su.step() - sa.step()) <= 1e-13
    lu, iu, ju, cu = su.leaves()
    la, ia, ja, ca = sa.leaves()
    np.testing.assert_array_equal(la, lu)
    assert np.abs(ca - cu).max() <= 1e-12


def test_hwfv1_adapts_with_haar_details():
    """At epsilon > 0 the HWFV1 grid coarsens where the piecewise-constant
    data are flat and keeps the finest level where they jump."""
    p = S.fv1(S.dam_break_circular(n=64, radius=6.0, L=6, mode=S.ADAPTIVE, eps=1e-3))
    s = oracle_sim(p)
    s.step()
    lev, ii, jj, c = s.leaves()
    assert 64 * 64 > len(lev) > 100 and lev.min() < 6 and lev.max() == 6
    assert np.abs(c[:, [1, 2, 4, 5, 7, 8]]).max() == 0.0
