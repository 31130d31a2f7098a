"""Ensembles (batched scenarios of uneven sizes, one CUDA graph per ensemble
step): every member ends exactly where it ends when stepped alone, through
step counts, run_to_time, interleaved member calls and the launch-shape
autotuner, with the adaptive members in batched launches over a (member,
block) work list or as one graph branch each."""
import numpy as np
import pytest

from paper_2107_02750_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _members(precisions, eps=1e-2, sides=(64, 96, 128, 192), count=4, seed=4):
    import paper_2107_02750_gb300 as M
    probs = S.ensemble(count=count, seed=seed, sides=sides, eps=eps)
    return probs, [M.solver_from_problem(p, precision=precisions[k % len(precisions)])
                   for k, p in enumerate(probs)]


def _same(a, b, what):
    la, ia, ja, ca = a.read_active()
    lb, ib, jb, cb = b.read_active()
    assert len(la) == len(lb), what
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(ja, jb)
    np.testing.assert_array_equal(ca, cb, err_msg=what)
    assert a.get_time() == b.get_time(), what


def test_ensemble_run_to_time_equals_members_alone():
    """Uneven sizes (64..192 cells a side, M in {1, 3}), both precisions,
    adaptive grids: run to 40 s as one ensemble and one by one."""
    import paper_2107_02750_gb300 as M
    probs, ens_members = _members([M.F32, M.F64])
    _, alone = _members([M.F32, M.F64])
    e = M.Ensemble(ens_members)
    launches = e.run_to_time(40.0)
    assert launches > 0
    for k, s in enumerate(alone):
        s.run_to_time(40.0)
        _same(ens_members[k], s, f"member {k}")
        assert abs(ens_members[k].get_time()[0] - 40.0) < 1e-12
    # a second leg continues from there
    e.run_to_time(55.0)
    for k, s in enumerate(alone):
        s.run_to_time(55.0)
        _same(ens_members[k], s, f"member {k}, second leg")


def test_ensemble_steps_interleaved_with_member_calls():
    import paper_2107_02750_gb300 as M
    probs, ens_members = _members([M.F64], count=3)
    _, alone = _members([M.F64], count=3)
    e = M.Ensemble(ens_members)
    e.step(5)
    ens_members[1].run_steps(3)  # a member's own call between ensemble calls
    e.step(2)
    for k, s in enumerate(alone):
        s.run_steps(5 + (3 if k == 1 else 0) + 2)
        _same(ens_members[k], s, f"member {k}")
    # a parameter change on a member rebuilds the ensemble graph
    ens_members[0].set_rain(1e-4, 1e9)
    alone[0].set_rain(1e-4, 1e9)
    e.step(4)
    for k, s in enumerate(alone):
        s.run_steps(4)
        _same(ens_members[k], s, f"member {k} after set_rain")


def test_autotuner_keeps_results_and_state():
    """The tuner times candidate launch shapes from a saved state, restores
    it, and keeps the fastest; FP64 results are unchanged by the shape."""
    import paper_2107_02750_gb300 as M
    probs, ens_members = _members([M.F64], count=3)
    _, alone = _members([M.F64], count=3)
    for s in ens_members + alone:
        s.run_steps(3)
    e = M.Ensemble(ens_members)
    chosen = e.tune(steps=3)
    assert chosen.shape == (3, 2)
    for k, s in enumerate(ens_members):
        assert tuple(chosen[k]) == s.launch_shape()
        assert 1 <= chosen[k, 0] <= 1216  # 152 x {1, 2, 4, 8}, capped by the member's size
        assert chosen[k, 1] in (64, 256, 1024)
        _same(s, alone[k], f"member {k} state after tuning")
    e.run_to_time(30.0)
    for k, s in enumerate(alone):
        s.run_to_time(30.0)
        _same(ens_members[k], s, f"member {k} after tuned run")


def test_ensemble_rejects_bad_members():
    import paper_2107_02750_gb300 as M
    _, ms = _members([M.F64], count=2)
    with pytest.raises(M.MwdgError):
        M.Ensemble([ms[0], ms[0]])
    fresh = M.Solver(M=1, N=1, L=4, dx=1.0, mode=M.ADAPTIVE)  # no initial state
    with pytest.raises(M.MwdgError):
        M.Ensemble([ms[1], fresh])


def test_ensemble_members_match_the_oracle():
    """Every FP64 member of an ensemble of uneven sizes (64..192 cells a side,
    M in {1, 3}, per-member Manning n and inflow scale, MWDG2 at eps = 1e-2)
    against the FP64 oracle stepping the same problem: after 40 ensemble
    steps, identical active sets and coefficients within 1e-9, and each
    member's time equal to the oracle's after its own 40 CFL steps."""
    import paper_2107_02750_gb300 as M
    from util import oracle_sim
    probs, members = _members([M.F64])
    e = M.Ensemble(members)
    e.step(40)
    for k, p in enumerate(probs):
        o = oracle_sim(p)
        for _ in range(40):
            o.step()
        lg, ig, jg, cg = members[k].read_active()
        lo, io, jo, co = o.leaves()
        assert len(lg) == len(lo), f"member {k}"
        np.testing.assert_array_equal(lg, lo)
        np.testing.assert_array_equal(ig, io)
        np.testing.assert_array_equal(jg, jo)
        assert np.abs(cg - co).max() <= 1e-9, f"member {k}"
        t, steps = members[k].get_time()
        assert steps == 40 and abs(t - o.t) <= 1e-9 * o.t


@pytest.mark.parametrize("batch", [0, 2, 64])
def test_batched_and_branch_ensembles_equal_members_alone(batch):
    """A mixed ensemble: three FP32 and two FP64 MWDG2 members of uneven sizes
    (in batched groups of up to `batch` members of one precision), a
    static-grid and a uniform-grid member (graph branches either way); 25
    ensemble steps, then run_to_time, every member bit for bit as when
    stepped alone."""
    import paper_2107_02750_gb300 as M
    from dataclasses import replace

    def build():
        probs = S.ensemble(count=5, seed=6, sides=(64, 96, 128, 192), eps=1e-2)
        extra = [replace(S.ensemble(count=1, seed=8, sides=(64,), eps=1e-2)[0], mode=S.STATIC),
                 replace(S.ensemble(count=1, seed=9, sides=(64,), eps=1e-2)[0], mode=S.UNIFORM)]
        precs = [M.F32, M.F64, M.F32, M.F64, M.F32, M.F64, M.F32]
        return [M.solver_from_problem(q, precision=precs[k]) for k, q in enumerate(probs + extra)]

    members, alone = build(), build()
    e = M.Ensemble(members, batch=batch)
    e.step(25)
    for k, s in enumerate(alone):
        s.run_steps(25)
        _same(members[k], s, f"member {k}")
    e.run_to_time(35.0)
    for k, s in enumerate(alone):
        s.run_to_time(35.0)
        _same(members[k], s, f"member {k} after run_to_time")
    # switching mid-run keeps the results
    e.set_batch(0 if batch else 3)
    e.step(5)
    for k, s in enumerate(alone):
        s.run_steps(5)
        _same(members[k], s, f"member {k} after switching")
