"""Anytime planning in the server (§III-C: the latest valid solution is kept while
the optimiser keeps improving it): best-so-far results published and readable
with peek, improvement rounds equal to the same refinement run in one plan,
cancellation that keeps the best, and ordinary requests served meanwhile.
Every failure here is made on the host."""
import time

import numpy as np
import pytest

import problems
from gpu_util import params_pair, run_plan
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plain():
    return problems.build(synth.PLAIN)


@pytest.mark.parametrize("pinned", [None, 0])
def test_rounds_equal_the_same_refinement_in_one_plan(plain, pinned):
    """R improvement rounds after the first pass run the kernels of a plan with
    smooth_rounds = R; when every round is published the result is bit-identical.
    With the default pinned pool each round's results pass through the launch's pinned
    staging; with none (pinned = 0) through pageable memory; either way they end in
    the request's own buffer."""
    pb = plain
    R = 3
    _, cp = params_pair(lm_iters=pb.w.lm_iters)
    _, cpR = params_pair(lm_iters=pb.w.lm_iters, smooth_rounds=R)
    rob = cppflow.robot_from_arm(pb.arm)
    first = run_plan(rob, cp, pb.cand, pb.targets, pb.K)
    ref = run_plan(rob, cpR, pb.cand, pb.targets, pb.K)
    with cppflow.Server(cp, hbm_budget=1 << 30, pinned_bytes=pinned) as srv:
        t = srv.submit(rob, pb.cand, pb.targets, pb.K, anytime_rounds=R)
        st, res = srv.wait(t)
        stats = srv.stats()
    assert st == cppflow.OK and res["report"]["valid"] == 1
    assert stats["improve_rounds"] == R and stats["improve_batches"] == R
    assert stats["published"] >= 1
    assert res["report"]["traj_len"] <= first["report"]["traj_len"]
    if res["rounds"] == R:          # the last round was the best: the plan's own result
        np.testing.assert_array_equal(res["q"], ref["q"])
        np.testing.assert_array_equal(res["err"], ref["err"])
    np.testing.assert_array_equal(res["sel"], first["sel"])


def test_peek_then_cancel_keeps_the_best(plain):
    pb = plain
    _, cp = params_pair(lm_iters=pb.w.lm_iters)
    rob = cppflow.robot_from_arm(pb.arm)
    with cppflow.Server(cp, hbm_budget=1 << 30) as srv:
        t = srv.submit(rob, pb.cand, pb.targets, pb.K, anytime_rounds=100000)
        seen = None
        for _ in range(20000):
            st, res = srv.peek(t)
            if st == cppflow.OK:
                seen = res
                break
            assert st == cppflow.PENDING
            time.sleep(0.0005)
        assert seen is not None and seen["report"]["valid"] == 1
        time.sleep(0.05)                      # let it improve a little
        st2, later = srv.peek(t)
        assert st2 == cppflow.OK
        assert later["report"]["traj_len"] <= seen["report"]["traj_len"]
        assert srv.cancel(t) == cppflow.OK
        st3, final = srv.wait(t)
        stats = srv.stats()
    assert st3 == cppflow.OK and final["report"]["valid"] == 1
    assert final["report"]["traj_len"] <= later["report"]["traj_len"]
    assert 0 < stats["improve_rounds"] < 100000


def test_ordinary_requests_are_served_while_others_improve(plain):
    pb = plain
    _, cp = params_pair(lm_iters=pb.w.lm_iters)
    rob = cppflow.robot_from_arm(pb.arm)
    other = problems.small(T=20, K=40, seed=3)
    orob = cppflow.robot_from_arm(other.arm)
    with cppflow.Server(cp, hbm_budget=1 << 30, max_inflight=2) as srv:
        ta = srv.submit(rob, pb.cand, pb.targets, pb.K, anytime_rounds=100000)
        tb = srv.submit(orob, other.cand, other.targets, other.K)
        st, res = srv.wait(tb, timeout_us=20_000_000)
        assert st == cppflow.OK
        alone = run_plan(orob, cp, other.cand, other.targets, other.K)
        np.testing.assert_array_equal(res["q"], alone["q"])
        assert srv.poll(ta)[0] == cppflow.PENDING       # still improving
        assert srv.cancel(ta) == cppflow.OK
        assert srv.wait(ta)[0] == cppflow.OK


def test_invalid_anytime_budget_is_refused(plain):
    pb = plain
    _, cp = params_pair()
    with cppflow.Server(cp, hbm_budget=1 << 30) as srv:
        with pytest.raises(cppflow.CppflowError):
            srv.submit(cppflow.robot_from_arm(pb.arm), pb.cand, pb.targets, pb.K,
                       anytime_rounds=-1)
