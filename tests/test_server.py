"""The serving loop (cpp_server_*): every plan is the same alone and in the mix;
admission by HBM budget; rejection of a request larger than the budget;
cancellation of queued requests; host-side validation. Failures are made on the
host (bad inputs, tiny budgets, cancelled tickets) -- nothing here faults a GPU."""
import math

import numpy as np
import pytest

import problems
from gpu_util import params_pair, run_plan
from paper_2309_09102_gb300 import cppflow

pytestmark = pytest.mark.gpu


def _mix(count, seed0=700):
    shapes = [(30, 40), (61, 128), (12, 7), (45, 256), (2, 3), (80, 96), (17, 33), (50, 512)]
    return [problems.small(T=shapes[i % len(shapes)][0], K=shapes[i % len(shapes)][1],
                           seed=seed0 + i) for i in range(count)]


def test_served_equals_alone():
    """Requests submitted together (batched, overlapping launches) return exactly what each
    returns from cpp_plan alone."""
    pbs = _mix(12)
    _, cp = params_pair(lm_iters=10)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    with cppflow.Server(cp, hbm_budget=1 << 30, max_inflight=2, max_batch=5) as srv:
        tickets = [srv.submit(robots[i], pb.cand, pb.targets, pb.K) for i, pb in enumerate(pbs)]
        results = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    assert stats["completed"] == len(pbs) and stats["batches"] >= 3
    for i, pb in enumerate(pbs):
        st, res = results[i]
        assert st == cppflow.OK
        alone = run_plan(robots[i], cp, pb.cand, pb.targets, pb.K)
        np.testing.assert_array_equal(res["sel"], alone["sel"])
        np.testing.assert_array_equal(res["q"], alone["q"])
        np.testing.assert_array_equal(res["err"], alone["err"])
        assert res["best"] == float(alone["best"])
        assert res["report"]["valid"] == alone["report"]["valid"]
        assert res["latency_ms"] > 0


def test_batches_staged_ahead_equal_alone():
    """One compute stream and batches of 2 from 6 same-class requests queued at once: while
    a batch runs, the next is formed and its inputs copied ahead; every result (report
    included) equals cpp_plan alone."""
    pbs = [problems.small(T=40, K=64, seed=760 + i) for i in range(6)]
    _, cp = params_pair(lm_iters=10)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    with cppflow.Server(cp, hbm_budget=1 << 30, max_inflight=1, max_batch=2) as srv:
        tickets = [srv.submit(robots[i], pb.cand, pb.targets, pb.K) for i, pb in enumerate(pbs)]
        results = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    # the first batch may leave before the others are submitted
    assert stats["completed"] == 6 and stats["batches"] >= 3 and stats["max_batch_seen"] == 2
    for i, pb in enumerate(pbs):
        st, res = results[i]
        assert st == cppflow.OK
        alone = run_plan(robots[i], cp, pb.cand, pb.targets, pb.K)
        np.testing.assert_array_equal(res["sel"], alone["sel"])
        np.testing.assert_array_equal(res["q"], alone["q"])
        assert res["report"] == alone["report"]


def test_borrowed_inputs_and_tiny_budget():
    """A budget that holds about one request at a time: every request still completes,
    admitted as memory frees up; a request larger than the whole budget is refused."""
    pbs = _mix(6, seed0=900)
    _, cp = params_pair(lm_iters=5)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    big = max(pb.cand.nbytes for pb in pbs)
    budget = 3 * big + (1 << 20)
    with cppflow.Server(cp, hbm_budget=budget, max_inflight=2) as srv:
        tickets = [srv.submit(robots[i], pb.cand, pb.targets, pb.K, borrow=True)
                   for i, pb in enumerate(pbs)]
        for t in tickets:
            st, res = srv.wait(t)
            assert st == cppflow.OK
        s = srv.stats()
        assert s["hbm_high_water"] <= budget
        huge = problems.small(T=200, K=512, seed=5)
        with pytest.raises(cppflow.CppflowError) as e:
            srv.submit(cppflow.robot_from_arm(huge.arm), huge.cand, huge.targets, huge.K)
        assert e.value.status == cppflow.ERR_BUDGET


def test_cancel_and_validation():
    pbs = _mix(40, seed0=1100)
    _, cp = params_pair(lm_iters=5)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    with cppflow.Server(cp, hbm_budget=1 << 30, max_inflight=1, max_batch=2) as srv:
        tickets = [srv.submit(robots[i], pb.cand, pb.targets, pb.K) for i, pb in enumerate(pbs)]
        cancelled = [t for t in tickets[20:] if srv.cancel(t) == cppflow.OK]
        for t in tickets:
            st, res = srv.wait(t)
            assert st == (cppflow.ERR_CANCELLED if t in cancelled else cppflow.OK)
        with pytest.raises(cppflow.CppflowError) as e:
            srv.poll(tickets[0])  # already collected
        assert e.value.status == cppflow.ERR_NOT_FOUND
        bad = pbs[0].targets.copy()
        bad[3, 4] = math.nan
        with pytest.raises(cppflow.CppflowError) as e:
            srv.submit(robots[0], pbs[0].cand, bad, pbs[0].K)
        assert e.value.status == cppflow.ERR_INVALID_ARG
        bad = pbs[0].targets.copy()
        bad[1, 3:] *= 1.01
        with pytest.raises(cppflow.CppflowError) as e:
            srv.submit(robots[0], pbs[0].cand, bad, pbs[0].K)
        assert e.value.status == cppflow.ERR_INVALID_ARG
        s = srv.stats()
    assert s["cancelled"] == len(cancelled)
    assert s["completed"] == len(pbs) - len(cancelled)


@pytest.mark.parametrize("budget", [0.0, 0.05, 0.5, 1000.0])
def test_throughput_form_mixed_k_equals_alone(budget):
    """Under load (latency_requests = 0: every launch in the throughput form) requests of
    different K share a launch; the search runs once per K bucket and form on forked
    streams, each request in the most efficient form within the time budget: one CTA,
    wide clusters of 512 or 256 successors per CTA, clusters of 128, else of 64 (a
    group's largest Kp sets the cluster, so a smaller request's last CTAs may own
    nothing). The budgets here move these small requests across all five forms. Every
    plan equals cpp_plan alone."""
    shapes = [(30, 1000), (45, 300), (20, 128), (61, 600), (12, 1024), (33, 260), (40, 90),
              (25, 544), (1, 700), (2, 513)]
    pbs = [problems.small(T=T, K=K, seed=800 + i) for i, (T, K) in enumerate(shapes)]
    _, cp = params_pair(lm_iters=10)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    with cppflow.Server(cp, hbm_budget=1 << 30, max_inflight=4, max_batch=64, latency_requests=0,
                        search_budget_ms=budget) as srv:
        tickets = [srv.submit(robots[i], pb.cand, pb.targets, pb.K) for i, pb in enumerate(pbs)]
        results = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    assert stats["completed"] == len(pbs)
    for i, pb in enumerate(pbs):
        st, res = results[i]
        assert st == cppflow.OK
        alone = run_plan(robots[i], cp, pb.cand, pb.targets, pb.K)
        np.testing.assert_array_equal(res["sel"], alone["sel"], err_msg=f"request {i}")
        np.testing.assert_array_equal(res["q"], alone["q"])
        np.testing.assert_array_equal(res["err"], alone["err"])
        assert res["best"] == float(alone["best"])


@pytest.mark.parametrize("pinned", [0, 96 << 10, 1 << 20])
def test_small_or_no_pinned_pool_equals_alone(pinned):
    """The pinned pool holds copied inputs until their launch retires and each launch's table
    and results while it is in flight; results then move into their requests. With no pool
    (pageable only), or one too small for more than a launch or two at a time, requests
    submitted together and collected only after all are submitted still return exactly
    what cpp_plan returns alone."""
    pbs = _mix(16, seed0=880)
    _, cp = params_pair(lm_iters=10)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    with cppflow.Server(cp, hbm_budget=1 << 30, max_inflight=4, max_batch=3,
                        pinned_bytes=pinned) as srv:
        tickets = [srv.submit(robots[i], pb.cand, pb.targets, pb.K) for i, pb in enumerate(pbs)]
        results = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    assert stats["completed"] == len(pbs) and stats["failed"] == 0
    for i, pb in enumerate(pbs):
        st, res = results[i]
        assert st == cppflow.OK
        alone = run_plan(robots[i], cp, pb.cand, pb.targets, pb.K)
        np.testing.assert_array_equal(res["sel"], alone["sel"])
        np.testing.assert_array_equal(res["q"], alone["q"])
        np.testing.assert_array_equal(res["err"], alone["err"])
        assert res["best"] == float(alone["best"])
