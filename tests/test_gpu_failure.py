"""Failure detection on the device without a fault: every wait in the kernels is bounded
and ends with CPP_ERR_TIMEOUT in the caller's device status. Here a wait on an mbarrier
that nothing completes (the flag that nobody sets) runs out after a short limit, with the
CTA-scope and the cluster-scope waits the search kernels use; the context stays usable."""
import time

import pytest

import problems
from gpu_util import params_pair, run_plan, torch
from paper_2309_09102_gb300 import cppflow

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cluster_scope", [False, True])
def test_bounded_wait_ends_with_timeout_status(cluster_scope):
    tt = torch()
    st = tt.zeros(1, dtype=tt.int32, device="cuda:0")
    limit_ns = 2_000_000
    tt.cuda.synchronize()
    t0 = time.perf_counter()
    cppflow.wait_selftest(limit_ns, cluster_scope, st)
    tt.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert int(st.item()) == cppflow.ERR_TIMEOUT
    assert elapsed >= limit_ns * 1e-9
    # the context is still usable: a plan right after matches a fresh one
    pb = problems.small(T=20, K=40, seed=31)
    _, cp = params_pair(lm_iters=10)
    res = run_plan(cppflow.robot_from_arm(pb.arm), cp, pb.cand, pb.targets, pb.K)
    assert res["status"] == 0 and res["report"]["valid"] == 1


def test_selftest_arguments_are_validated():
    tt = torch()
    st = tt.zeros(1, dtype=tt.int32, device="cuda:0")
    with pytest.raises(cppflow.CppflowError):
        cppflow.wait_selftest(10, False, st)
    with pytest.raises(cppflow.CppflowError):
        cppflow.wait_selftest(1_000_000, False, None)
