"""The host-memory plain path, the FP64 Jacobian, the LM work counters and the
arithmetic throughput probe, through the C ABI.

cpp_plan_host is cpp_plan with the copies in and out included, so its results
must equal cpp_plan's bit for bit. The FP64 Jacobian is compared with the
oracle's (the matrix of the LM step, §III-C). The LM counters must count every
waypoint once and at most lm_iters iterations each. The probe must report the
lane operations of its own launch and run at a plausible rate.
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_util import DEV, params_pair, run_plan, torch
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T,K,seed", [(50, 32, 41), (37, 130, 42)])
def test_plan_host_equals_plan(T, K, seed):
    tt = torch()
    pb = problems.small(T=T, K=K, seed=seed)
    _, cp = params_pair(lm_iters=10)
    rob = cppflow.robot_from_arm(pb.arm)
    ref = run_plan(rob, cp, pb.cand, pb.targets, pb.K)
    T_, n, Kp = pb.cand.shape
    ws = tt.empty(cppflow.plan_host_workspace_size(T, K, Kp, n), dtype=tt.uint8, device=DEV)
    cand = tt.from_numpy(pb.cand).pin_memory().numpy()
    sel = np.full(T, -1, np.int32)
    best = np.zeros(1, np.float32)
    q = np.zeros((T, n), np.float32)
    err = np.zeros((T, 2))
    rep = cppflow.Report()
    for _ in range(2):  # a second call reuses the workspace
        st = cppflow.plan_host(rob, cp, cand, pb.targets, K, ws, sel, best, q, err, rep)
        assert st == cppflow.OK
        np.testing.assert_array_equal(sel, ref["sel"])
        assert best[0] == ref["best"]
        np.testing.assert_array_equal(q, ref["q"])
        np.testing.assert_array_equal(err, ref["err"])
        assert rep.as_dict() == ref["report"]


def test_plan_host_rejects_small_workspace():
    tt = torch()
    pb = problems.small(T=10, K=16, seed=43)
    _, cp = params_pair()
    rob = cppflow.robot_from_arm(pb.arm)
    ws = tt.empty(256, dtype=tt.uint8, device=DEV)
    with pytest.raises(cppflow.CppflowError):
        cppflow.plan_host(rob, cp, pb.cand, pb.targets, pb.K, ws)


def test_jacobian_f64_matches_oracle():
    tt = torch()
    for n, wrist in ((7, False), (9, True)):
        arm = synth.draw_arm(5 + n, n, wrist)
        orob = oracle.make_robot(arm.a, arm.d, arm.alpha, arm.lo, arm.hi, arm.theta0)
        q = np.random.default_rng(n).uniform(-2.5, 2.5, (37, n))
        J = tt.empty(37, 6, n, dtype=tt.float64, device=DEV)
        cppflow.jacobian_f64(cppflow.robot_from_arm(arm), tt.from_numpy(q).to(DEV), J)
        got = J.cpu().numpy()
        for c in range(37):
            np.testing.assert_allclose(got[c], oracle.jacobian(orob, q[c]), rtol=0, atol=1e-12)


def test_lm_counters_count_waypoints_and_iterations():
    tt = torch()
    pb = problems.small(T=70, K=40, seed=44)
    _, cp = params_pair(lm_iters=12)
    rob = cppflow.robot_from_arm(pb.arm)
    q0 = pb.cand[:, :, 0].astype(np.float32)
    qo = tt.empty(70, pb.w.n, dtype=tt.float32, device=DEV)
    tt.cuda.synchronize()
    cppflow.counters_reset()
    cppflow.lm_refine(rob, cp, tt.from_numpy(q0).to(DEV), tt.from_numpy(pb.targets).to(DEV), qo)
    cppflow.lm_refine(rob, cp, tt.from_numpy(q0).to(DEV), tt.from_numpy(pb.targets).to(DEV), qo)
    tt.cuda.synchronize()
    c = cppflow.counters_read()
    assert c["lm_waypoints"] == 2 * 70
    assert 2 * 70 <= c["lm_iterations"] <= 2 * 70 * 12   # every start is far from exact
    assert c["lm_iterations"] % 2 == 0                     # the two runs are identical


@pytest.mark.parametrize("kind", [cppflow.PROBE_FP32, cppflow.PROBE_FP64])
def test_peak_probe_reports_its_work(kind):
    tt = torch()
    sink = tt.zeros(1, dtype=tt.float64, device=DEV)
    sms = tt.cuda.get_device_properties(0).multi_processor_count
    st = tt.cuda.current_stream()
    ops = cppflow.peak_probe(kind, 2, 4096, sink)   # warm-up
    e0, e1 = tt.cuda.Event(enable_timing=True), tt.cuda.Event(enable_timing=True)
    e0.record(st)
    ops = cppflow.peak_probe(kind, 2, 4096, sink)
    e1.record(st)
    tt.cuda.synchronize()
    assert ops == 2 * sms * 256 * 8 * 4096 * 2
    rate = ops / (e0.elapsed_time(e1) / 1e3)
    assert rate > 1e11   # far below any GB300 rate, far above a broken probe
    with pytest.raises(cppflow.CppflowError):
        cppflow.peak_probe(7, 2, 4096, sink)
