"""GPU parity of the §III-C trajectory-length step and of the alternation of pose
phases with such steps (cpp_smooth_step, params.smooth_rounds).

The step is compared with the oracle's block-tridiagonal solve on the same FP32
trajectory (the GPU stores FP32, so within one FP32 ulp); the gate (every waypoint
within tau) bit-exactly; the whole alternation against the oracle's at the
end-to-end tolerances, and batched against alone bit for bit.
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_util import JUMP_TOL, TAU_POS, TAU_ROT, dev, params_pair, run_plan, torch
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu

ULP_TOL = 3e-7  # one FP32 ulp at |q| <= 2.8 rad


def gpu_smooth(robot, params, q32, targets):
    tt = torch()
    qd = dev(q32)
    st = tt.zeros(1, dtype=tt.int32, device="cuda:0")
    cppflow.smooth_step(robot, params, qd, dev(targets), st)
    tt.cuda.synchronize()
    assert int(st.item()) == 0
    return qd.cpu().numpy()


def smooth_path(seed, T, n, amp=0.8):
    r = np.random.default_rng(seed)
    t = np.linspace(0, 1, T)[:, None]
    q = r.uniform(-1, 1, n) + amp * np.sin(2 * np.pi * r.uniform(0.5, 2, n) * t + r.uniform(0, 6, n))
    return (q + r.normal(0, 0.02, (T, n))).astype(np.float32)   # jitter for the step to remove


@pytest.mark.parametrize("T,n,lam", [(2, 7, 1.0), (50, 7, 0.1), (300, 7, 1.0), (2000, 9, 10.0)])
def test_smooth_step_matches_oracle(T, n, lam):
    """Targets are the FK of the trajectory itself, so the gate is open."""
    arm = synth.draw_arm(7 + n, n)
    orob = problems.oracle_robot(arm)
    q32 = np.clip(smooth_path(T, T, n), arm.lo + 0.1, arm.hi - 0.1).astype(np.float32)
    targets = oracle.fk_pose(orob, q32.astype(np.float64))
    _, cp = params_pair(smooth_lambda=lam)
    got = gpu_smooth(cppflow.robot_from_arm(arm), cp, q32, targets)
    ref, ok = oracle.diff_step(orob, q32.astype(np.float64), lam)
    assert ok
    np.testing.assert_allclose(got, ref, rtol=0, atol=ULP_TOL)
    assert not np.array_equal(got, q32)


def test_smooth_step_gate_and_clamp():
    T, n = 80, 7
    arm = synth.draw_arm(3, n)
    orob = problems.oracle_robot(arm)
    rob = cppflow.robot_from_arm(arm)
    q32 = np.clip(smooth_path(5, T, n), arm.lo + 0.1, arm.hi - 0.1).astype(np.float32)
    targets = oracle.fk_pose(orob, q32.astype(np.float64))
    _, cp = params_pair()
    bad = targets.copy()
    bad[40, 0] += 0.01                      # one waypoint 1 cm off: no step
    np.testing.assert_array_equal(gpu_smooth(rob, cp, q32, bad), q32)
    # at the limits: the step is clamped (and equals the oracle's clamped step)
    edge = q32.copy()
    edge[::2, 1] = arm.hi[1]
    edge[1::2, 1] = arm.lo[1]
    t_edge = oracle.fk_pose(orob, edge.astype(np.float64))
    got = gpu_smooth(rob, cp, edge, t_edge)
    assert np.all(got[:, 1] <= arm.hi[1]) and np.all(got[:, 1] >= arm.lo[1])
    np.testing.assert_allclose(got, oracle.diff_step(orob, edge.astype(np.float64), 1.0)[0],
                               rtol=0, atol=ULP_TOL)


@pytest.fixture(scope="module")
def plain():
    return problems.build(synth.PLAIN)


def test_alternation_matches_oracle(plain):
    pb = plain
    op, cp0 = params_pair(lm_iters=pb.w.lm_iters)
    _, cp3 = params_pair(lm_iters=pb.w.lm_iters, smooth_rounds=3, smooth_lambda=1.0)
    base = run_plan(cppflow.robot_from_arm(pb.arm), cp0, pb.cand, pb.targets, pb.K)
    out = run_plan(cppflow.robot_from_arm(pb.arm), cp3, pb.cand, pb.targets, pb.K)
    np.testing.assert_array_equal(out["sel"], base["sel"])          # the search is unchanged
    seed = pb.cand[np.arange(pb.w.T), :, out["sel"]].astype(np.float64)
    ref, taken = oracle.lm_smooth(pb.robot, op, seed, pb.targets, 3, 1.0)
    assert taken == 3
    rep = out["report"]
    assert rep["valid"] == 1 and rep["max_pos"] <= TAU_POS and rep["max_rot"] <= TAU_ROT
    _, rref = oracle.check(pb.robot, op, ref, pb.targets)
    assert abs(rep["mjac"] - rref["mjac"]) <= JUMP_TOL
    assert abs(rep["traj_len"] - rref["traj_len"]) <= JUMP_TOL * pb.w.T
    np.testing.assert_allclose(out["q"], ref, rtol=0, atol=1e-4)
    # smoother than the pose-only refinement
    assert rep["mjac"] < base["report"]["mjac"]
    assert rep["traj_len"] < base["report"]["traj_len"]


def test_alternation_batched_equals_alone(plain):
    """Three requests in one batch with smooth_rounds = 2 give the plans each gives alone."""
    tt = torch()
    pbs = [plain] + [problems.build(synth.Workload(f"sm_{r}", 7, 40 + 10 * r, 64, 0.03, 0.2, 0.0, 10,
                                                     arm_seed=20 + r, path_seed=30 + r,
                                                     cand_seed=40 + r)) for r in range(2)]
    _, cp = params_pair(lm_iters=10, smooth_rounds=2, smooth_lambda=0.5)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    alone = [run_plan(robots[r], cp, pb.cand, pb.targets, pb.K) for r, pb in enumerate(pbs)]
    bufs, descs = [], []
    for r, pb in enumerate(pbs):
        T, n, Kp = pb.cand.shape
        b = dict(cand=dev(pb.cand), targets=dev(pb.targets),
                 sel=tt.empty(T, dtype=tt.int32, device="cuda:0"),
                 q=tt.empty(T, n, dtype=tt.float32, device="cuda:0"),
                 err=tt.empty(T, 2, dtype=tt.float64, device="cuda:0"),
                 rep=tt.zeros(cppflow.REPORT_BYTES, dtype=tt.uint8, device="cuda:0"),
                 best=tt.empty(1, dtype=tt.float32, device="cuda:0"))
        bufs.append(b)
        descs.append(cppflow.PlanDesc(T, pb.K, Kp, r, b["cand"].data_ptr(), b["targets"].data_ptr(),
                                      b["sel"].data_ptr(), b["q"].data_ptr(), b["err"].data_ptr(),
                                      b["rep"].data_ptr(), b["best"].data_ptr()))
    ws = tt.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=tt.uint8, device="cuda:0")
    st = tt.zeros(len(descs), dtype=tt.int32, device="cuda:0")
    batch = cppflow.Batch(robots, cp, descs, ws, st)
    assert batch.launches(cppflow.STAGE_LM) == 5      # pose, (step, pose) x 2
    batch.run(cppflow.STAGE_ALL)
    tt.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    for r in range(len(pbs)):
        np.testing.assert_array_equal(bufs[r]["sel"].cpu().numpy(), alone[r]["sel"])
        np.testing.assert_array_equal(bufs[r]["q"].cpu().numpy(), alone[r]["q"])
        np.testing.assert_array_equal(bufs[r]["err"].cpu().numpy(), alone[r]["err"])
