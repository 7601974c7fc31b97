"""Workload-level GPU parity: the batched uneven launch and the 9-DoF near-singular
stress case (T = 2000, K = 1024).

The oracle finishes a prefix of the stress lattice in seconds, so the search is
compared bit-exactly there; at full size the checks are properties that hold at
any size (the backtracked path's own FP32 cost equals the reported minimum, the
FP64 LM meets 1 mm / 0.1 deg at every waypoint and tracks the oracle's joint
jumps) plus sampled node costs against the oracle.
"""
import math

import numpy as np
import pytest

import oracle
import problems
from gpu_util import (JUMP_TOL, TAU_POS, TAU_ROT, dev, params_pair, path_cost_f32, run_dp, run_lm,
                      run_mask, torch)
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu


def test_batched_uneven_launch_matches_oracle():
    """Requests of the batched uneven workload (T ~ U{50..1000}, K in {128, 256, 512},
    arms from 8 seeded chains) in one launch per stage: every search equals the oracle's
    FP32 search on the same node costs, every refined plan is valid."""
    tt = torch()
    ws_ = [synth.batched_request(r) for r in range(10)]
    pbs = [problems.build(w) for w in ws_]
    _, cp = params_pair(lm_iters=20)
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    keep, descs = [], []
    for r, pb in enumerate(pbs):
        T, n, Kp = pb.cand.shape
        b = dict(cand=dev(pb.cand), targets=dev(pb.targets),
                 sel=tt.empty(T, dtype=tt.int32, device="cuda:0"),
                 q=tt.empty(T, n, dtype=tt.float32, device="cuda:0"),
                 err=tt.empty(T, 2, dtype=tt.float64, device="cuda:0"),
                 rep=tt.zeros(cppflow.REPORT_BYTES, dtype=tt.uint8, device="cuda:0"),
                 best=tt.empty(1, dtype=tt.float32, device="cuda:0"))
        keep.append(b)
        descs.append(cppflow.PlanDesc(T, pb.K, Kp, r, b["cand"].data_ptr(), b["targets"].data_ptr(),
                                      b["sel"].data_ptr(), b["q"].data_ptr(), b["err"].data_ptr(),
                                      b["rep"].data_ptr(), b["best"].data_ptr()))
    ws = tt.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=tt.uint8, device="cuda:0")
    st = tt.zeros(len(descs), dtype=tt.int32, device="cuda:0")
    cppflow.plan_batch(robots, cp, descs, ws, st)
    tt.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    for r, pb in enumerate(pbs):
        g = run_mask(robots[r], cp, pb.cand, pb.targets, pb.K)
        ref = oracle.dp_f32(pb.cand, g.pen, pb.K)
        np.testing.assert_array_equal(keep[r]["sel"].cpu().numpy(), ref["sel"])
        assert float(keep[r]["best"].item()) == float(ref["best"])
        rep = cppflow.report_from_bytes(keep[r]["rep"].cpu().numpy().tobytes())
        assert rep["valid"] == 1, (r, rep)
        assert rep["max_pos"] <= TAU_POS and rep["max_rot"] <= TAU_ROT


@pytest.fixture(scope="module")
def stress():
    return problems.build(synth.STRESS)


def test_stress_search_prefix_bit_exact(stress):
    """The first 120 waypoints of the 9-DoF, K = 1024 lattice: identical indices and cost."""
    pb = stress
    Tp = 120
    cand = np.ascontiguousarray(pb.cand[:Tp])
    tg = np.ascontiguousarray(pb.targets[:Tp])
    _, cp = params_pair()
    g = run_mask(cppflow.robot_from_arm(pb.arm), cp, cand, tg, pb.K)
    got = run_dp(cand, g.pen, pb.K)
    ref = oracle.dp_f32(cand, g.pen, pb.K)
    np.testing.assert_array_equal(got["sel"], ref["sel"])
    assert got["best"] == ref["best"]


def test_stress_full_size_properties(stress):
    """Full T = 2000, K = 1024: the path returned by backtracking costs exactly the reported
    minimum (recomputed independently in FP32), and sampled node costs match the oracle."""
    pb = stress
    _, cp = params_pair()
    g = run_mask(cppflow.robot_from_arm(pb.arm), cp, pb.cand, pb.targets, pb.K)
    got = run_dp(pb.cand, g.pen, pb.K)
    assert got["status"] == 0
    assert path_cost_f32(pb.cand, g.pen, pb.K, got["sel"]) == got["best"]
    rng = np.random.default_rng(5)
    rows = rng.choice(pb.w.T, 40, replace=False)
    op, _ = params_pair()
    m, pen, err = oracle.mask(pb.robot, op, np.ascontiguousarray(pb.cand[rows]),
                              np.ascontiguousarray(pb.targets[rows]), pb.K)
    near = (np.abs(err[..., 0] - op.tau_pos) <= 1e-5) | (np.abs(err[..., 1] - op.tau_rot) <= 1e-5)
    np.testing.assert_array_equal(g.pen[rows][~near], pen[~near])
    np.testing.assert_array_equal(g.mask[rows][~near], m[~near])


def test_stress_lm_fp64_vs_fp32_vs_oracle(stress):
    """Near-singular wrist (joint 6 within 0.02 rad of 0): the all-FP64 GPU LM meets
    1 mm / 0.1 deg everywhere and its max joint jump is within 1e-4 rad of the oracle's;
    the FP32-Jacobian LM's errors are reported beside it."""
    pb = stress
    op, cp = params_pair(lm_iters=20)
    g = run_mask(cppflow.robot_from_arm(pb.arm), cp, pb.cand, pb.targets, pb.K)
    seed = run_dp(pb.cand, g.pen, pb.K)["seed"]
    q_orc, _, _ = oracle.lm(pb.robot, op, seed.astype(np.float64), pb.targets)
    e_orc, rep_orc = oracle.check(pb.robot, op, q_orc, pb.targets)
    out = {}
    for mode in (0, 1):
        _, cpm = params_pair(lm_iters=20, lm_fp64=mode)
        q, err = run_lm(cppflow.robot_from_arm(pb.arm), cpm, seed, pb.targets)
        _, rep = oracle.check(pb.robot, op, q.astype(np.float64), pb.targets)
        out[mode] = (q, err, rep)
    q64, err64, rep64 = out[1]
    assert rep_orc["n_pose_fail"] == 0
    assert np.max(err64[:, 0]) <= TAU_POS and np.max(err64[:, 1]) <= TAU_ROT
    assert abs(rep64["mjac"] - rep_orc["mjac"]) <= JUMP_TOL
    q32, err32, rep32 = out[0]
    print(f"stress LM: oracle max pos {rep_orc['max_pos']:.2e} m rot {math.degrees(rep_orc['max_rot']):.2e} deg "
          f"mjac {rep_orc['mjac']:.6f}; fp64 GPU max pos {err64[:, 0].max():.2e} m rot "
          f"{math.degrees(err64[:, 1].max()):.2e} deg mjac {rep64['mjac']:.6f}; fp32-Jacobian GPU max pos "
          f"{err32[:, 0].max():.2e} m rot {math.degrees(err32[:, 1].max()):.2e} deg mjac {rep32['mjac']:.6f}")
    assert np.max(err32[:, 0]) <= TAU_POS and np.max(err32[:, 1]) <= TAU_ROT
