"""Pins for the oracle's Levenberg-Marquardt refinement (§III-C) and its trajectory
report (§II constraints and metrics), plus the seeded input generator.

LM is pinned by the textbook inverse kinematics of a planar 3R arm (both elbow
branches), by its accept/reject invariant (F never increases), by the freeze and
free-joint rules, and end to end on the 50-waypoint plain workload.
"""
import math

import numpy as np
import pytest

import problems
from paper_2309_09102_gb300 import synth
from problems import DEG

RNG = np.random.default_rng(5)


def planar3(orc, a, lo=-3.1, hi=3.1):
    return orc.make_robot(a, [0, 0, 0], [0, 0, 0], [lo] * 3, [hi] * 3)


def planar3_ik(a, x, y, phi):
    """Both analytic solutions of a planar 3R arm for (x, y, phi)."""
    a1, a2, a3 = a
    wx, wy = x - a3 * math.cos(phi), y - a3 * math.sin(phi)
    c2 = (wx * wx + wy * wy - a1 * a1 - a2 * a2) / (2 * a1 * a2)
    sols = []
    for s in (1.0, -1.0):
        q2 = s * math.acos(c2)
        q1 = math.atan2(wy, wx) - math.atan2(a2 * math.sin(q2), a1 + a2 * math.cos(q2))
        q3 = phi - q1 - q2
        q3 = (q3 + math.pi) % (2 * math.pi) - math.pi
        sols.append(np.array([q1, q2, q3]))
    return sols


def test_lm_converges_to_both_planar_branches(orc):
    a = [0.4, 0.3, 0.15]
    robot = planar3(orc, a)
    P = orc.make_params(lm_iters=40, freeze_cost=1e-20)  # run to FP64 convergence
    for _ in range(10):
        x, y = RNG.uniform(0.2, 0.5), RNG.uniform(-0.3, 0.3)
        phi = RNG.uniform(-1, 1)
        R = np.array([[math.cos(phi), -math.sin(phi), 0], [math.sin(phi), math.cos(phi), 0], [0, 0, 1]])
        t7 = np.concatenate([[x, y, 0.0], orc.R_to_quat(R)])
        for sol in planar3_ik(a, x, y, phi):
            seed = sol + RNG.normal(0, 0.05, 3)
            q, hist, _ = orc.lm(robot, P, seed[None], t7[None], want_hist=True)
            np.testing.assert_allclose(q[0], sol, atol=1e-8)


def test_lm_monotone_and_converges_on_plain_workload(orc):
    """F never increases (accept/reject rule); from the search seed every waypoint of the
    T = 50, K = 32 workload reaches 1 mm / 0.1 deg in 10 iterations."""
    pb = problems.build(synth.PLAIN)
    out = orc.plan(pb.robot, pb.params, pb.cand, pb.targets, pb.K)
    assert out["status"] == 0
    seed = pb.cand[np.arange(pb.w.T), :, out["sel"]].astype(np.float64)
    q, hist, iters = orc.lm(pb.robot, pb.params, seed, pb.targets, want_hist=True)
    assert np.all(np.diff(hist, axis=1) <= 0.0)
    np.testing.assert_array_equal(q, out["q"])
    rep = out["report"]
    assert rep["n_pose_fail"] == 0
    assert rep["max_pos"] <= 1e-3 and rep["max_rot"] <= 0.1 * DEG
    assert rep["n_limit_fail"] == 0
    assert rep["valid"] == 1


def test_lm_freezes_at_solution(orc):
    arm = synth.draw_arm(3, 7)
    robot = problems.oracle_robot(arm)
    q = RNG.uniform(-2, 2, (4, 7))
    t = orc.fk_pose(robot, q)
    P = orc.make_params(lm_iters=10)
    q2, hist, iters = orc.lm(robot, P, q, t, want_hist=True)
    assert np.all(iters == 0)
    np.testing.assert_array_equal(q2, q)


def test_lm_free_mask_and_clamp(orc):
    arm = synth.draw_arm(4, 7)
    robot = problems.oracle_robot(arm)
    q_true = RNG.uniform(-2, 2, (6, 7))
    t = orc.fk_pose(robot, q_true)
    seed = q_true + RNG.normal(0, 0.1, q_true.shape)
    mask = synth.wrong_branch_free_mask(7)  # joints 5..7 (1-based) move
    P = orc.make_params(lm_iters=15, free_mask=mask)
    q, _, _ = orc.lm(robot, P, seed, t)
    np.testing.assert_array_equal(q[:, :4], seed[:, :4])
    assert np.any(np.abs(q[:, 4:] - seed[:, 4:]) > 0)
    # a target reachable only outside the limits: the result stays inside them
    robot2 = planar3(orc, [0.4, 0.3, 0.15], lo=-1.0, hi=1.0)
    t2 = orc.fk_pose(robot2, np.array([[0.2, 1.6, -0.3]]))
    q2, _, _ = orc.lm(robot2, orc.make_params(lm_iters=30), np.array([[0.2, 0.9, -0.3]]), t2)
    assert np.all(q2 <= 1.0) and np.all(q2 >= -1.0)


def test_check_report_closed_form(orc):
    """mjac, summed L-inf jump, trajectory length and the 7 deg / limit flags on a
    hand-made trajectory of a planar arm whose poses are the targets."""
    robot = planar3(orc, [0.3, 0.2, 0.1], lo=-2.0, hi=2.0)
    P = orc.make_params()
    q = np.array([[0.0, 0.0, 0.0], [0.05, -0.02, 0.0], [0.05, 0.10, 0.03], [0.05, 0.10, 0.03]])
    t = orc.fk_pose(robot, q)
    err, rep = orc.check(robot, P, q, t)
    assert rep["mjac"] == pytest.approx(0.12)
    assert rep["sum_linf"] == pytest.approx(0.05 + 0.12 + 0.0)
    assert rep["traj_len"] == pytest.approx(0.05 + 0.02 + 0.12 + 0.03)
    assert rep["n_jump_fail"] == 0 and rep["n_limit_fail"] == 0 and rep["valid"] == 1
    q2 = q.copy()
    q2[2, 1] = 0.10 + 8 * DEG  # an 8 deg step in and out
    q2[3, 0] = 2.5             # outside the limit
    _, rep2 = orc.check(robot, P, q2, t)
    assert rep2["n_jump_fail"] == 2 and rep2["n_limit_fail"] == 1
    assert rep2["n_pose_fail"] == 2 and rep2["valid"] == 0


# --------------------------------------------------------------------- generator
def test_splitmix64_reference_value():
    """SplitMix64 from state 0: the first output is 0xE220A8397B1DCDAF (published
    reference sequence of the generator)."""
    from paper_2309_09102_gb300.synth import _mix, _GOLDEN
    assert int(_mix(np.uint64(0) + _GOLDEN)) == 0xE220A8397B1DCDAF


def test_generator_is_deterministic_and_shaped():
    w = synth.SINGLE
    d1 = synth.draw_candidates(w.cand_seed, 30, w.K, w.n, w.p_wb, w.p_out)
    d2 = synth.draw_candidates(w.cand_seed, 30, w.K, w.n, w.p_wb, w.p_out)
    np.testing.assert_array_equal(d1.noise, d2.noise)
    assert abs(d1.noise.std() - 1.0) < 0.01 and abs(d1.noise.mean()) < 0.01
    assert abs(d1.wb.mean() - w.p_wb) < 0.01 and abs(d1.out.mean() - w.p_out) < 0.01
    for T in (50, 300, 2000):
        truth = synth.draw_truth(7, 7, T)
        assert np.max(np.abs(np.diff(truth, axis=0))) <= 5 * DEG + 1e-12
        assert np.max(np.abs(truth)) <= 2.6
    tw = synth.draw_truth(5, 9, 2000, wrist=True)
    assert np.max(np.abs(tw[:, 5])) <= 0.02 + 1e-12


def test_assemble_layout_and_outliers():
    T, K, n = 6, 40, 7
    truth = RNG.uniform(-1, 1, (T, n))
    q_wb = truth + 1.0
    d = synth.draw_candidates(9, T, K, n, 0.3, 0.2)
    lo, hi = np.full(n, -2.8), np.full(n, 2.8)
    c = synth.assemble(truth, q_wb, d, 0.05, lo, hi)
    assert c.shape == (T, n, 64) and c.dtype == np.float32
    assert np.all(c[:, :, K:] == 0)
    ti, ki = np.nonzero(d.out)
    jj = d.out_joint[ti, ki]
    v = c[ti, jj, ki]
    assert np.all((v > 2.8) | (v < -2.8))
    inl = ~d.out & ~d.wb
    resid = (c[:, :, :K].transpose(0, 2, 1) - truth[:, None, :])[inl]
    assert abs(resid.std() / 0.05 - 1) < 0.05
