"""Oracle-built problem instances for the tests.

Inputs come from the seeded generator (random draws + assembly); the two steps
of input construction that need kinematics -- target poses = FK(true path) and
the wrong-branch re-solve -- are done here with the CPU oracle, so no input or
expected value in the tests ever comes from the CUDA path.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import oracle
from paper_2309_09102_gb300 import synth


@dataclass
class Problem:
    w: synth.Workload
    arm: synth.Arm
    robot: oracle.Robot
    params: oracle.Params
    truth: np.ndarray      # [T][n] FP64
    targets: np.ndarray    # [T][7] FP64 xyz + wxyz
    q_wb: np.ndarray       # [T][n] FP64
    cand: np.ndarray       # [T][n][Kp] FP32
    K: int
    Kp: int


def oracle_robot(arm: synth.Arm) -> oracle.Robot:
    return oracle.make_robot(arm.a, arm.d, arm.alpha, arm.lo, arm.hi, arm.theta0)


def build(w: synth.Workload, coherent: bool = False, **param_overrides) -> Problem:
    """Oracle-built problem of a workload; coherent=True draws lane-coherent candidates
    (synth.draw_candidates_coherent) instead of independent ones."""
    oracle.build()
    arm = synth.draw_arm(w.arm_seed, w.n, w.wrist)
    robot = oracle_robot(arm)
    truth = synth.draw_truth(w.path_seed, w.n, w.T, w.wrist)
    targets = oracle.fk_pose(robot, truth)
    free = synth.wrong_branch_free_mask(w.n)
    if free:
        P_wb = oracle.make_params(lm_iters=30, free_mask=free)
        q_wb, _, _ = oracle.lm(robot, P_wb, synth.wrong_branch_start(truth), targets)
    else:
        q_wb = truth.copy()
    draw = synth.draw_candidates_coherent if coherent else synth.draw_candidates
    draws = draw(w.cand_seed, w.T, w.K, w.n, w.p_wb, w.p_out)
    cand = synth.assemble(truth, q_wb, draws, w.sigma, arm.lo, arm.hi)
    kw = dict(lm_iters=w.lm_iters, lambda0=w.lambda0)
    kw.update(param_overrides)
    params = oracle.make_params(**kw)
    return Problem(w, arm, robot, params, truth, targets, q_wb, cand, w.K, cand.shape[2])


def small(T=12, K=40, n=7, seed=11, sigma=0.05, p_wb=0.25, p_out=0.1, lm_iters=10,
          wrist=False) -> Problem:
    """A small instance that spans several warps and a ragged K tail."""
    w = synth.Workload(f"small_T{T}_K{K}_n{n}_s{seed}", n, T, K, sigma, p_wb, p_out, lm_iters,
                       wrist=wrist, arm_seed=seed, path_seed=seed + 1, cand_seed=seed + 2)
    return build(w)


DEG = math.pi / 180.0
