"""Pins for the oracle's cpf-BatchOpt (§III, commented text: the smoothest candidate
trajectories refined directly) and the lane-coherent generator it needs.

Lane smoothness is pinned by a fixture worked by hand (including an FP32 rounding
that FP64 would not make) and bit-exactly by NumPy's FP32 differences and a stable
argsort; the refinement by orc_lm on the same lane; the choice by the reports;
end to end on the coherent plain workload.
"""
import numpy as np

import oracle
import problems
from paper_2309_09102_gb300 import synth


def test_lane_mjac_and_selection_match_numpy():
    pb = problems.build(synth.PLAIN, coherent=True)
    cand = pb.cand.copy()
    cand[7, 2, 5] = np.nan                       # a non-finite lane goes last
    m = oracle.lane_mjac_f32(cand, pb.K)
    d = np.abs(np.diff(cand[:, :, :pb.K], axis=0)).max(axis=(0, 1))
    ref = np.where(np.isfinite(cand[:, :, :pb.K]).all(axis=(0, 1)), d, np.float32(np.inf))
    np.testing.assert_array_equal(m, ref.astype(np.float32))
    out = oracle.batch_opt(pb.robot, pb.params, cand, pb.targets, pb.K, lanes=pb.K)
    np.testing.assert_array_equal(out["sel"], np.argsort(ref, kind="stable"))
    assert out["sel"][-1] == 5 and np.isinf(out["mjac"][-1])


def test_lane_mjac_hand_computed():
    """Three lanes of T = 3, n = 2 worked by hand (padding lane 3 ignored): lane 0 has
    steps (0.5, 0.25) and (0.25, 1.25), so 1.25; lane 1 is constant, 0; lane 2 jumps by 2
    and back, 2. Lane 4 of a second fixture holds 1 and 1e-8 on consecutive waypoints:
    in FP32 the difference rounds to exactly 1 (1e-8 is below half an ulp of 1), not the
    FP64 value 0.99999999; a lane holding inf is +inf."""
    lanes = np.array([
        [[0.0, 0.0], [0.5, -0.25], [0.75, 1.0]],
        [[1.0, 2.0], [1.0, 2.0], [1.0, 2.0]],
        [[0.0, 0.0], [-2.0, 0.0], [0.0, 0.0]],
        [[9.0, 9.0], [-9.0, 9.0], [9.0, -9.0]],   # padding lane, never read
    ], np.float32)                                  # [k][i][j]
    cand = np.ascontiguousarray(np.transpose(lanes, (1, 2, 0)))  # [T][n][Kp]
    np.testing.assert_array_equal(oracle.lane_mjac_f32(cand, 3),
                                  np.array([1.25, 0.0, 2.0], np.float32))
    two = np.zeros((2, 1, 4), np.float32)
    two[0, 0, 0], two[1, 0, 0] = 1.0, 1e-8
    two[1, 0, 1] = np.inf
    m = oracle.lane_mjac_f32(two, 2)
    assert m[0] == np.float32(1.0) and np.isinf(m[1])


def test_each_lane_is_refined_as_its_own_trajectory():
    pb = problems.build(synth.PLAIN, coherent=True)
    out = oracle.batch_opt(pb.robot, pb.params, pb.cand, pb.targets, pb.K, lanes=3)
    for l, k in enumerate(out["sel"]):
        seed = pb.cand[:, :, k].astype(np.float64)
        q, _, _ = oracle.lm(pb.robot, pb.params, seed, pb.targets)
        np.testing.assert_array_equal(out["q"][l], q)
        _, rep = oracle.check(pb.robot, pb.params, q, pb.targets)
        assert rep == out["reports"][l]
    valid = [r["valid"] for r in out["reports"]]
    assert out["best"] == (valid.index(1) if 1 in valid else -1)


def test_batch_opt_needs_coherent_lanes():
    """On lane-coherent candidates the smoothest lane refines to a valid plan; on
    independent draws (every candidate its own branch and noise) no lane does."""
    coh = problems.build(synth.PLAIN, coherent=True)
    out = oracle.batch_opt(coh.robot, coh.params, coh.cand, coh.targets, coh.K, lanes=5)
    assert out["best"] == 0 and out["reports"][0]["valid"] == 1
    ind = problems.build(synth.PLAIN)
    out2 = oracle.batch_opt(ind.robot, ind.params, ind.cand, ind.targets, ind.K, lanes=5)
    assert out2["best"] == -1


def test_coherent_generator():
    d = synth.draw_candidates_coherent(3, 400, 64, 7, 0.25, 0.05, rho=0.98)
    assert np.all(d.wb == d.wb[0][None, :])                  # branch chosen per lane
    assert abs(d.noise.std() - 1.0) < 0.1
    c = np.corrcoef(d.noise[1:, :, 0].ravel(), d.noise[:-1, :, 0].ravel())[0, 1]
    assert abs(c - 0.98) < 0.01
