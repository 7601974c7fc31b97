"""The paper's own search objective (min-max mjac, §III-B) and its re-search with appended
candidates, on the GPU against the oracle.

The min-max recurrence uses only max and min, so the GPU's indices and cost must equal
the oracle's exactly; the search path's mjac reported by the backtracking kernel must
equal the oracle's mjac of the same selection. The re-search masks only the appended
lanes of a resident lattice; the result must equal a search of the full lattice by the
oracle, and its mjac can only go down.
"""
import math

import numpy as np
import pytest

import oracle
import problems
from gpu_util import dev, params_pair, run_dp_ex, run_mask, torch
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T,K,n,wrist", [(30, 40, 7, False), (20, 300, 7, False), (12, 600, 9, True),
                                         (9, 60, 6, False), (6, 50, 3, False), (1, 8, 7, False)])
def test_minmax_search_matches_oracle(T, K, n, wrist):
    pb = problems.small(T=T, K=K, n=n, wrist=wrist, seed=77 + T + K)
    _, cp = params_pair(tau_pos=0.05, tau_rot=math.radians(5.0))
    g = run_mask(cppflow.robot_from_arm(pb.arm), cp, pb.cand, pb.targets, pb.K)
    for objective in (cppflow.DP_SUM, cppflow.DP_MINMAX):
        got = run_dp_ex(pb.cand, g.pen, pb.K, objective)
        ref = oracle.dp_f32(pb.cand, g.pen, pb.K, objective=objective)
        np.testing.assert_array_equal(got["sel"], ref["sel"])
        assert got["best"] == ref["best"]
        assert got["mjac"] == np.float32(oracle.path_mjac_f32(pb.cand, ref["sel"]))


def test_minmax_batched_throughput_kernel():
    """40 requests (one CTA each, not clusters) under the min-max objective."""
    tt = torch()
    pbs = [problems.small(T=5 + (i % 4), K=420 + 8 * (i % 5), seed=5000 + i) for i in range(40)]
    _, cp = params_pair(tau_pos=0.05, tau_rot=math.radians(5.0), lm_iters=5,
                        dp_objective=cppflow.DP_MINMAX)
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
    cppflow.plan_batch(robots, cp, descs, ws, tt.zeros(40, dtype=tt.int32, device="cuda:0"))
    tt.cuda.synchronize()
    for r, pb in enumerate(pbs):
        g = run_mask(robots[r], cp, pb.cand, pb.targets, pb.K)
        ref = oracle.dp_f32(pb.cand, g.pen, pb.K, objective=1)
        np.testing.assert_array_equal(keep[r]["sel"].cpu().numpy(), ref["sel"])
        assert float(keep[r]["best"].item()) == float(ref["best"])


def test_research_with_appended_candidates():
    """Search 32 candidates with the min-max objective; if the path's mjac exceeds 12 deg
    (the paper's re-search threshold) append 64 more candidates to the same resident
    lattice, mask only those, and search again. Each stage equals the oracle's search of
    the lattice it sees, and the mjac does not increase."""
    tt = torch()
    K0, K1 = 32, 96
    w = synth.Workload("research_T80", 7, 80, K1, 0.08, 0.35, 0.05, 10, arm_seed=21, path_seed=22,
                       cand_seed=23)
    pb = problems.build(w)          # K1 candidates; the first K0 lanes form the first search
    T, n, Kp = pb.cand.shape
    _, cp = params_pair()
    rob = cppflow.robot_from_arm(pb.arm)
    cand_d = dev(pb.cand)
    tg = dev(pb.targets)
    mask = tt.empty(T, Kp, dtype=tt.uint8, device="cuda:0")
    pen = tt.empty(T, Kp, dtype=tt.float32, device="cuda:0")
    ws = tt.empty(cppflow.dp_workspace_size(T, Kp), dtype=tt.uint8, device="cuda:0")
    sel = tt.empty(T, dtype=tt.int32, device="cuda:0")
    best = tt.empty(1, dtype=tt.float32, device="cuda:0")
    mj = tt.empty(1, dtype=tt.float32, device="cuda:0")
    st = tt.zeros(1, dtype=tt.int32, device="cuda:0")
    # first search: lanes [0, K0)
    cppflow.mask(rob, cp, cand_d, tg, K0, mask, pen)
    cppflow.dp_search_ex(cand_d, pen, K0, cppflow.DP_MINMAX, ws, sel, best, None, mj, st)
    tt.cuda.synchronize()
    pen0 = pen.cpu().numpy().copy()
    ref0 = oracle.dp_f32(pb.cand, pen0, K0, objective=1)
    np.testing.assert_array_equal(sel.cpu().numpy(), ref0["sel"])
    mjac0 = float(mj.item())
    assert mjac0 == np.float32(oracle.path_mjac_f32(pb.cand, ref0["sel"]))
    # re-search: mask only the appended lanes [K0, K1), keep the first search's costs
    cppflow.mask_range(rob, cp, cand_d, tg, K1, K0, mask, pen)
    cppflow.dp_search_ex(cand_d, pen, K1, cppflow.DP_MINMAX, ws, sel, best, None, mj, st)
    tt.cuda.synchronize()
    pen1 = pen.cpu().numpy()
    np.testing.assert_array_equal(pen1[:, :K0], pen0[:, :K0])      # retained
    full = run_mask(rob, cp, pb.cand, pb.targets, K1)               # mask of the whole lattice
    np.testing.assert_array_equal(pen1[:, :K1], full.pen[:, :K1])
    ref1 = oracle.dp_f32(pb.cand, pen1, K1, objective=1)
    np.testing.assert_array_equal(sel.cpu().numpy(), ref1["sel"])
    assert float(mj.item()) <= mjac0
    print(f"re-search: mjac {math.degrees(mjac0):.2f} deg with {K0} candidates -> "
          f"{math.degrees(float(mj.item())):.2f} deg with {K1}")
