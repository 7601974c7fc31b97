"""Cluster launches over requests of different Kp.

A cluster launch is sized for its largest Kp, so a smaller request leaves the
last CTAs of its cluster without successors. Those CTAs must stay out of the
record exchange: if they took part as receivers only, the CTAs that own
successors would not wait for them and could run more than one layer ahead,
into record buffers and mbarrier phases the idle CTAs had not finished with.
The search then stalls on the bounded wait (status CPP_ERR_TIMEOUT) when the
idle CTAs fall behind, which happens when other kernels share their SMs.

This file runs mixed-Kp batches in the cluster form: alone against the oracle's
FP32 search (§III-B) on the GPU's node costs, then many at once on several
streams, repeatedly, where every request must finish with status 0 and the same
indices and costs as alone.
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_util import dev, params_pair, run_mask, torch
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu

# largest Kp 1024 sets the cluster; K = 100 owns 1 or 2 of its CTAs, K = 40 (Kp 64) one
MIXED = [(40, 1000), (120, 100), (70, 300), (50, 600), (90, 128), (60, 40)]


def workload(r, T, K, base):
    return synth.Workload(f"extent_r{r}", 7, T, K, 0.05, 0.25, 0.05, 20, 1e-3,
                          arm_seed=100 + (r % 8), path_seed=base + r, cand_seed=base + 50 + r)


def make_batch(pbs, cp, stream):
    tt = torch()
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
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
    batch = cppflow.Batch(robots, cp, descs, ws, st, stream)
    # no heavy split: one forward launch over the whole table, which a batch this
    # small takes in the cluster form
    batch.set_split(0.0, 0, stream)
    return dict(batch=batch, bufs=bufs, ws=ws, st=st, robots=robots, stream=stream)


def outputs(B):
    return [(b["sel"].cpu().numpy(), b["best"].cpu().numpy()) for b in B["bufs"]]


def test_mixed_kp_cluster_launch_matches_the_oracle():
    tt = torch()
    pbs = [problems.build(workload(r, T, K, 7100)) for r, (T, K) in enumerate(MIXED)]
    _, cp = params_pair(lm_iters=10)
    stream = tt.cuda.Stream()
    B = make_batch(pbs, cp, stream)
    try:
        B["batch"].run(cppflow.STAGE_ALL, stream)
        stream.synchronize()
        assert B["batch"].launches(cppflow.STAGE_DP_FORWARD) == 1
        assert np.all(B["st"].cpu().numpy() == 0)
        for r, pb in enumerate(pbs):
            g = run_mask(B["robots"][r], cp, pb.cand, pb.targets, pb.K)
            ref = oracle.dp_f32(pb.cand, g.pen, pb.K)
            np.testing.assert_array_equal(B["bufs"][r]["sel"].cpu().numpy(), ref["sel"])
            assert float(B["bufs"][r]["best"].item()) == float(ref["best"])
    finally:
        B["batch"].close()


def test_mixed_kp_cluster_launches_side_by_side():
    tt = torch()
    _, cp = params_pair(lm_iters=10)
    n_batches, reps = 12, 4
    batches = []
    try:
        for j in range(n_batches):
            shapes = MIXED[j % len(MIXED):] + MIXED[:j % len(MIXED)]
            pbs = [problems.build(workload(r, T, K, 7300 + 100 * j)) for r, (T, K) in enumerate(shapes)]
            batches.append(make_batch(pbs, cp, tt.cuda.Stream()))
        alone = []
        for B in batches:
            B["batch"].run(cppflow.STAGE_ALL, B["stream"])
            B["stream"].synchronize()
            assert np.all(B["st"].cpu().numpy() == 0)
            alone.append(outputs(B))
        for _ in range(reps):
            for B in batches:
                B["st"].zero_()
                for b in B["bufs"]:
                    b["sel"].fill_(-7)
                    b["best"].fill_(-7.0)
            tt.cuda.synchronize()
            for B in batches:
                B["batch"].run(cppflow.STAGE_ALL, B["stream"])
            tt.cuda.synchronize()
            for j, B in enumerate(batches):
                assert np.all(B["st"].cpu().numpy() == 0), f"batch {j}"
                for (s0, b0), (s1, b1) in zip(alone[j], outputs(B)):
                    np.testing.assert_array_equal(s1, s0)
                    np.testing.assert_array_equal(b1, b0)
    finally:
        for B in batches:
            B["batch"].close()
