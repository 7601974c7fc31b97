"""Scheduling of the search stage for uneven batches, the tuner and CUDA graph
replay: every schedule gives bit-identical plans, equal to the oracle's FP32
search on the same node costs.

The batch mixes short and long requests with K in {128, 256, 512}, so a small
heavy threshold splits it into one cluster launch per cluster size (2, 4 and 8
CTAs) beside the one-CTA launch of the rest.
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_util import TAU_POS, TAU_ROT, dev, params_pair, run_mask, run_plan, torch
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu

SHAPES = [(40, 128), (300, 512), (60, 256), (200, 512), (80, 128), (250, 256), (30, 512),
          (120, 128), (300, 256), (45, 512), (150, 128), (90, 256), (260, 512), (35, 128)]


def workload(r, T, K):
    return synth.Workload(f"sched_r{r}", 7, T, K, 0.05, 0.25, 0.05, 20, 1e-3,
                          arm_seed=100 + (r % 8), path_seed=5100 + r, cand_seed=5200 + r)


@pytest.fixture(scope="module")
def batch_setup():
    tt = torch()
    pbs = [problems.build(workload(r, T, K)) for r, (T, K) in enumerate(SHAPES)]
    _, cp = params_pair(lm_iters=20)
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
    stream = tt.cuda.Stream()
    batch = cppflow.Batch(robots, cp, descs, ws, st, stream)
    return dict(pbs=pbs, cp=cp, robots=robots, bufs=bufs, descs=descs, ws=ws, st=st,
                stream=stream, batch=batch)


def clear(S):
    for b in S["bufs"]:
        for k in ("sel", "q", "err", "best"):
            b[k].fill_(-7)
        b["rep"].zero_()
    S["st"].zero_()


def results(S):
    torch().cuda.synchronize()
    assert np.all(S["st"].cpu().numpy() == 0)
    return [dict(sel=b["sel"].cpu().numpy(), best=b["best"].cpu().numpy(), q=b["q"].cpu().numpy(),
                 err=b["err"].cpu().numpy(), rep=b["rep"].cpu().numpy()) for b in S["bufs"]]


def assert_same(a, b):
    for x, y in zip(a, b):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k], err_msg=k)


def run_with(S, alpha, cpc=0):
    clear(S)
    S["batch"].set_split(alpha, cpc, S["stream"])
    S["batch"].run(cppflow.STAGE_ALL, S["stream"])
    S["stream"].synchronize()
    return results(S)


def test_every_split_gives_the_same_plans_as_the_oracle(batch_setup):
    S = batch_setup
    base = run_with(S, 0.0)
    assert S["batch"].launches(cppflow.STAGE_DP_FORWARD) == 1
    # the oracle's FP32 search on the GPU's node costs, and valid refined plans
    for r, pb in enumerate(S["pbs"]):
        g = run_mask(S["robots"][r], S["cp"], pb.cand, pb.targets, pb.K)
        ref = oracle.dp_f32(pb.cand, g.pen, pb.K)
        np.testing.assert_array_equal(base[r]["sel"], ref["sel"])
        assert float(base[r]["best"][0]) == float(ref["best"])
        rep = cppflow.report_from_bytes(base[r]["rep"].tobytes())
        assert rep["valid"] == 1 and rep["max_pos"] <= TAU_POS and rep["max_rot"] <= TAU_ROT
    # a small threshold: one cluster launch per cluster size (2, 4, 8 CTAs), no one-CTA launch
    split = run_with(S, 0.01)
    assert S["batch"].launches(cppflow.STAGE_DP_FORWARD) == 3
    assert_same(split, base)
    # 128 candidates per cluster CTA: K = 256 and K = 512 as clusters of 2 and 4 CTAs,
    # K = 128 (a single CTA's worth) on the one-CTA form
    assert_same(run_with(S, 0.01, 128), base)
    assert S["batch"].launches(cppflow.STAGE_DP_FORWARD) == 3
    # the default threshold (the two K = 512, T = 300 requests and a few more run as clusters)
    assert_same(run_with(S, 2.0), base)
    assert_same(run_with(S, 0.5, 128), base)
    # clusters only for K = 512: K = 256 requests stay one CTA each
    S["batch"].set_cluster_min_kp(512, S["stream"])
    try:
        assert_same(run_with(S, 0.01), base)
        assert S["batch"].launches(cppflow.STAGE_DP_FORWARD) == 2
    finally:
        S["batch"].set_cluster_min_kp(0, S["stream"])


def test_graph_replay_equals_run(batch_setup):
    S = batch_setup
    base = run_with(S, 1.0)
    assert S["batch"].launches(cppflow.STAGE_DP_FORWARD) >= 2   # the fork/join is captured too
    S["batch"].capture(cppflow.STAGE_ALL, S["stream"])
    clear(S)
    torch().cuda.synchronize()
    S["batch"].replay(S["stream"])
    S["stream"].synchronize()
    assert_same(results(S), base)
    clear(S)
    torch().cuda.synchronize()
    for _ in range(3):
        S["batch"].replay(S["stream"])
    S["stream"].synchronize()
    assert_same(results(S), base)
    # the legacy default stream cannot be captured
    rc = cppflow.lib().cpp_batch_capture(S["batch"].handle, cppflow.STAGE_ALL, None)
    assert rc == cppflow.ERR_INVALID_ARG


def test_graph_replay_equals_each_plan_alone(batch_setup):
    """The whole uneven batch under a tuned schedule, captured into one CUDA graph
    (cluster groups on forked streams, the persistent LM grid) and replayed: every
    request's plan equals cpp_plan run on that request alone, bit for bit, and its
    search equals the oracle's FP32 search."""
    S = batch_setup
    S["batch"].tune(None, S["stream"])
    try:
        S["batch"].capture(cppflow.STAGE_ALL, S["stream"])
        clear(S)
        torch().cuda.synchronize()
        S["batch"].replay(S["stream"])
        S["stream"].synchronize()
        got = results(S)
        for r, pb in enumerate(S["pbs"]):
            alone = run_plan(S["robots"][r], S["cp"], pb.cand, pb.targets, pb.K)
            np.testing.assert_array_equal(got[r]["sel"], alone["sel"], err_msg=f"request {r}")
            np.testing.assert_array_equal(got[r]["q"], alone["q"])
            np.testing.assert_array_equal(got[r]["err"], alone["err"])
            assert float(got[r]["best"][0]) == float(alone["best"])
            g = run_mask(S["robots"][r], S["cp"], pb.cand, pb.targets, pb.K)
            np.testing.assert_array_equal(got[r]["sel"], oracle.dp_f32(pb.cand, g.pen, pb.K)["sel"])
    finally:
        S["batch"].set_split(0.0, 0, S["stream"])


def test_tuner_and_its_table(batch_setup, tmp_path):
    S = batch_setup
    table = tmp_path / "tune.txt"
    r1 = S["batch"].tune(str(table), S["stream"])
    assert r1["timed"] >= 2 and r1["from_table"] == 0
    assert r1["dp_ms"] > 0 and r1["dp_ms"] <= r1["dp_ms_unsplit"]
    assert r1["mask_tasks_per_warp"] in (1, 2, 4, 8, 16)
    assert 0 < r1["mask_ms"] <= r1["mask_ms_default"]
    lines = table.read_text().split("\n")
    assert len([x for x in lines if x]) == 1
    key, alpha, cpc, ms, tpw, mk, bud = lines[0].split()
    assert key.startswith("n7_obj0_") and float(alpha) == pytest.approx(r1["alpha"], rel=1e-6)
    assert int(cpc) == r1["cands_per_cta"] and int(tpw) == r1["mask_tasks_per_warp"]
    assert int(mk) == r1["cluster_min_kp"] and int(mk) in (0, 256, 512)
    assert float(bud) == pytest.approx(r1["budget_ms"], rel=1e-6) and float(bud) >= 0
    after = results_after_run(S)
    r2 = S["batch"].tune(str(table), S["stream"])
    assert r2["from_table"] == 1 and r2["timed"] == 0
    assert r2["alpha"] == pytest.approx(r1["alpha"], rel=1e-6) and r2["heavy"] == r1["heavy"]
    assert r2["mask_tasks_per_warp"] == r1["mask_tasks_per_warp"]
    assert r2["cluster_min_kp"] == r1["cluster_min_kp"]
    assert r2["budget_ms"] == pytest.approx(r1["budget_ms"], rel=1e-6)
    assert_same(results_after_run(S), after)
    assert_same(after, run_with(S, 0.0))
    # an entry written before the mask knob existed (four fields): the default
    table.write_text(f"{key} {alpha} {cpc} {ms}\n")
    r3 = S["batch"].tune(str(table), S["stream"])
    assert r3["from_table"] == 1 and r3["mask_tasks_per_warp"] == 4 and r3["cluster_min_kp"] == 0
    assert r3["budget_ms"] == 0
    # an entry with a search-time budget: per-request forms
    table.write_text(f"{key} 0 0 {ms} 4 0 1.0\n")
    r4 = S["batch"].tune(str(table), S["stream"])
    assert r4["from_table"] == 1 and r4["budget_ms"] == pytest.approx(1.0) and r4["heavy"] == 6
    assert_same(results_after_run(S), after)
    S["batch"].set_split(0.0, 0, S["stream"])


@pytest.mark.parametrize("budget", [0.05, 0.3, 1.0, 3.0, 10.0])
def test_budget_schedules_give_the_same_plans(batch_setup, budget):
    """Per-request search forms within a time budget (the serving loop's policy): small
    budgets put every request on clusters of 64 successors per CTA (2, 4 and 8 CTAs),
    1 ms mixes wide clusters of 256 per CTA with them, 3 ms clusters of 128, 10 ms only
    the T = 300, K = 512 request on a wide cluster (estimated 10.2 ms on one CTA). Every schedule gives the same
    plans, bit for bit; a budget <= 0 is refused."""
    S = batch_setup
    base = run_with(S, 0.0)
    groups = {0.05: 3, 0.3: 4, 1.0: 4, 3.0: 3, 10.0: 2}[budget]  # cluster groups + one-CTA
    try:
        clear(S)
        S["batch"].set_budget(budget, S["stream"])
        S["batch"].run(cppflow.STAGE_ALL, S["stream"])
        S["stream"].synchronize()
        assert_same(results(S), base)
        assert S["batch"].launches(cppflow.STAGE_DP_FORWARD) == groups
        rc = cppflow.lib().cpp_batch_set_budget(S["batch"].handle, 0.0, None)
        assert rc == cppflow.ERR_INVALID_ARG
    finally:
        S["batch"].set_split(0.0, 0, S["stream"])


@pytest.mark.parametrize("tpw", [1, 2, 8, 16, 64])
def test_mask_tasks_per_warp_gives_the_same_plans(batch_setup, tpw):
    """Waypoints per warp of the mask stage (tasks of 128 candidates per warp) change
    only the launch shape, never a result."""
    S = batch_setup
    base = run_with(S, 1.0)
    S["batch"].set_mask_tasks(tpw)
    try:
        assert_same(run_with(S, 1.0), base)
    finally:
        S["batch"].set_mask_tasks(0)
    with pytest.raises(cppflow.CppflowError):
        S["batch"].set_mask_tasks(65)


def results_after_run(S):
    clear(S)
    S["batch"].run(cppflow.STAGE_ALL, S["stream"])
    S["stream"].synchronize()
    return results(S)


WIDE = [(40, 1024), (25, 700), (33, 520), (50, 300), (20, 1000), (31, 128), (3, 1024), (1, 600),
        (28, 800)]


@pytest.mark.parametrize("objective", [0, 1])
def test_wide_clusters_match_the_oracle(objective):
    """The wide cluster form (256 or 512 successors per CTA, only node costs crossing the
    cluster) on a batch with K up to 1024 and ragged tails (Kp not a multiple of the
    tile, so the last CTA of a cluster owns fewer successors), T = 1 and T = 3
    included: indices and costs equal the oracle's FP32 search on the GPU's node costs,
    for both objectives, and equal the one-CTA form bit for bit."""
    tt = torch()
    pbs = [problems.build(workload(900 + r, T, K)) for r, (T, K) in enumerate(WIDE)]
    _, cp = params_pair(lm_iters=10, dp_objective=objective)
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
    stream = tt.cuda.Stream()
    batch = cppflow.Batch(robots, cp, descs, ws, st, stream)
    S = dict(bufs=bufs, st=st, stream=stream, batch=batch)
    try:
        base = run_with(S, 0.0)            # one CTA per request
        for r, pb in enumerate(pbs):
            g = run_mask(robots[r], cp, pb.cand, pb.targets, pb.K)
            ref = oracle.dp_f32(pb.cand, g.pen, pb.K, objective)
            np.testing.assert_array_equal(base[r]["sel"], ref["sel"])
            assert float(base[r]["best"][0]) == float(ref["best"])
        for cpc in (256, 512):
            wide = run_with(S, 1e-9, cpc)
            assert S["batch"].launches(cppflow.STAGE_DP_FORWARD) >= 2
            for r in range(len(pbs)):
                np.testing.assert_array_equal(wide[r]["sel"], base[r]["sel"], err_msg=f"cpc {cpc} r {r}")
                np.testing.assert_array_equal(wide[r]["best"], base[r]["best"])
                np.testing.assert_array_equal(wide[r]["q"], base[r]["q"])
    finally:
        batch.close()
