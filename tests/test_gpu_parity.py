"""GPU vs oracle parity for every stage of the planner core, through the C ABI.

Bars: FK within 1e-5 m / rad of FP64; masks bit-exact outside a 1e-5 guard band
around the thresholds; search indices and cost bit-exact given the same node
costs; refined trajectories within 1 mm / 0.1 deg and their max joint jump
within 1e-4 rad of the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
import problems
from gpu_util import (FK_TOL, GUARD, JUMP_TOL, TAU_POS, TAU_ROT, dev, params_pair, path_cost_f32,
                      run_dp, run_lm, run_mask, run_plan, torch)
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(2024)


def crob(arm):
    return cppflow.robot_from_arm(arm)


# --------------------------------------------------------------------- FK
@pytest.mark.parametrize("n,wrist", [(7, False), (9, True), (3, False), (12, False)])
def test_fk_batch_matches_oracle(n, wrist):
    tt = torch()
    arm = synth.draw_arm(40 + n, n, wrist)
    orob = problems.oracle_robot(arm)
    N = 1000 + 37  # several blocks and a ragged tail
    q = RNG.uniform(-2.8, 2.8, (N, n)).astype(np.float32)
    R = tt.empty(9, N, dtype=tt.float32, device="cuda:0")
    p = tt.empty(3, N, dtype=tt.float32, device="cuda:0")
    cppflow.fk_batch(crob(arm), dev(q.T.copy()), R, p)
    tt.cuda.synchronize()
    R, p = R.cpu().numpy(), p.cpu().numpy()
    for t in range(0, N, 7):
        Ro, po = oracle.fk(orob, q[t].astype(np.float64))
        assert np.max(np.abs(R[:, t].reshape(3, 3) - Ro)) <= FK_TOL
        assert np.max(np.abs(p[:, t] - po)) <= FK_TOL


def test_fk_pose_f64_matches_oracle():
    tt = torch()
    arm = synth.draw_arm(7, 7)
    orob = problems.oracle_robot(arm)
    q = RNG.uniform(-2.8, 2.8, (333, 7))
    out = tt.empty(333, 7, dtype=tt.float64, device="cuda:0")
    cppflow.fk_pose_f64(crob(arm), dev(q), out)
    tt.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), oracle.fk_pose(orob, q), atol=1e-12)


# --------------------------------------------------------------------- mask
def _mask_compare(pb, **kw):
    op, cp = params_pair(**kw)
    g = run_mask(crob(pb.arm), cp, pb.cand, pb.targets, pb.K)
    m, pen, err = oracle.mask(pb.robot, op, pb.cand, pb.targets, pb.K)
    # errors
    finite = np.isfinite(err[..., 0])
    assert np.all(np.isfinite(g.err[..., 0]) == finite)
    assert np.max(np.abs(g.err[finite] - err[finite])) <= FK_TOL
    # bits outside the guard band
    near_tau = (np.abs(err[..., 0] - op.tau_pos) <= GUARD) | (np.abs(err[..., 1] - op.tau_rot) <= GUARD)
    ok = ~near_tau
    np.testing.assert_array_equal(g.mask[ok], m[ok])
    np.testing.assert_array_equal(g.pen[ok], pen[ok])
    # limit bits never depend on the guard band
    lim = np.uint8(cppflow.MASK_OUT | cppflow.MASK_NEAR | cppflow.MASK_NONFINITE | cppflow.MASK_PAD)
    np.testing.assert_array_equal(g.mask & lim, m & lim)
    return g, m, near_tau.sum()


@pytest.mark.parametrize("T,K,n,wrist", [(12, 40, 7, False), (9, 130, 9, True), (5, 33, 3, False),
                                         (4, 70, 12, False), (3, 1, 7, False)])
def test_mask_matches_oracle(T, K, n, wrist):
    pb = problems.small(T=T, K=K, n=n, wrist=wrist, seed=T * 100 + K)
    _mask_compare(pb)                                          # 1 mm / 0.1 deg: almost all POSE
    g, m, guarded = _mask_compare(pb, tau_pos=0.05, tau_rot=math.radians(5.0))  # bits vary
    assert guarded <= max(2, m.size // 1000)


@pytest.mark.parametrize("T,K,n,wrist,tau_deg", [(12, 300, 7, False, 5.0), (9, 130, 9, True, 5.0),
                                                  (6, 200, 6, False, 2.0), (4, 70, 12, False, 95.0)])
def test_mask_decides_alike_with_and_without_errors(T, K, n, wrist, tau_deg):
    """The mask stage with an error buffer (cpp_mask returning the pose errors) and without
    one (every plan path) takes the pose decision the same way, from squared distances and
    the geodesic's trace and skew parts, so mask bits and node costs are identical, also at
    a rotation threshold above pi / 2 (the atan2 form of the test)."""
    tt = torch()
    pb = problems.small(T=T, K=K, n=n, wrist=wrist, seed=T * 7 + K)
    _, cp = params_pair(tau_pos=0.05, tau_rot=math.radians(tau_deg))
    Kp = pb.cand.shape[2]
    outs = []
    for want_err in (True, False):
        m = tt.empty(T, Kp, dtype=tt.uint8, device="cuda:0")
        p = tt.empty(T, Kp, dtype=tt.float32, device="cuda:0")
        e = tt.empty(T, Kp, 2, dtype=tt.float32, device="cuda:0") if want_err else None
        cppflow.mask(crob(pb.arm), cp, dev(pb.cand), dev(pb.targets), pb.K, m, p, e)
        tt.cuda.synchronize()
        outs.append((m.cpu().numpy(), p.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    pose = (outs[0][0] & np.uint8(cppflow.MASK_POSE)) != 0
    assert pose.any() and not pose.all()  # the thresholds split the candidates


def test_mask_nonfinite_and_padding():
    pb = problems.small(T=4, K=30, seed=5)
    cand = pb.cand.copy()
    cand[1, 2, 3] = np.nan
    cand[2, 0, 7] = np.inf
    op, cp = params_pair()
    g = run_mask(crob(pb.arm), cp, cand, pb.targets, pb.K)
    assert g.mask[1, 3] == cppflow.MASK_NONFINITE and np.isinf(g.pen[1, 3])
    assert g.mask[2, 7] == cppflow.MASK_NONFINITE and np.isinf(g.pen[2, 7])
    assert np.all(g.mask[:, pb.K:] == cppflow.MASK_PAD) and np.all(np.isinf(g.pen[:, pb.K:]))
    assert np.all(np.isnan(g.err[:, pb.K:]))


# --------------------------------------------------------------------- search
@pytest.mark.parametrize("T,K,n,wrist", [(50, 32, 7, False), (20, 100, 7, False), (7, 1, 7, False),
                                         (2, 5, 7, False), (15, 257, 7, False), (11, 600, 9, True),
                                         (6, 45, 6, False), (8, 50, 3, False), (5, 1200, 7, False),
                                         (1, 9, 7, False)])
def test_dp_matches_oracle_bit_exact(T, K, n, wrist):
    """The GPU search fed the GPU's own node costs returns the oracle's FP32 indices and cost."""
    pb = problems.small(T=T, K=K, n=n, wrist=wrist, seed=3 * T + K)
    op, cp = params_pair(tau_pos=0.05, tau_rot=math.radians(5.0))
    g = run_mask(crob(pb.arm), cp, pb.cand, pb.targets, pb.K)
    got = run_dp(pb.cand, g.pen, pb.K)
    ref = oracle.dp_f32(pb.cand, g.pen, pb.K)
    np.testing.assert_array_equal(got["sel"], ref["sel"])
    assert got["best"] == ref["best"]
    assert got["status"] == 0
    np.testing.assert_array_equal(got["seed"], pb.cand[np.arange(T), :, ref["sel"]])


def test_dp_ties_and_infeasible():
    T, K, n = 6, 40, 7
    base = RNG.normal(0, 0.2, (T, n, 20)).astype(np.float32)
    cand = np.zeros((T, n, 40), np.float32)
    cand[:, :, :20] = base
    cand[:, :, 20:] = base
    pen = np.zeros((T, 40), np.float32)
    got = run_dp(cand, pen, K)
    ref = oracle.dp_f32(cand, pen, K)
    assert np.all(got["sel"] < 20)
    np.testing.assert_array_equal(got["sel"], ref["sel"])
    pen[3, :] = np.inf
    got = run_dp(cand, pen, K)
    assert got["status"] == cppflow.ERR_INFEASIBLE and np.isinf(got["best"])
    np.testing.assert_array_equal(got["sel"], oracle.dp_f32(cand, pen, K)["sel"])


# --------------------------------------------------------------------- LM
def test_lm_matches_oracle_plain_workload():
    pb = problems.build(synth.PLAIN)
    op, cp = params_pair(lm_iters=pb.w.lm_iters)
    g = run_mask(crob(pb.arm), cp, pb.cand, pb.targets, pb.K)
    seed = run_dp(pb.cand, g.pen, pb.K)["seed"]
    q_gpu, err_gpu = run_lm(crob(pb.arm), cp, seed, pb.targets)
    q_orc, _, _ = oracle.lm(pb.robot, op, seed.astype(np.float64), pb.targets)
    e_orc, rep_orc = oracle.check(pb.robot, op, q_orc, pb.targets)
    e_gpu, rep_gpu = oracle.check(pb.robot, op, q_gpu.astype(np.float64), pb.targets)
    assert np.max(err_gpu[:, 0]) <= TAU_POS and np.max(err_gpu[:, 1]) <= TAU_ROT
    np.testing.assert_allclose(err_gpu, e_gpu, atol=1e-12)   # device FP64 check == host FP64
    assert rep_orc["n_pose_fail"] == 0 and rep_gpu["n_pose_fail"] == 0
    assert abs(rep_gpu["mjac"] - rep_orc["mjac"]) <= JUMP_TOL
    assert np.max(np.abs(q_gpu - q_orc)) <= 1e-3


def test_lm_fp64_mode_and_free_mask():
    pb = problems.small(T=16, K=32, n=9, wrist=True, seed=77, lm_iters=20)
    op, cp = params_pair(lm_iters=20, lm_fp64=1)
    seed = pb.truth + RNG.normal(0, 0.02, pb.truth.shape)
    q_gpu, err = run_lm(crob(pb.arm), cp, seed.astype(np.float32), pb.targets)
    q_orc, _, _ = oracle.lm(pb.robot, op, seed.astype(np.float32).astype(np.float64), pb.targets)
    assert np.max(err[:, 0]) <= TAU_POS and np.max(err[:, 1]) <= TAU_ROT
    assert np.max(np.abs(q_gpu - q_orc)) <= 1e-4
    mask = synth.wrong_branch_free_mask(9)
    op2, cp2 = params_pair(lm_iters=10, free_mask=mask)
    q2, _ = run_lm(crob(pb.arm), cp2, seed.astype(np.float32), pb.targets)
    np.testing.assert_array_equal(q2[:, :4], seed.astype(np.float32)[:, :4])


# --------------------------------------------------------------------- whole plan
@pytest.mark.parametrize("w", [synth.PLAIN, synth.SINGLE], ids=lambda w: w.name)
def test_plan_matches_oracle(w):
    pb = problems.build(w)
    op, cp = params_pair(lm_iters=w.lm_iters, lambda0=w.lambda0)
    got = run_plan(crob(pb.arm), cp, pb.cand, pb.targets, pb.K)
    g = run_mask(crob(pb.arm), cp, pb.cand, pb.targets, pb.K)
    ref_dp = oracle.dp_f32(pb.cand, g.pen, pb.K)
    np.testing.assert_array_equal(got["sel"], ref_dp["sel"])
    assert got["best"] == ref_dp["best"]
    ref = oracle.plan(pb.robot, op, pb.cand, pb.targets, pb.K)
    assert got["status"] == 0 and ref["status"] == 0
    r = got["report"]
    assert r["valid"] == 1 and ref["report"]["valid"] == 1
    assert r["max_pos"] <= TAU_POS and r["max_rot"] <= TAU_ROT
    assert abs(r["mjac"] - ref["report"]["mjac"]) <= JUMP_TOL
    assert abs(r["sum_linf"] - ref["report"]["sum_linf"]) <= JUMP_TOL * pb.w.T


@pytest.mark.parametrize("count", [6, 24])
def test_batch_equals_alone(count):
    """Requests of different T and K in one batched launch give exactly the results each
    gets alone (same kernels, same inputs), report included. A lone request's FP64 check
    runs as an 8-CTA cluster; a batch of 24 (more clusters than SMs) runs one CTA per
    request with the same summation order."""
    tt = torch()
    base = [(30, 40), (61, 128), (12, 7), (45, 256), (2, 3), (700, 16)]
    shapes = [base[i % len(base)] for i in range(count)]
    pbs = [problems.small(T=T, K=K, seed=500 + i) for i, (T, K) in enumerate(shapes)]
    op, cp = params_pair(lm_iters=10)
    robots = [crob(pb.arm) for pb in pbs]
    keep, descs = [], []
    for r, pb in enumerate(pbs):
        T, n, Kp = pb.cand.shape
        bufs = dict(cand=dev(pb.cand), targets=dev(pb.targets),
                    sel=tt.empty(T, dtype=tt.int32, device="cuda:0"),
                    q=tt.empty(T, n, dtype=tt.float32, device="cuda:0"),
                    err=tt.empty(T, 2, dtype=tt.float64, device="cuda:0"),
                    rep=tt.zeros(cppflow.REPORT_BYTES, dtype=tt.uint8, device="cuda:0"),
                    best=tt.empty(1, dtype=tt.float32, device="cuda:0"))
        keep.append(bufs)
        d = cppflow.PlanDesc(T, pb.K, Kp, r, bufs["cand"].data_ptr(), bufs["targets"].data_ptr(),
                             bufs["sel"].data_ptr(), bufs["q"].data_ptr(), bufs["err"].data_ptr(),
                             bufs["rep"].data_ptr(), bufs["best"].data_ptr())
        descs.append(d)
    ws = tt.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=tt.uint8, device="cuda:0")
    st = tt.zeros(len(descs), dtype=tt.int32, device="cuda:0")
    cppflow.plan_batch(robots, cp, descs, ws, st)
    tt.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    for r, pb in enumerate(pbs):
        alone = run_plan(robots[r], cp, pb.cand, pb.targets, pb.K)
        np.testing.assert_array_equal(keep[r]["sel"].cpu().numpy(), alone["sel"])
        np.testing.assert_array_equal(keep[r]["q"].cpu().numpy(), alone["q"])
        np.testing.assert_array_equal(keep[r]["err"].cpu().numpy(), alone["err"])
        assert float(keep[r]["best"].item()) == float(alone["best"])
        assert cppflow.report_from_bytes(keep[r]["rep"].cpu().numpy().tobytes()) == alone["report"]


@pytest.mark.parametrize("n", [7, 9, 6])
def test_dp_nonfinite_candidates_and_padding(n):
    """NaN / inf candidates (node cost +inf, as the mask gives them) and NaN padding lanes:
    the GPU search ignores NaN terms exactly like the oracle's fmaxf / strict-< scan."""
    T, K, Kp = 9, 70, 96
    rng = np.random.default_rng(n)
    cand = rng.normal(0, 0.3, (T, n, Kp)).astype(np.float32)
    cand[:, :, K:] = np.nan
    pen = np.zeros((T, Kp), np.float32)
    pen[:, K:] = np.inf
    for (i, k, j) in [(2, 5, 0), (4, 0, n - 1), (7, 69, 3), (0, 1, 1)]:
        cand[i, j, k] = np.nan
        pen[i, k] = np.inf
    cand[5, 2, 10] = np.inf
    pen[5, 10] = np.inf
    pen[3, ::3] = 10.0
    got = run_dp(cand, pen, K)
    ref = oracle.dp_f32(cand, pen, K)
    np.testing.assert_array_equal(got["sel"], ref["sel"])
    assert got["best"] == ref["best"]


def test_large_batch_search_kernel_matches_oracle():
    """A batch too large for one wave of clusters (40 requests x 8-CTA clusters > 152 SMs)
    runs the one-CTA-per-request search; each result equals the oracle's FP32 search on the
    GPU's node costs, including requests with non-finite candidates."""
    tt = torch()
    pbs = [problems.small(T=6 + (i % 5), K=400 + 16 * (i % 7), seed=3000 + i) for i in range(40)]
    for i in (3, 17):
        pbs[i].cand[2, 1, 5] = np.nan
    _, cp = params_pair(tau_pos=0.05, tau_rot=math.radians(5.0), lm_iters=5)
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
    for r, pb in enumerate(pbs):
        g = run_mask(robots[r], cp, pb.cand, pb.targets, pb.K)
        ref = oracle.dp_f32(pb.cand, g.pen, pb.K)
        np.testing.assert_array_equal(keep[r]["sel"].cpu().numpy(), ref["sel"])
        assert float(keep[r]["best"].item()) == float(ref["best"])


def test_dp_largest_supported_lattice():
    """The largest Kp the generic search holds in shared memory at n = 7 (3616 nodes per
    layer, K = 3600 with a ragged tail) against the oracle; one lane beyond is refused."""
    T, K, n = 3, 3600, 7
    rng = np.random.default_rng(11)
    cand = rng.normal(0, 0.5, (T, n, 3616)).astype(np.float32)
    pen = np.where(rng.uniform(size=(T, 3616)) < 0.1, np.float32(10), np.float32(0))
    pen[:, K:] = np.inf
    got = run_dp(cand, pen, K)
    ref = oracle.dp_f32(cand, pen, K)
    np.testing.assert_array_equal(got["sel"], ref["sel"])
    assert got["best"] == ref["best"]
    tt = torch()
    too_big = 3648
    ws = tt.empty(cppflow.dp_workspace_size(T, too_big), dtype=tt.uint8, device="cuda:0")
    with pytest.raises(cppflow.CppflowError):
        cppflow.dp_search(dev(np.zeros((T, n, too_big), np.float32)),
                          dev(np.zeros((T, too_big), np.float32)), too_big, ws,
                          tt.empty(T, dtype=tt.int32, device="cuda:0"),
                          tt.empty(1, dtype=tt.float32, device="cuda:0"),
                          tt.empty(T, n, dtype=tt.float32, device="cuda:0"))


def test_full_size_batch_in_the_benchmark_configuration():
    """24 requests of the T = 300, K = 512 workload in one batch -- too many for clusters,
    so the search runs the one-CTA kernel with four successors per thread, as in the
    benchmark. Three sampled requests equal the oracle's FP32 search bit for bit; every
    request's backtracked path costs exactly its reported minimum and its plan is valid."""
    tt = torch()
    base = synth.SINGLE
    ws_ = [synth.Workload(f"fs_{r}", base.n, base.T, base.K, base.sigma, base.p_wb, base.p_out,
                          base.lm_iters, base.lambda0, arm_seed=100 + r % 8, path_seed=7000 + r,
                          cand_seed=9000 + r) for r in range(24)]
    pbs = [problems.build(w) for w in ws_]
    _, cp = params_pair(lm_iters=base.lm_iters, lambda0=base.lambda0)
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
    batch = cppflow.Batch(robots, cp, descs, ws, st)
    assert batch.launches(cppflow.STAGE_DP_FORWARD) == 1      # one launch, no split
    batch.run(cppflow.STAGE_ALL)
    tt.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    for r, pb in enumerate(pbs):
        sel = keep[r]["sel"].cpu().numpy()
        best = float(keep[r]["best"].item())
        g = run_mask(robots[r], cp, pb.cand, pb.targets, pb.K)
        assert float(path_cost_f32(pb.cand, g.pen, pb.K, sel)) == best
        rep = cppflow.report_from_bytes(keep[r]["rep"].cpu().numpy().tobytes())
        assert rep["valid"] == 1, (r, rep)
        if r in (0, 11, 23):
            ref = oracle.dp_f32(pb.cand, g.pen, pb.K)
            np.testing.assert_array_equal(sel, ref["sel"])
            assert best == float(ref["best"])
