"""GPU parity of collision checking (§III-B collision cost; §III-C capsule and
cuboid distances): cpp_mask_geo against oracle.mask_geo, the search's use of the
collision cost, and a collision model per request in batches and in the server.

Distances are solved in FP32 on the GPU and in FP64 in the oracle, so COLLIDE
bits are compared exactly except where the oracle's clearance lies within
COLL_GUARD of zero (counted), and clearances within COLL_TOL.
"""
import numpy as np
import pytest

import oracle
import problems
from gpu_util import GUARD, dev, params_pair, torch
from paper_2309_09102_gb300 import cppflow, synth

pytestmark = pytest.mark.gpu

COLL_TOL = 1e-5     # m: FP32 frames (~1e-6) and distances against FP64
COLL_GUARD = 1e-5   # m: clearances this close to 0 are excluded from the bit check


def model(pb, boxes=3, radius=0.03, seed=11):
    return synth.with_boxes(synth.link_capsules(pb.arm, radius=radius), seed, boxes)


def gpu_mask_geo(pb, cp, geo):
    tt = torch()
    T, n, Kp = pb.cand.shape
    m = tt.empty(T, Kp, dtype=tt.uint8, device="cuda:0")
    p = tt.empty(T, Kp, dtype=tt.float32, device="cuda:0")
    e = tt.empty(T, Kp, 2, dtype=tt.float32, device="cuda:0")
    c = tt.empty(T, Kp, dtype=tt.float32, device="cuda:0")
    g = cppflow.geometry_from(geo) if geo is not None else None
    cppflow.mask_geo(cppflow.robot_from_arm(pb.arm), cp, g, dev(pb.cand), dev(pb.targets), pb.K,
                     m, p, e, c)
    tt.cuda.synchronize()
    return m.cpu().numpy(), p.cpu().numpy(), e.cpu().numpy(), c.cpu().numpy()


def compare(pb, op, cp, geo):
    gm, gp, ge, gc = gpu_mask_geo(pb, cp, geo)
    om, opn, oe, oc = oracle.mask_geo(pb.robot, op, oracle.make_geometry(geo), cp.pen_collide,
                                      pb.cand, pb.targets, pb.K)
    K = pb.K
    guard_pose = (np.abs(oe[:, :K, 0] - op.tau_pos) < GUARD) | (np.abs(oe[:, :K, 1] - op.tau_rot) < GUARD)
    guard_coll = np.abs(oc[:, :K]) < COLL_GUARD
    ok = ~(guard_pose | guard_coll)
    np.testing.assert_array_equal(gm[:, :K][ok], om[:, :K][ok])
    np.testing.assert_array_equal(gp[:, :K][ok], opn[:, :K][ok])
    np.testing.assert_array_equal(gm[:, K:], om[:, K:])
    fin = np.isfinite(oc[:, :K])
    np.testing.assert_allclose(gc[:, :K][fin], oc[:, :K][fin], rtol=0, atol=COLL_TOL)
    frac = float(np.mean((om[:, :K] & oracle.COLLIDE) > 0))
    return frac, int((~ok).sum())


def test_mask_geo_matches_oracle_plain():
    pb = problems.build(synth.PLAIN)
    op, cp = params_pair()
    frac, guarded = compare(pb, op, cp, model(pb))
    assert 0.02 < frac < 0.5 and guarded <= 5
    # self-collision only, thicker capsules
    frac2, _ = compare(pb, op, cp, model(pb, boxes=0, radius=0.06))
    assert frac2 > 0


def test_mask_geo_matches_oracle_at_scale():
    """The T = 300, K = 512 workload with 4 boxes (150k candidates)."""
    pb = problems.build(synth.SINGLE)
    op, cp = params_pair(lm_iters=20)
    frac, guarded = compare(pb, op, cp, model(pb, boxes=4, seed=5))
    assert frac > 0.01 and guarded <= 50


def test_without_a_model_the_mask_is_unchanged():
    pb = problems.build(synth.PLAIN)
    _, cp = params_pair()
    gm, gp, ge, gc = gpu_mask_geo(pb, cp, None)
    tt = torch()
    T, n, Kp = pb.cand.shape
    m = tt.empty(T, Kp, dtype=tt.uint8, device="cuda:0")
    p = tt.empty(T, Kp, dtype=tt.float32, device="cuda:0")
    cppflow.mask(cppflow.robot_from_arm(pb.arm), cp, dev(pb.cand), dev(pb.targets), pb.K, m, p)
    tt.cuda.synchronize()
    np.testing.assert_array_equal(gm, m.cpu().numpy())
    np.testing.assert_array_equal(gp, p.cpu().numpy())
    assert np.all(np.isinf(gc[:, :pb.K]))


def plan_geo(pb, cp, geo):
    tt = torch()
    T, n, Kp = pb.cand.shape
    ws = tt.empty(cppflow.plan_workspace_size(T, pb.K, Kp, n), dtype=tt.uint8, device="cuda:0")
    out = dict(sel=tt.empty(T, dtype=tt.int32, device="cuda:0"),
               best=tt.empty(1, dtype=tt.float32, device="cuda:0"),
               q=tt.empty(T, n, dtype=tt.float32, device="cuda:0"),
               err=tt.empty(T, 2, dtype=tt.float64, device="cuda:0"),
               rep=tt.zeros(cppflow.REPORT_BYTES, dtype=tt.uint8, device="cuda:0"))
    g = cppflow.geometry_from(geo) if geo is not None else None
    cppflow.plan_geo(cppflow.robot_from_arm(pb.arm), cp, g, dev(pb.cand), dev(pb.targets), pb.K, ws,
                     out["sel"], out["best"], out["q"], out["err"], out["rep"])
    tt.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_search_avoids_colliding_candidates():
    pb = problems.build(synth.PLAIN)
    op, cp = params_pair()
    geo = model(pb, boxes=4, seed=3)
    out = plan_geo(pb, cp, geo)
    gm, gp, _, _ = gpu_mask_geo(pb, cp, geo)
    ref = oracle.dp_f32(pb.cand, gp, pb.K)        # the oracle's search on the GPU's node costs
    np.testing.assert_array_equal(out["sel"], ref["sel"])
    assert float(out["best"][0]) == float(ref["best"])
    T = pb.w.T
    chosen = gm[np.arange(T), out["sel"]]
    free_somewhere = np.any((gm[:, :pb.K] & cppflow.MASK_COLLIDE) == 0, axis=1)
    assert not np.any((chosen & cppflow.MASK_COLLIDE) & free_somewhere)
    # without the model the same lattice picks some colliding candidates
    plain = plan_geo(pb, cp, None)
    assert np.any((gm[np.arange(T), plain["sel"]] & cppflow.MASK_COLLIDE) > 0)


def test_models_per_request_in_batches_and_the_server():
    tt = torch()
    pbs = [problems.build(synth.PLAIN)] + [
        problems.build(synth.Workload(f"cg_{r}", 7, 30 + 10 * r, 64, 0.03, 0.2, 0.05, 10,
                                      arm_seed=50 + r, path_seed=60 + r, cand_seed=70 + r))
        for r in range(2)]
    _, cp = params_pair(lm_iters=10)
    geos = [model(pbs[0], boxes=3), None, model(pbs[2], boxes=2, seed=9)]
    robots = [cppflow.robot_from_arm(pb.arm) for pb in pbs]
    alone = [plan_geo(pb, cp, geos[r]) for r, pb in enumerate(pbs)]
    gstructs = [cppflow.geometry_from(g) if g is not None else None for g in geos]
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
        d = cppflow.PlanDesc(T, pb.K, Kp, r, b["cand"].data_ptr(), b["targets"].data_ptr(),
                             b["sel"].data_ptr(), b["q"].data_ptr(), b["err"].data_ptr(),
                             b["rep"].data_ptr(), b["best"].data_ptr())
        if gstructs[r] is not None:
            d.geometry = cppflow.C.addressof(gstructs[r])
        descs.append(d)
    ws = tt.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=tt.uint8, device="cuda:0")
    st = tt.zeros(len(descs), dtype=tt.int32, device="cuda:0")
    cppflow.plan_batch(robots, cp, descs, ws, st)
    tt.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    for r in range(len(pbs)):
        np.testing.assert_array_equal(bufs[r]["sel"].cpu().numpy(), alone[r]["sel"])
        np.testing.assert_array_equal(bufs[r]["q"].cpu().numpy(), alone[r]["q"])
    with cppflow.Server(cp, hbm_budget=1 << 30) as srv:
        tks = [srv.submit(robots[r], pb.cand, pb.targets, pb.K, geometry=gstructs[r])
               for r, pb in enumerate(pbs)]
        for r, tk in enumerate(tks):
            status, res = srv.wait(tk)
            assert status == cppflow.OK
            np.testing.assert_array_equal(res["sel"], alone[r]["sel"])
            np.testing.assert_array_equal(res["q"], alone[r]["q"])


# ------------------------------------------------------------------ collision rows of r_diff
def near_threshold(orob, g, q, margin, w, eps=1e-4):
    """True if some row's clearance lies within eps of the margin, or some shape pair
    is within eps of touching (the FP32 and FP64 active sets could differ)."""
    for qi in q:
        a, _ = oracle.collision_rows(orob, g, qi, margin - eps, w)
        b, _ = oracle.collision_rows(orob, g, qi, margin + eps, w)
        if len(a) != len(b):
            return True
        sm, em = oracle.clearance(orob, g, qi)
        radii = [g.caps[c].radius for c in range(g.n_caps)]
        if min(sm, em) < -min(radii) + eps:   # closest points (nearly) coincide somewhere
            return True
    return False


def test_smooth_step_geo_matches_oracle():
    """Targets are the FK of the trajectory (the gate is open); a box sits next to the
    trajectory's middle so rows are active at several waypoints."""
    tt = torch()
    n, T = 7, 40
    done = 0
    for seed in range(30):
        arm = synth.draw_arm(30 + seed, n)
        orob = problems.oracle_robot(arm)
        q32 = synth.draw_truth(200 + seed, n, T).astype(np.float32)
        A, B = oracle.capsules_world(orob, oracle.make_geometry(synth.link_capsules(arm)),
                                     q32[T // 2].astype(np.float64))
        geo = synth.link_capsules(arm, radius=0.02)
        axis = B[4] - A[4]
        perp = np.cross(axis, [0.0, 0.0, 1.0])
        if np.linalg.norm(perp) < 1e-3 * np.linalg.norm(axis):
            perp = np.cross(axis, [1.0, 0.0, 0.0])
        centre = 0.5 * (A[4] + B[4]) + 0.07 * perp / np.linalg.norm(perp)   # beside the link
        geo = synth.Geometry(geo.cap_frame, geo.cap_a, geo.cap_b, geo.cap_r, geo.pairs,
                             np.eye(3)[None], centre[None], np.full((1, 3), 0.03))
        g = oracle.make_geometry(geo)
        margin, w, lam = 0.05, 3.0, 1.0
        if near_threshold(orob, g, q32.astype(np.float64), margin, w):
            continue
        ref, ok, rows = oracle.diff_step_geo(orob, g, q32.astype(np.float64), lam, margin, w)
        if rows == 0:
            continue
        _, cp = params_pair(smooth_lambda=lam, coll_margin=margin, coll_weight=w)
        qd = dev(q32)
        ws = tt.empty(cppflow.smooth_workspace_size(T, n), dtype=tt.uint8, device="cuda:0")
        st = tt.zeros(1, dtype=tt.int32, device="cuda:0")
        cppflow.smooth_step_geo(cppflow.robot_from_arm(arm), cp, cppflow.geometry_from(geo), qd,
                                dev(oracle.fk_pose(orob, q32.astype(np.float64))), ws, st)
        tt.cuda.synchronize()
        assert int(st.item()) == 0
        np.testing.assert_allclose(qd.cpu().numpy(), ref, rtol=0, atol=2e-6)
        # without the rows it is the plain step
        ref0, _ = oracle.diff_step(orob, q32.astype(np.float64), lam)
        assert np.abs(ref - ref0).max() > 1e-4
        done += 1
        if done == 3:
            break
    assert done >= 2


def test_alternation_with_collision_rows():
    """Pose phases alternating with collision-aware steps: valid plans whose smallest
    clearance along the path is at least that of the plain alternation; batched equals
    alone."""
    tt = torch()
    pb = problems.build(synth.PLAIN)
    geo = model(pb, boxes=3, radius=0.03, seed=11)
    g = oracle.make_geometry(geo)
    _, cp_plain = params_pair(lm_iters=10, smooth_rounds=3, smooth_lambda=1.0)
    _, cp = params_pair(lm_iters=10, smooth_rounds=3, smooth_lambda=1.0, coll_margin=0.05,
                        coll_weight=5.0)
    out = plan_geo(pb, cp, geo)
    base = plan_geo(pb, cp_plain, geo)   # same search, steps without collision rows
    np.testing.assert_array_equal(out["sel"], base["sel"])
    rep = cppflow.report_from_bytes(out["rep"].tobytes())
    assert rep["valid"] == 1
    cl = lambda q: min(min(oracle.clearance(pb.robot, g, qi)) for qi in q.astype(np.float64))
    assert cl(out["q"]) >= cl(base["q"]) - 1e-6
    # one request with the model and one without, batched
    pb2 = problems.build(synth.Workload("cg_b", 7, 40, 64, 0.03, 0.2, 0.05, 10, arm_seed=77,
                                       path_seed=78, cand_seed=79))
    alone2 = plan_geo(pb2, cp, None)
    robots = [cppflow.robot_from_arm(pb.arm), cppflow.robot_from_arm(pb2.arm)]
    gs = cppflow.geometry_from(geo)
    bufs, descs = [], []
    for r, p_ in enumerate((pb, pb2)):
        T, n, Kp = p_.cand.shape
        b = dict(cand=dev(p_.cand), targets=dev(p_.targets),
                 sel=tt.empty(T, dtype=tt.int32, device="cuda:0"),
                 q=tt.empty(T, n, dtype=tt.float32, device="cuda:0"),
                 err=tt.empty(T, 2, dtype=tt.float64, device="cuda:0"),
                 rep=tt.zeros(cppflow.REPORT_BYTES, dtype=tt.uint8, device="cuda:0"),
                 best=tt.empty(1, dtype=tt.float32, device="cuda:0"))
        bufs.append(b)
        d = cppflow.PlanDesc(T, p_.K, Kp, r, b["cand"].data_ptr(), b["targets"].data_ptr(),
                             b["sel"].data_ptr(), b["q"].data_ptr(), b["err"].data_ptr(),
                             b["rep"].data_ptr(), b["best"].data_ptr())
        if r == 0:
            d.geometry = cppflow.C.addressof(gs)
        descs.append(d)
    ws = tt.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=tt.uint8, device="cuda:0")
    st = tt.zeros(2, dtype=tt.int32, device="cuda:0")
    batch = cppflow.Batch(robots, cp, descs, ws, st)
    assert batch.launches(cppflow.STAGE_LM) == 1 + 3 * 3
    batch.run(cppflow.STAGE_ALL)
    tt.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    np.testing.assert_array_equal(bufs[0]["q"].cpu().numpy(), out["q"])
    np.testing.assert_array_equal(bufs[1]["q"].cpu().numpy(), alone2["q"])
