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
