"""Pins for the oracle's collision model (§III-B collision cost, §III-C capsule /
cuboid distances).

Segment-segment and segment-box distances are pinned by brute force over dense
grids of the QP's variables (for the box, the exact point-box distance of each
sampled point: clamping a point to an axis-aligned box is the closest box point)
and by closed forms; capsule placement by the independently pinned FK frames;
the mask's collision bit and cost by construction (a box around the whole robot,
an empty model).
"""
import math

import numpy as np
import pytest

import oracle
import problems
from paper_2309_09102_gb300 import synth

RNG = np.random.default_rng(23)


def brute_seg_seg(a1, b1, a2, b2, m=801):
    s = np.linspace(0, 1, m)
    P = a1[None] + s[:, None] * (b1 - a1)[None]
    Q = a2[None] + s[:, None] * (b2 - a2)[None]
    d = ((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)
    return d.min()


def brute_seg_box(a, b, half, m=20001):
    t = np.linspace(0, 1, m)
    X = a[None] + t[:, None] * (b - a)[None]
    C = np.clip(X, -half, half)
    return ((X - C) ** 2).sum(-1).min()


@pytest.mark.parametrize("case", range(40))
def test_seg_seg_matches_brute_force(case):
    a1, b1, a2, b2 = RNG.normal(0, 1, (4, 3))
    if case % 5 == 0:            # nearly parallel
        b2 = a2 + (b1 - a1) + RNG.normal(0, 1e-3, 3)
    if case % 7 == 0:            # degenerate: a point
        b1 = a1.copy()
    d2, s, t = oracle.seg_seg_dist2(a1, b1, a2, b2)
    g = brute_seg_seg(a1, b1, a2, b2)
    assert d2 <= g + 1e-12                          # exact is no worse than any grid point
    assert math.sqrt(g) - math.sqrt(d2) <= 4e-3     # the grid finds it to its resolution
    P, Q = a1 + s * (b1 - a1), a2 + t * (b2 - a2)
    assert ((P - Q) ** 2).sum() == pytest.approx(d2, rel=1e-12, abs=1e-15)
    assert 0 <= s <= 1 and 0 <= t <= 1


def test_seg_seg_closed_forms():
    z = np.zeros(3)
    e = lambda *v: np.array(v, float)
    assert oracle.seg_seg_dist2(z, e(1, 0, 0), e(0.2, 0.5, 0), e(0.7, 0.5, 0))[0] == pytest.approx(0.25)
    assert oracle.seg_seg_dist2(e(-1, 0, 0), e(1, 0, 0), e(0, -1, 0.3), e(0, 1, 0.3))[0] == pytest.approx(0.09)
    assert oracle.seg_seg_dist2(z, e(1, 0, 0), e(2, 0, 0), e(3, 0, 0))[0] == pytest.approx(1.0)
    assert oracle.seg_seg_dist2(z, z, e(0, 3, 4), e(0, 3, 4))[0] == pytest.approx(25.0)
    assert oracle.seg_seg_dist2(z, e(2, 0, 0), e(1, -1, 0), e(1, 1, 0))[0] == 0.0   # crossing


@pytest.mark.parametrize("case", range(40))
def test_seg_box_matches_brute_force(case):
    half = RNG.uniform(0.05, 0.5, 3)
    a, b = RNG.normal(0, 0.8, (2, 3))
    if case % 6 == 0:
        b = a.copy()
    d2, t = oracle.seg_box_dist2(a, b, half)
    g = brute_seg_box(a, b, half)
    assert d2 <= g + 1e-12
    assert math.sqrt(g) - math.sqrt(d2) <= 2e-4
    X = a + t * (b - a)
    assert ((X - np.clip(X, -half, half)) ** 2).sum() == pytest.approx(d2, rel=1e-12, abs=1e-15)


def test_seg_box_closed_forms():
    h = np.array([0.2, 0.2, 0.2])
    e = lambda *v: np.array(v, float)
    assert oracle.seg_box_dist2(e(-1, 0, 0.5), e(1, 0, 0.5), h)[0] == pytest.approx(0.09)
    assert oracle.seg_box_dist2(e(-1, 0, 0), e(1, 0, 0), h)[0] == 0.0             # through it
    assert oracle.seg_box_dist2(e(0.5, 0.5, 0.5), e(0.5, 0.5, 0.5), h)[0] == pytest.approx(3 * 0.09)
    assert oracle.seg_box_dist2(e(1, 1, 0), e(1, 1, 0), h)[0] == pytest.approx(2 * 0.64)


def test_capsules_follow_the_frames():
    """Link capsules of synth.link_capsules run from frame j's origin to frame j-1's
    (oracle.fk_frames, pinned separately), in any configuration."""
    arm = synth.draw_arm(4, 7)
    rob = problems.oracle_robot(arm)
    g = oracle.make_geometry(synth.link_capsules(arm))
    for _ in range(5):
        q = RNG.uniform(-2.5, 2.5, 7)
        z, o, _, _ = oracle.fk_frames(rob, q)
        A, B = oracle.capsules_world(rob, g, q)
        np.testing.assert_allclose(A, o[1:8], atol=1e-12)
        np.testing.assert_allclose(B, o[0:7], atol=1e-12)


def test_clearance_and_mask_collision_bit(orc):
    pb = problems.build(synth.PLAIN)
    geo = synth.link_capsules(pb.arm, radius=0.0)
    # zero radius and no obstacles: clearance = smallest segment distance >= 0
    g0 = oracle.make_geometry(geo)
    sm, em = oracle.clearance(pb.robot, g0, pb.truth[0])
    assert sm >= 0 and em == math.inf
    # an empty model equals the plain mask; a box around the whole robot collides everywhere
    empty = oracle.make_geometry(synth.Geometry(geo.cap_frame[:0], geo.cap_a[:0], geo.cap_b[:0],
                                                geo.cap_r[:0], geo.pairs[:0], np.zeros((0, 3, 3)),
                                                np.zeros((0, 3)), np.zeros((0, 3))))
    ref_m, ref_pen, _ = orc.mask(pb.robot, pb.params, pb.cand, pb.targets, pb.K)
    m, pen, err, cl = oracle.mask_geo(pb.robot, pb.params, empty, 100.0, pb.cand, pb.targets, pb.K)
    np.testing.assert_array_equal(m, ref_m)
    np.testing.assert_array_equal(pen, ref_pen)
    assert np.all(np.isinf(cl[:, :pb.K]))
    big = synth.Geometry(geo.cap_frame, geo.cap_a, geo.cap_b, geo.cap_r + 0.02, geo.pairs[:0],
                         np.eye(3)[None], np.zeros((1, 3)), np.full((1, 3), 5.0))
    m2, pen2, _, cl2 = oracle.mask_geo(pb.robot, pb.params, oracle.make_geometry(big), 100.0,
                                        pb.cand, pb.targets, pb.K)
    assert np.all(m2[:, :pb.K] & oracle.COLLIDE)
    np.testing.assert_array_equal(pen2[:, :pb.K], ref_pen[:, :pb.K] + np.float32(100))
    assert np.all(cl2[:, :pb.K] < 0)
    assert np.all(m2[:, pb.K:] == oracle.PAD)


def test_self_collision_of_a_folded_arm():
    """A planar 3-link arm folded back on itself: links 1 and 3 overlap (clearance < 0);
    stretched out they are a full link apart."""
    rob = oracle.make_robot([0.3, 0.3, 0.3], [0, 0, 0], [0, 0, 0], [-3.1] * 3, [3.1] * 3)
    arm = synth.Arm(a=np.array([0.3, 0.3, 0.3]), d=np.zeros(3), alpha=np.zeros(3),
                    lo=np.full(3, -3.1), hi=np.full(3, 3.1))
    g = oracle.make_geometry(synth.link_capsules(arm, radius=0.02))
    sm, _ = oracle.clearance(rob, g, np.array([0.0, 0.0, 0.0]))
    assert sm == pytest.approx(0.3 - 0.04, abs=1e-12)
    sm2, _ = oracle.clearance(rob, g, np.array([0.0, math.pi - 0.2, math.pi - 0.2]))
    assert sm2 < 0


# ------------------------------------------------------------------ collision rows of r_diff
@pytest.mark.parametrize("seed", range(6))
def test_collision_rows_gradients_match_finite_differences(seed):
    arm = synth.draw_arm(4 + seed, 7)
    rob = problems.oracle_robot(arm)
    g = oracle.make_geometry(synth.with_boxes(synth.link_capsules(arm), 3 + seed, 3))
    q = np.random.default_rng(seed).uniform(-2, 2, 7)
    res, J = oracle.collision_rows(rob, g, q, 10.0, 1.5)   # d_safe = 10 m: every row active
    assert len(res) >= 30 and np.all(res > 0)
    h = 1e-6
    for j in range(7):
        e = np.zeros(7)
        e[j] = h
        rp, _ = oracle.collision_rows(rob, g, q + e, 10.0, 1.5)
        rm, _ = oracle.collision_rows(rob, g, q - e, 10.0, 1.5)
        np.testing.assert_allclose((rp - rm) / (2 * h), J[:, j], atol=1e-6)


def test_collision_rows_hinge():
    """Only pairs closer than d_safe contribute, with residual w (d_safe - d)."""
    arm = synth.draw_arm(9, 7)
    rob = problems.oracle_robot(arm)
    g = oracle.make_geometry(synth.link_capsules(arm, radius=0.02))
    q = np.zeros(7)
    sm, _ = oracle.clearance(rob, g, q)
    res, _ = oracle.collision_rows(rob, g, q, sm + 0.01, 2.0)
    assert len(res) >= 1 and res.max() == pytest.approx(2.0 * 0.01, rel=1e-9)
    res0, _ = oracle.collision_rows(rob, g, q, sm - 1e-9, 2.0)
    assert len(res0) == 0


def dense_step_geo(rob, g, q, lam, d_safe, w):
    """One damped Gauss-Newton step on [differences; collision rows] from the explicit
    stacked Jacobian (NumPy dense solve)."""
    T, n = q.shape
    rows, cols = [], []
    for i in range(T - 1):
        Jd = np.zeros((n, T * n))
        Jd[:, i * n:(i + 1) * n] = -np.eye(n)
        Jd[:, (i + 1) * n:(i + 2) * n] = np.eye(n)
        rows.append(Jd)
        cols.append(q[i + 1] - q[i])
    for i in range(T):
        res, J = oracle.collision_rows(rob, g, q[i], d_safe, w)
        if len(res):
            Jc = np.zeros((len(res), T * n))
            Jc[:, i * n:(i + 1) * n] = J
            rows.append(Jc)
            cols.append(res)
    Jt = np.concatenate(rows)
    r = np.concatenate(cols)
    delta = -np.linalg.solve(Jt.T @ Jt + lam * np.eye(T * n), Jt.T @ r)
    return q + delta.reshape(T, n)


def test_diff_step_geo_matches_dense_and_reduces_to_diff_step():
    arm = synth.Arm(a=np.full(7, 0.25), d=np.full(7, 0.1), alpha=np.array([0, 1.57, -1.57, 0, 1.57, -1.57, 0]),
                    lo=np.full(7, -50.0), hi=np.full(7, 50.0))
    rob = problems.oracle_robot(arm)
    g = oracle.make_geometry(synth.with_boxes(synth.link_capsules(arm), 7, 4))
    q = np.random.default_rng(3).uniform(-1.5, 1.5, (12, 7))
    out, ok, rows = oracle.diff_step_geo(rob, g, q, 0.7, 0.5, 1.3)
    assert ok and rows > 0
    np.testing.assert_allclose(out, dense_step_geo(rob, g, q, 0.7, 0.5, 1.3), rtol=1e-9, atol=1e-11)
    # w = 0: the collision rows vanish and the step is the plain trajectory-length step
    out0, _, _ = oracle.diff_step_geo(rob, g, q, 0.7, 0.5, 0.0)
    np.testing.assert_allclose(out0, oracle.diff_step(rob, q, 0.7)[0], rtol=1e-12, atol=1e-14)


def test_diff_steps_push_a_trajectory_out_of_a_box():
    """A trajectory whose middle waypoints graze a box: repeated steps with the
    collision rows (strong weight) raise the smallest clearance along it."""
    arm = synth.draw_arm(12, 7)
    rob = problems.oracle_robot(arm)
    q = synth.draw_truth(5, 7, 20)
    A, B = oracle.capsules_world(rob, oracle.make_geometry(synth.link_capsules(arm)), q[10])
    centre = 0.5 * (A[5] + B[5])
    geo = synth.link_capsules(arm, radius=0.02)
    geo = synth.Geometry(geo.cap_frame, geo.cap_a, geo.cap_b, geo.cap_r, geo.pairs[:0],
                         np.eye(3)[None], centre[None], np.full((1, 3), 0.03))
    g = oracle.make_geometry(geo)
    cl = lambda x: min(oracle.clearance(rob, g, qi)[1] for qi in x)
    before = cl(q)
    assert before < 0
    x = q.copy()
    for _ in range(5):
        x, ok, rows = oracle.diff_step_geo(rob, g, x, 1.0, 0.05, 20.0)
        assert ok
    assert cl(x) > before + 0.01
