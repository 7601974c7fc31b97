"""Pins for the oracle's forward kinematics, rotation routines and Jacobian (§II, §III-C).

Each check compares the oracle with something other than its own formula:
textbook closed forms (planar arms, a single DH link), SciPy's rotation
routines, rigid-motion invariants, and central finite differences.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2309_09102_gb300 import synth

RNG = np.random.default_rng(1234)


def planar_robot(orc, a, theta0=None):
    n = len(a)
    return orc.make_robot(a, np.zeros(n), np.zeros(n), -np.full(n, 3.0), np.full(n, 3.0), theta0)


def test_planar_closed_form(orc):
    """Planar nR (alpha = d = 0): x = sum a_i cos(sum theta), y = sum a_i sin(...), yaw = sum theta."""
    for n in (2, 3, 5):
        a = RNG.uniform(0.1, 0.5, n)
        th0 = RNG.uniform(-0.3, 0.3, n)
        robot = planar_robot(orc, a, th0)
        for _ in range(20):
            q = RNG.uniform(-2.5, 2.5, n)
            cum = np.cumsum(q + th0)
            R, p = orc.fk(robot, q)
            assert p[0] == pytest.approx(np.sum(a * np.cos(cum)), abs=1e-12)
            assert p[1] == pytest.approx(np.sum(a * np.sin(cum)), abs=1e-12)
            assert p[2] == pytest.approx(0.0, abs=1e-15)
            np.testing.assert_allclose(R, Rotation.from_euler("z", cum[-1]).as_matrix(), atol=1e-12)


def test_single_link_closed_form(orc):
    """One standard DH link: p = (a cos t, a sin t, d), R = Rz(t) Rx(alpha) (SciPy intrinsic ZX)."""
    for _ in range(30):
        a, d = RNG.uniform(-0.5, 0.5, 2)
        al = RNG.choice([0.0, math.pi / 2, -math.pi / 2, RNG.uniform(-3, 3)])
        t = RNG.uniform(-3, 3)
        robot = orc.make_robot([a], [d], [al], [-4.0], [4.0])
        R, p = orc.fk(robot, [t])
        np.testing.assert_allclose(p, [a * math.cos(t), a * math.sin(t), d], atol=1e-14)
        np.testing.assert_allclose(R, Rotation.from_euler("ZX", [t, al]).as_matrix(), atol=1e-14)


def _random_robot(orc, n=7, wrist=False, seed=3):
    arm = synth.draw_arm(seed, n, wrist)
    return orc.make_robot(arm.a, arm.d, arm.alpha, arm.lo, arm.hi), arm


def test_rotation_orthonormal(orc):
    robot, _ = _random_robot(orc)
    for _ in range(50):
        R, _ = orc.fk(robot, RNG.uniform(-2.8, 2.8, 7))
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)


def test_joint_screw_invariant(orc):
    """Turning joint j by delta moves the end effector rigidly about the axis (z_j, o_j):
    p' = o + Rot(z, delta)(p - o), R' = Rot(z, delta) R. Catches index, sign and frame errors."""
    for seed in (3, 4, 5):
        robot, _ = _random_robot(orc, seed=seed)
        for _ in range(10):
            q = RNG.uniform(-2.5, 2.5, 7)
            z, o, R, p = orc.fk_frames(robot, q)
            for j in range(7):
                dlt = RNG.uniform(-1, 1)
                q2 = q.copy()
                q2[j] += dlt
                R2, p2 = orc.fk(robot, q2)
                Rot = Rotation.from_rotvec(dlt * z[j]).as_matrix()
                np.testing.assert_allclose(p2, o[j] + Rot @ (p - o[j]), atol=1e-12)
                np.testing.assert_allclose(R2, Rot @ R, atol=1e-12)


def test_spherical_wrist_center_fixed(orc):
    """With a5 = a6 = d6 = 0 (1-based) the wrist centre (origin after joint 6) does not
    depend on joints 5 and 6, and joint 6 = 0 aligns the axes of joints 5 and 7."""
    robot, arm = _random_robot(orc, n=9, wrist=True, seed=8)
    q = RNG.uniform(-2, 2, 9)
    z, o, _, _ = orc.fk_frames(robot, q)
    for _ in range(10):
        q2 = q.copy()
        q2[4] += RNG.uniform(-1, 1)
        q2[5] += RNG.uniform(-1, 1)
        _, o2, _, _ = orc.fk_frames(robot, q2)
        np.testing.assert_allclose(o2[6], o[6], atol=1e-12)
    q[5] = 0.0
    z, _, _, _ = orc.fk_frames(robot, q)
    assert abs(abs(np.dot(z[4], z[6])) - 1.0) < 1e-12


def test_quaternion_routines_match_scipy(orc):
    for _ in range(100):
        rot = Rotation.random(random_state=int(RNG.integers(1 << 30)))
        x, y, z, w = rot.as_quat()
        np.testing.assert_allclose(orc.quat_to_R([w, x, y, z]), rot.as_matrix(), atol=1e-14)
        q = orc.R_to_quat(rot.as_matrix())
        ref = np.array([w, x, y, z]) * (1.0 if w >= 0 else -1.0)
        np.testing.assert_allclose(q, ref, atol=1e-12)
    # branch coverage: rotations by pi about each axis (trace = -1)
    for ax in np.eye(3):
        M = Rotation.from_rotvec(math.pi * ax).as_matrix()
        np.testing.assert_allclose(orc.quat_to_R(orc.R_to_quat(M)), M, atol=1e-12)


def test_geodesic_angle(orc):
    """Geodesic distance = angle of R1^T R2 (SciPy magnitude); exact for R vs R Rz(eps)."""
    for _ in range(100):
        r1 = Rotation.random(random_state=int(RNG.integers(1 << 30)))
        r2 = Rotation.random(random_state=int(RNG.integers(1 << 30)))
        ref = (r1.inv() * r2).magnitude()
        assert orc.rot_angle(r1.as_matrix(), r2.as_matrix()) == pytest.approx(ref, abs=1e-12)
    R = Rotation.random(random_state=7).as_matrix()
    for eps in (1e-9, 1e-6, math.radians(0.1), 1.0, math.pi - 1e-6, math.pi):
        for axis in "xyz":
            R2 = R @ Rotation.from_euler(axis, eps).as_matrix()
            assert orc.rot_angle(R, R2) == pytest.approx(eps, rel=1e-9, abs=1e-15)


def test_log_rot_matches_scipy(orc):
    for _ in range(200):
        rv = Rotation.random(random_state=int(RNG.integers(1 << 30))).as_rotvec()
        M = Rotation.from_rotvec(rv).as_matrix()
        np.testing.assert_allclose(orc.log_rot(M), rv, atol=1e-10)
    for ang in (1e-12, 1e-8, 1e-6 * 0.9, 1e-5, math.pi - 1e-5, math.pi - 1e-7):
        ax = RNG.normal(size=3)
        ax /= np.linalg.norm(ax)
        M = Rotation.from_rotvec(ang * ax).as_matrix()
        w = orc.log_rot(M)
        np.testing.assert_allclose(w, ang * ax, atol=max(1e-12, 1e-7 * ang) if ang < 3 else 2e-7)


def test_jacobian_matches_central_differences(orc):
    """Geometric Jacobian vs central differences of FK (position, and the world-frame
    rotation vector log(R(q+h) R(q-h)^T) / 2h), h = 1e-6: relative error <= 1e-6."""
    for seed in (3, 4, 9):
        robot, _ = _random_robot(orc, seed=seed)
        for _ in range(5):
            q = RNG.uniform(-2.5, 2.5, 7)
            J = orc.jacobian(robot, q)
            h = 1e-6
            Jfd = np.zeros_like(J)
            for j in range(7):
                qp, qm = q.copy(), q.copy()
                qp[j] += h
                qm[j] -= h
                Rp, pp = orc.fk(robot, qp)
                Rm, pm = orc.fk(robot, qm)
                Jfd[:3, j] = (pp - pm) / (2 * h)
                Jfd[3:, j] = orc.log_rot(Rp @ Rm.T) / (2 * h)
            scale = np.max(np.abs(J))
            assert np.max(np.abs(J - Jfd)) <= 1e-6 * scale


def test_residual_first_order(orc):
    """e(q*) = 0 at the target's own configuration, and e(q* + dq) ~ -J dq to first order."""
    robot, _ = _random_robot(orc, seed=4)
    q = RNG.uniform(-2.5, 2.5, 7)
    t7 = orc.fk_pose(robot, q[None])[0]
    np.testing.assert_allclose(orc.residual(robot, q, t7), 0.0, atol=1e-13)
    dq = RNG.normal(size=7) * 1e-5
    e = orc.residual(robot, q + dq, t7)
    J = orc.jacobian(robot, q)
    np.testing.assert_allclose(e, -J @ dq, atol=1e-9)


def test_fk_pose_round_trip(orc):
    robot, _ = _random_robot(orc, seed=6)
    q = RNG.uniform(-2.5, 2.5, (20, 7))
    poses = orc.fk_pose(robot, q)
    for i in range(20):
        R, p = orc.fk(robot, q[i])
        np.testing.assert_allclose(poses[i, :3], p, atol=0)
        np.testing.assert_allclose(orc.quat_to_R(poses[i, 3:]), R, atol=1e-14)
        assert poses[i, 3] >= 0.0
