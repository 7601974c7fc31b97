"""Pins for the oracle's trajectory-length step (§III-C "Trajectory length", the
differencing residual of the non-stationary objective) and its block-tridiagonal
solver.

The solver is pinned by NumPy's dense solve of the assembled matrix; the step by
the dense least-squares formula built from the explicit differencing matrix, by
the T = 2 closed form, and by invariants (joint means preserved, constant
trajectories fixed, the differencing cost falls, limits hold); the alternation by
its end-to-end effect on the plain workload and by its phase order on a redundant
planar arm, where the order changes q.
"""
import numpy as np
import pytest

import oracle
import problems
from paper_2309_09102_gb300 import synth

RNG = np.random.default_rng(17)


def dense_from_blocks(Dg, Off):
    T, n, _ = Dg.shape
    A = np.zeros((T * n, T * n))
    for i in range(T):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = Dg[i]
        if i + 1 < T:
            A[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = Off[i]
            A[(i + 1) * n:(i + 2) * n, i * n:(i + 1) * n] = Off[i].T
    return A


def random_spd_blocks(T, n):
    Off = RNG.normal(0, 1, (max(T - 1, 1), n, n))
    Dg = np.zeros((T, n, n))
    for i in range(T):
        M = RNG.normal(0, 1, (n, n))
        # Gershgorin: the diagonal block dominates the two coupling blocks
        c = (np.abs(Off[i - 1]).sum() if i > 0 else 0) + (np.abs(Off[i]).sum() if i + 1 < T else 0)
        Dg[i] = M @ M.T + (c + 1.0) * np.eye(n)
    return Dg, Off[:max(T - 1, 0)] if T > 1 else Off


@pytest.mark.parametrize("T,n", [(1, 3), (2, 1), (7, 3), (12, 7), (40, 9)])
def test_block_tridiag_solve_matches_dense(T, n):
    Dg, Off = random_spd_blocks(T, n)
    b = RNG.normal(0, 1, (T, n))
    x, ok = oracle.block_tridiag_solve(Dg, Off, b)
    assert ok
    A = dense_from_blocks(Dg, Off if T > 1 else np.zeros((0, n, n)))
    assert np.all(np.linalg.eigvalsh(A) > 0)
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(A, b.ravel()), rtol=1e-10, atol=1e-12)


def test_block_tridiag_solve_rejects_indefinite():
    Dg = np.stack([np.eye(2), -np.eye(2)])
    _, ok = oracle.block_tridiag_solve(Dg, np.zeros((1, 2, 2)), np.ones((2, 2)))
    assert not ok


def wide_robot(n):
    return oracle.make_robot([0.2] * n, [0.1] * n, [0.0] * n, [-50.0] * n, [50.0] * n)


def dense_diff_step(q, lam):
    """delta = -(D^T D + lam I)^{-1} D^T D q with D the explicit differencing matrix."""
    T, n = q.shape
    D = np.zeros(((T - 1) * n, T * n))
    for i in range(T - 1):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = -np.eye(n)
        D[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] = np.eye(n)
    r = D @ q.ravel()
    delta = -np.linalg.solve(D.T @ D + lam * np.eye(T * n), D.T @ r)
    return (q.ravel() + delta).reshape(T, n)


@pytest.mark.parametrize("T,n,lam", [(2, 1, 0.5), (5, 3, 1.0), (30, 7, 0.1), (30, 7, 10.0)])
def test_diff_step_matches_dense_least_squares(T, n, lam):
    q = RNG.normal(0, 1, (T, n))
    out, ok = oracle.diff_step(wide_robot(n), q, lam)
    assert ok
    np.testing.assert_allclose(out, dense_diff_step(q, lam), rtol=1e-10, atol=1e-12)


def test_diff_step_two_waypoints_closed_form():
    """T = 2, n = 1: the difference r becomes r * lam / (2 + lam), symmetrically."""
    for lam in (0.01, 1.0, 7.5):
        q = np.array([[0.3], [1.1]])
        out, _ = oracle.diff_step(wide_robot(1), q, lam)
        r = 0.8
        assert out[1, 0] - out[0, 0] == pytest.approx(r * lam / (2 + lam), rel=1e-12)
        assert out[0, 0] + out[1, 0] == pytest.approx(1.4, rel=1e-12)


def test_diff_step_invariants():
    T, n = 25, 7
    rob = wide_robot(n)
    q = RNG.normal(0, 1, (T, n))
    fd = lambda x: 0.5 * np.sum(np.diff(x, axis=0) ** 2)
    out, _ = oracle.diff_step(rob, q, 1.0)
    np.testing.assert_allclose(out.mean(axis=0), q.mean(axis=0), atol=1e-12)   # 1^T L = 0
    assert fd(out) < fd(q)
    const = np.tile(RNG.normal(0, 1, n), (T, 1))
    np.testing.assert_array_equal(oracle.diff_step(rob, const, 1.0)[0], const)
    small, _ = oracle.diff_step(rob, q, 100.0)
    assert np.abs(small - q).max() < np.abs(out - q).max()   # more damping, smaller step
    one, _ = oracle.diff_step(rob, q[:1], 1.0)               # T = 1: nothing to difference
    np.testing.assert_array_equal(one, q[:1])


def test_diff_step_clamps_to_limits():
    rob = oracle.make_robot([0.2] * 2, [0.1] * 2, [0.0] * 2, [-1.0] * 2, [1.0] * 2)
    q = np.array([[1.0, -1.0], [-1.0, 1.0], [1.0, -1.0]])
    out, _ = oracle.diff_step(rob, q, 0.05)
    assert np.all(out <= 1.0) and np.all(out >= -1.0)


def test_alternation_on_plain_workload(orc):
    """Pose phases alternating with trajectory-length steps: zero rounds is plain LM;
    with rounds the result stays valid and its differencing cost falls."""
    pb = problems.build(synth.PLAIN)
    out = orc.plan(pb.robot, pb.params, pb.cand, pb.targets, pb.K)
    seed = pb.cand[np.arange(pb.w.T), :, out["sel"]].astype(np.float64)
    q0, _ = oracle.lm_smooth(pb.robot, pb.params, seed, pb.targets, 0, 1.0)
    np.testing.assert_array_equal(q0, oracle.lm(pb.robot, pb.params, seed, pb.targets)[0])
    q3, taken = oracle.lm_smooth(pb.robot, pb.params, seed, pb.targets, 3, 1.0)
    assert taken == 3
    _, rep = oracle.check(pb.robot, pb.params, q3, pb.targets)
    assert rep["valid"] == 1
    fd = lambda x: 0.5 * np.sum(np.diff(x, axis=0) ** 2)
    assert fd(q3) < fd(q0)
    # a phase that leaves a waypoint outside tau takes no trajectory-length step
    tight = oracle.make_params(tau_pos=1e-12, tau_rot=1e-12)
    _, none = oracle.lm_smooth(pb.robot, tight, seed, pb.targets, 2, 1.0)
    assert none == 0


def test_alternation_order_on_redundant_planar_arm():
    """§III-C orders the phases: a pose phase first, a trajectory-length step only after a
    pose phase has brought every waypoint within tau, and a pose phase last. On a planar
    4R arm (one redundant joint, every in-plane target reached exactly) the trajectory-length
    steps move the configurations along the redundancy, so the order is visible in q: the
    result equals the phases composed in that order (each phase pinned above on its own)
    and differs from the order that starts with a trajectory-length step."""
    n, T = 4, 6
    rob = oracle.make_robot([0.3, 0.25, 0.2, 0.15], [0.0] * n, [0.0] * n, [-3.0] * n, [3.0] * n)
    P = oracle.make_params(lm_iters=40)
    t = np.linspace(0.0, 1.0, T)[:, None]
    truth = np.array([0.2, 0.5, -0.4, 0.3]) + 0.3 * np.sin(np.pi * t + np.array([0.0, 1.0, 2.0, 3.0]))
    targets = oracle.fk_pose(rob, truth)
    q0 = truth + np.random.default_rng(5).normal(0.0, 0.15, (T, n))
    lam, rounds = 0.5, 2

    def pose(q):
        return oracle.lm(rob, P, q, targets)[0]

    def gated_diff(q):
        _, rep = oracle.check(rob, P, q, targets)
        return oracle.diff_step(rob, q, lam)[0] if rep["n_pose_fail"] == 0 else q

    got, taken = oracle.lm_smooth(rob, P, q0, targets, rounds, lam)
    assert taken == rounds
    q = q0
    for _ in range(rounds):
        q = gated_diff(pose(q))
    np.testing.assert_array_equal(got, pose(q))
    q = q0
    for _ in range(rounds):
        q = pose(oracle.diff_step(rob, q, lam)[0])
    swapped = pose(q)
    assert np.abs(swapped - got).max() > 1e-6
    fd = lambda x: 0.5 * np.sum(np.diff(x, axis=0) ** 2)
    assert fd(got) < fd(pose(q0))
