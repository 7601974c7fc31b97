"""Pins for the oracle's masking (§II joint limits / pose error, §III-B node costs) and
its dynamic-programming search (§III-B).

The search is pinned by brute-force enumeration of all K^T selections on tiny
lattices, summed left to right in FP32 with NumPy scalars; ties by duplicated
candidates; closed forms for K = 1; infeasible and padded lattices.
"""
import itertools
import math

import numpy as np
import pytest

from problems import DEG

RNG = np.random.default_rng(99)
f32 = np.float32


# --------------------------------------------------------------------- masking
def planar(orc, a, lo=-2.8, hi=2.8):
    n = len(a)
    return orc.make_robot(a, np.zeros(n), np.zeros(n), np.full(n, lo), np.full(n, hi))


def lattice_from(qs):
    """qs: list (T) of lists (K) of joint vectors -> [T][n][Kp=32] FP32."""
    T, K, n = len(qs), len(qs[0]), len(qs[0][0])
    c = np.zeros((T, n, 32), np.float32)
    for i in range(T):
        for k in range(K):
            c[i, :, k] = qs[i][k]
    return c


def test_mask_bits_and_costs(orc):
    """Planar 3R with a3 = 0: turning joint 3 changes only the orientation, so the rotation
    error equals the joint offset exactly and the position error is 0."""
    robot = orc.make_robot([0.3, 0.25, 0.0], [0, 0, 0], [0, 0, 0], [-2.8] * 3, [2.8] * 3)
    P = orc.make_params()
    q0 = np.array([0.4, -0.7, 0.2], np.float32).astype(np.float64)  # exact in FP32
    t = orc.fk_pose(robot, q0[None])
    m = 1.5 * DEG
    cases = [
        (q0, 0, 0.0),                                   # exact, inside
        (q0 + [0, 0, 0.05 * DEG], 0, 0.0),              # 0.05 deg: below tau_rot
        (q0 + [0, 0, 0.15 * DEG], 4, 100.0),            # 0.15 deg: POSE
        ([2.8 - m / 2, -0.7, 0.2], 2 | 4, 110.0),       # near upper limit; pose off
        ([-2.9, -0.7, 0.2], 1 | 2 | 4, 110.0),          # outside lower limit
        ([0.4, float("nan"), 0.2], 8, math.inf),        # non-finite
        ([0.4, -0.7, float("inf")], 8, math.inf),
    ]
    cand = lattice_from([[c[0] for c in cases]])
    mask, pen, err = orc.mask(robot, P, cand, t, K=len(cases))
    for k, (_, bits, cost) in enumerate(cases):
        assert mask[0, k] == bits, k
        assert pen[0, k] == f32(cost), k
    assert err[0, 0, 0] == pytest.approx(0.0, abs=1e-15)
    assert err[0, 0, 1] == pytest.approx(0.0, abs=1e-15)
    assert err[0, 1, 0] == pytest.approx(0.0, abs=1e-15)
    dq = float(f32(q0[2] + 0.05 * DEG)) - q0[2]  # the FP32 candidate's actual offset
    assert err[0, 1, 1] == pytest.approx(dq, rel=1e-9)
    assert np.all(mask[0, len(cases):] == orc.PAD)
    assert np.all(np.isinf(pen[0, len(cases):]))


def test_mask_position_error_is_translation(orc):
    """A target translated by v has position error |v| and rotation error 0."""
    robot = planar(orc, [0.3, 0.2, 0.1])
    P = orc.make_params()
    q = np.array([0.3, 0.5, -0.4], np.float32).astype(np.float64)  # exact in FP32
    t = orc.fk_pose(robot, q[None]).copy()
    v = np.array([0.0006, -0.0005, 0.0007])
    t[0, :3] += v
    _, _, err = orc.mask(robot, P, lattice_from([[q]]), t, K=1)
    assert err[0, 0, 0] == pytest.approx(np.linalg.norm(v), rel=1e-9)
    assert err[0, 0, 1] == pytest.approx(0.0, abs=1e-12)


def test_mask_thresholds_are_fp32_rounded(orc):
    """Reading: limit tests compare the FP32 joint value with FP32-rounded thresholds
    (lo + margin formed in FP64, rounded once): equality is inside, one ulp beyond is out."""
    lo, hi = -2.8, 2.8
    robot = planar(orc, [0.3, 0.2], lo, hi)
    P = orc.make_params(tau_pos=10.0, tau_rot=10.0)  # disable the pose bit
    nlo = f32(lo + P.near_margin)
    hi32 = f32(hi)
    qs = [[nlo, 0.0], [np.nextafter(nlo, f32(-10)), 0.0], [hi32, 0.0],
          [np.nextafter(hi32, f32(10)), 0.0]]
    cand = lattice_from([qs])
    t = np.tile([0, 0, 0, 1.0, 0, 0, 0], (1, 1))
    mask, pen, _ = orc.mask(robot, P, cand, t, K=4)
    assert list(mask[0, :4]) == [0, 2, 2, 3]
    assert list(pen[0, :4]) == [0.0, 10.0, 10.0, 10.0]


# --------------------------------------------------------------------- search
def linf32(a, b):
    d = f32(abs(f32(a[0]) - f32(b[0])))
    for j in range(1, len(a)):
        d = max(d, f32(abs(f32(a[j]) - f32(b[j]))))
    return f32(d)


def rel_pen(pen, K):
    """Node costs relative to each waypoint's cheapest node (0 offset if all are +inf)."""
    m = pen[:, :K].min(axis=1)
    m = np.where(np.isinf(m), f32(0), m).astype(np.float32)
    return (pen - m[:, None]).astype(np.float32)


def brute_force(cand, pen, K):
    """All K^T selections; cost summed left to right in FP32 exactly as the search
    associates it: c = r_0; c = (c + jump_i) + r_i with r = relative node cost."""
    T = cand.shape[0]
    r = rel_pen(pen, K)
    best, best_paths, costs = None, [], {}
    for path in itertools.product(range(K), repeat=T):
        c = f32(r[0, path[0]])
        c64 = float(pen[0, path[0]])
        for i in range(1, T):
            d = linf32(cand[i - 1, :, path[i - 1]], cand[i, :, path[i]])
            c = f32(f32(c + d) + r[i, path[i]])
            c64 += float(np.max(np.abs(cand[i - 1, :, path[i - 1]].astype(np.float64)
                                       - cand[i, :, path[i]].astype(np.float64)))) + float(pen[i, path[i]])
        costs[path] = (c, c64)
        if best is None or c < best:
            best, best_paths = c, [path]
        elif c == best:
            best_paths.append(path)
    return best, best_paths, costs


@pytest.mark.parametrize("T,K,n,seed", [(2, 4, 3, 0), (4, 3, 7, 1), (5, 4, 2, 2), (6, 4, 7, 3),
                                        (6, 2, 1, 4), (3, 4, 9, 5)])
def test_dp_equals_brute_force(orc, T, K, n, seed):
    rng = np.random.default_rng(seed)
    Kp = 32
    cand = np.zeros((T, n, Kp), np.float32)
    cand[:, :, :K] = rng.normal(0, 0.3, (T, n, K)).astype(np.float32)
    pen = np.full((T, Kp), np.inf, np.float32)
    pen[:, :K] = rng.choice([0.0, 10.0, 100.0, 110.0], (T, K)).astype(np.float32)
    out = orc.dp_f32(cand, pen, K)
    best, paths, costs = brute_force(cand, pen, K)
    assert out["status"] == 0
    assert out["best"] == best                     # bit-exact min
    assert costs[tuple(out["sel"])][0] == best     # the DP path attains it
    # indices are asserted where the FP64 optimum is unique by > 1e-6
    c64 = sorted(v[1] for v in costs.values())
    if len(c64) > 1 and c64[1] - c64[0] > 1e-6:
        opt = min(costs, key=lambda p: costs[p][1])
        assert tuple(out["sel"]) == opt
        assert tuple(orc.dp_f64(cand, pen, K)["sel"]) == opt


def test_dp_ties_take_lowest_index(orc):
    """Duplicated candidates: every backpointer and the final argmin take the lowest index."""
    rng = np.random.default_rng(7)
    T, K, n = 5, 6, 7
    cand = np.zeros((T, n, 32), np.float32)
    base = rng.normal(0, 0.2, (T, n, 3)).astype(np.float32)
    cand[:, :, 0:3] = base
    cand[:, :, 3:6] = base  # k and k + 3 are identical
    pen = np.zeros((T, 32), np.float32)
    pen[:, K:] = np.inf
    out = orc.dp_f32(cand, pen, K)
    assert np.all(out["sel"] < 3)
    # an all-equal lattice: everything ties, so index 0 everywhere
    cand2 = np.zeros((T, n, 32), np.float32)
    out2 = orc.dp_f32(cand2, pen, K)
    assert np.all(out2["sel"] == 0) and out2["best"] == 0.0


def test_dp_single_candidate_closed_form(orc):
    """K = 1: the only path; every relative node cost is 0, so the cost is the sum of the
    L-inf jumps in FP32 order."""
    rng = np.random.default_rng(3)
    T, n = 9, 7
    cand = np.zeros((T, n, 32), np.float32)
    cand[:, :, 0] = rng.normal(0, 1, (T, n)).astype(np.float32)
    pen = np.full((T, 32), np.inf, np.float32)
    pen[:, 0] = rng.choice([0.0, 10.0], T).astype(np.float32)
    out = orc.dp_f32(cand, pen, 1)
    c = f32(0)
    for i in range(1, T):
        c = f32(f32(c + linf32(cand[i - 1, :, 0], cand[i, :, 0])) + f32(0))
    assert np.all(out["sel"] == 0) and out["best"] == c


def test_dp_infeasible_and_nonfinite(orc):
    rng = np.random.default_rng(5)
    T, K, n = 4, 5, 3
    cand = np.zeros((T, n, 32), np.float32)
    cand[:, :, :K] = rng.normal(0, 0.2, (T, n, K))
    pen = np.zeros((T, 32), np.float32)
    pen[:, K:] = np.inf
    pen[2, :K] = np.inf
    assert orc.dp_f32(cand, pen, K)["status"] == 3
    assert orc.dp_f64(cand, pen, K)["status"] == 3
    # a NaN candidate carries +inf and is never chosen, even when its neighbours are closest
    pen[2, :K] = 0.0
    cand[:, :, 1] = 0.0
    cand[2, 0, 1] = np.nan
    pen[2, 1] = np.inf
    out = orc.dp_f32(cand, pen, K)
    assert out["status"] == 0 and out["sel"][2] != 1


def test_dp_padding_never_selected(orc):
    """Lanes k >= K are outside the lattice, even when their values would be cheapest."""
    T, K, n = 4, 3, 2
    cand = np.ones((T, n, 32), np.float32)
    cand[:, :, :K] = np.arange(T * n * K, dtype=np.float32).reshape(T, n, K)
    cand[:, :, K:] = 0.0
    pen = np.zeros((T, 32), np.float32)
    out = orc.dp_f32(cand, pen, K)
    assert np.all(out["sel"] < K)


def test_dp_f64_twin_agrees_when_separated(orc):
    rng = np.random.default_rng(11)
    T, K, n = 20, 24, 7
    cand = np.zeros((T, n, 32), np.float32)
    cand[:, :, :K] = rng.normal(0, 0.5, (T, n, K))
    pen = np.full((T, 32), np.inf, np.float32)
    pen[:, :K] = 0.0
    a = orc.dp_f32(cand, pen, K)
    b = orc.dp_f64(cand, pen, K)
    assert abs(a["best"] - b["best"]) < 1e-4
    np.testing.assert_array_equal(a["sel"], b["sel"])


# --------------------------------------------------------------------- min-max objective (§III-B)
def brute_force_minmax(cand, pen, K):
    """All K^T selections under the paper's objective: a path costs the max of its per-step
    L-inf jumps and of its relative node costs (max/min are exact: no rounding)."""
    T = cand.shape[0]
    r = rel_pen(pen, K)
    costs = {}
    for path in itertools.product(range(K), repeat=T):
        c = r[0, path[0]]
        for i in range(1, T):
            c = max(c, linf32(cand[i - 1, :, path[i - 1]], cand[i, :, path[i]]), r[i, path[i]])
        costs[path] = f32(c)
    return min(costs.values()), costs


@pytest.mark.parametrize("T,K,n,seed", [(3, 4, 3, 0), (5, 3, 7, 1), (6, 4, 2, 2), (4, 4, 9, 3)])
def test_minmax_dp_equals_brute_force(orc, T, K, n, seed):
    rng = np.random.default_rng(100 + seed)
    cand = np.zeros((T, n, 32), np.float32)
    cand[:, :, :K] = rng.normal(0, 0.4, (T, n, K)).astype(np.float32)
    pen = np.full((T, 32), np.inf, np.float32)
    pen[:, :K] = rng.choice([0.0, 0.0, 10.0, 100.0], (T, K)).astype(np.float32)
    out = orc.dp_f32(cand, pen, K, objective=1)
    best, costs = brute_force_minmax(cand, pen, K)
    assert out["status"] == 0
    assert out["best"] == best
    assert costs[tuple(out["sel"])] == best  # the backtracked path attains it


def test_minmax_closed_forms_and_bottleneck(orc):
    rng = np.random.default_rng(8)
    T, n = 12, 7
    # K = 1: the cost is the largest jump of the only path
    cand = np.zeros((T, n, 32), np.float32)
    cand[:, :, 0] = rng.normal(0, 1, (T, n)).astype(np.float32)
    pen = np.full((T, 32), np.inf, np.float32)
    pen[:, 0] = 0.0
    out = orc.dp_f32(cand, pen, 1, objective=1)
    assert out["best"] == f32(max(linf32(cand[i - 1, :, 0], cand[i, :, 0]) for i in range(1, T)))
    # with no node costs the min-max path's mjac is the smallest of all paths', so at most
    # the min-sum path's; and the reported cost is that path's mjac
    K = 20
    cand = rng.normal(0, 0.3, (T, n, 32)).astype(np.float32)
    pen = np.zeros((T, 32), np.float32)
    pen[:, K:] = np.inf
    mm = orc.dp_f32(cand, pen, K, objective=1)
    ms = orc.dp_f32(cand, pen, K, objective=0)
    assert mm["best"] == f32(orc.path_mjac_f32(cand, mm["sel"]))
    assert orc.path_mjac_f32(cand, mm["sel"]) <= orc.path_mjac_f32(cand, ms["sel"])
    # a node cost of 10 (near a limit) outweighs any revolute jump
    pen[5, :K] = 10.0
    pen[5, 3] = 0.0
    mm2 = orc.dp_f32(cand, pen, K, objective=1)
    assert mm2["sel"][5] == 3 and mm2["best"] < 10.0
