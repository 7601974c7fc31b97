"""Seeded synthetic inputs for the CppFlow planner core.

This module draws random numbers and assembles arrays; it holds none of the
planner's arithmetic (no forward kinematics, errors, search or optimisation).
Two steps of input construction need the planner's own maths -- the target
path is FK of the true joint trajectory, and a wrong-branch configuration is
re-solved by LM on a subset of joints -- so the caller passes those results in:
the tests build them with the CPU oracle, the benchmark with the CUDA library.

The learned IK generator of the paper (IKFlow, §III-A) is replaced by
"true trajectory + Gaussian noise, with some candidates on a wrong IK branch
and some outside the joint limits", the structure §III-A and §III-B describe:
K plans of T slowly varying configurations, among which the search picks.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator -- value i
of a stream is mix(state + (i + 1) * golden) -- uniform doubles take the top
53 bits, normals use the Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids (one per purpose, so every draw is independent of array sizes)
S_ARM, S_TRUTH, S_NOISE, S_WB, S_OUT, S_OUTJ, S_OUTSIGN, S_OUTMAG, S_MIX, S_GEO = range(1, 11)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_state(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ _mix(np.uint64(stream) * _GOLDEN))
    return np.uint64(s)


def raw_u64(seed: int, stream: int, count: int) -> np.ndarray:
    state = _stream_state(seed, stream)
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(state + idx * _GOLDEN)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Doubles in [0, 1)."""
    return (raw_u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller (one normal per pair of uniforms)."""
    u = uniform(seed, stream, 2 * count).reshape(count, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))  # 1 - u in (0, 1]
    return r * np.cos(2.0 * math.pi * u[:, 1])


# --------------------------------------------------------------------- arms
@dataclass
class Arm:
    """Revolute DH chain: a, d (m), alpha, theta0, lo, hi (rad)."""
    a: np.ndarray
    d: np.ndarray
    alpha: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    theta0: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.theta0 is None:
            self.theta0 = np.zeros_like(self.a)

    @property
    def n(self) -> int:
        return len(self.a)


def draw_arm(seed: int, n: int = 7, wrist: bool = False, limit: float = 2.8) -> Arm:
    """Random arm: a, d ~ U(0.05, 0.4) m, alpha uniform in {0, +pi/2, -pi/2},
    limits +-2.8 rad. With ``wrist`` joints 5-7 (1-based) form a spherical wrist:
    a5 = a6 = d6 = 0, alpha5 = -pi/2, alpha6 = +pi/2."""
    u = uniform(seed, S_ARM, 3 * n).reshape(3, n)
    a = 0.05 + 0.35 * u[0]
    d = 0.05 + 0.35 * u[1]
    choice = np.minimum((u[2] * 3).astype(int), 2)
    alpha = np.array([0.0, math.pi / 2, -math.pi / 2])[choice]
    if wrist:
        assert n >= 7
        a[4] = 0.0
        a[5] = 0.0
        d[5] = 0.0
        alpha[4] = -math.pi / 2
        alpha[5] = math.pi / 2
    return Arm(a=a, d=d, alpha=alpha, lo=np.full(n, -limit), hi=np.full(n, limit))


# --------------------------------------------------------------------- collision model
@dataclass
class Geometry:
    """Collision model of a request (input data only): capsules fixed to DH frames
    (frame 0 = base, j = the frame after joint j) with end points a, b in that frame
    and a radius; the self-collision pairs (capsule indices); cuboid obstacles, each
    the rotation R and centre p of its frame in the world and its half extents."""
    cap_frame: np.ndarray   # [C] int
    cap_a: np.ndarray       # [C][3]
    cap_b: np.ndarray       # [C][3]
    cap_r: np.ndarray       # [C]
    pairs: np.ndarray       # [P][2] int
    box_R: np.ndarray       # [B][3][3]
    box_p: np.ndarray       # [B][3]
    box_half: np.ndarray    # [B][3]


def link_capsules(arm: Arm, radius: float = 0.03, skip: int = 2) -> Geometry:
    """One capsule per link: in frame j (j = 1..n) from the frame's origin to the
    origin of frame j-1, which sits at (-a_j, -d_j sin alpha_j, -d_j cos alpha_j)
    there whatever q_j (the link is rigid). Pairs: capsules at least ``skip``
    links apart (neighbours share a joint and always touch). No obstacles."""
    n = arm.n
    frame = np.arange(1, n + 1)
    a = np.zeros((n, 3))
    b = np.stack([-arm.a, -arm.d * np.sin(arm.alpha), -arm.d * np.cos(arm.alpha)], axis=1)
    pairs = np.array([(u, v) for u in range(n) for v in range(u + skip, n)], dtype=np.int32)
    return Geometry(frame, a, b, np.full(n, radius), pairs.reshape(-1, 2),
                    np.zeros((0, 3, 3)), np.zeros((0, 3)), np.zeros((0, 3)))


def with_boxes(geo: Geometry, seed: int, count: int, reach: tuple = (0.3, 0.9),
               half: tuple = (0.03, 0.12)) -> Geometry:
    """Add ``count`` cuboids: centre at a uniform direction and a distance U(reach)
    from the base, half extents U(half), rotated by U(-pi, pi) about the world z."""
    u = uniform(seed, S_GEO, 7 * count).reshape(count, 7)
    phi = (2 * u[:, 0] - 1) * math.pi
    ct = 2 * u[:, 1] - 1
    az = 2 * math.pi * u[:, 2]
    st = np.sqrt(1 - ct * ct)
    dist = reach[0] + (reach[1] - reach[0]) * u[:, 3]
    p = np.stack([st * np.cos(az), st * np.sin(az), ct], axis=1) * dist[:, None]
    h = half[0] + (half[1] - half[0]) * u[:, 4:7]
    R = np.zeros((count, 3, 3))
    R[:, 0, 0] = np.cos(phi); R[:, 0, 1] = -np.sin(phi)
    R[:, 1, 0] = np.sin(phi); R[:, 1, 1] = np.cos(phi)
    R[:, 2, 2] = 1.0
    return Geometry(geo.cap_frame, geo.cap_a, geo.cap_b, geo.cap_r, geo.pairs,
                    np.concatenate([geo.box_R, R]), np.concatenate([geo.box_p, p]),
                    np.concatenate([geo.box_half, h]))


# --------------------------------------------------------------------- truth
def draw_truth(seed: int, n: int, T: int, wrist: bool = False, max_jump_deg: float = 5.0,
               wrist_amp: float = 0.02) -> np.ndarray:
    """Smooth joint trajectory q_j(t) = c_j + sum_m A_jm sin(2 pi f_jm t + phi_jm),
    t = i / (T - 1): |c_j| <= 2.0, sum_m A_jm <= 0.6, frequencies scaled so the
    largest per-step change is at most ``max_jump_deg``. With ``wrist`` joint 6
    (1-based) stays within ``wrist_amp`` of 0 (a near-singular wrist)."""
    u = uniform(seed, S_TRUTH, n * 11).reshape(n, 11)
    c = -2.0 + 4.0 * u[:, 0]
    total = 0.2 + 0.4 * u[:, 1]
    w = u[:, 2:5] + 0.05
    A = w / w.sum(axis=1, keepdims=True) * total[:, None]
    f = 0.25 + 1.25 * u[:, 5:8]
    phi = 2.0 * math.pi * u[:, 8:11]
    if wrist:
        c[5] = 0.0
        A[5] *= wrist_amp / A[5].sum()
    # derivative bound sum_m A 2 pi f per unit t, i.e. / (T - 1) per step
    bound = (A * 2.0 * math.pi * f).sum(axis=1) / max(T - 1, 1)
    cap = math.radians(max_jump_deg)
    scale = np.minimum(1.0, cap / np.maximum(bound, 1e-300))
    f = f * scale[:, None]
    t = np.arange(T, dtype=np.float64) / max(T - 1, 1)
    q = c[None, :] + (A[None, :, :] * np.sin(2.0 * math.pi * f[None, :, :] * t[:, None, None]
                                              + phi[None, :, :])).sum(axis=2)
    return q  # [T][n] FP64


def wrong_branch_start(truth: np.ndarray, joint: int = 3) -> np.ndarray:
    """Start of the wrong-branch re-solve: joint 4 (1-based) negated. Arms with
    fewer than 5 joints have no wrong branch (the true configuration is returned)."""
    q = truth.copy()
    if q.shape[1] > joint + 1:
        q[:, joint] = -q[:, joint]
    return q


def wrong_branch_free_mask(n: int, first: int = 4) -> int:
    """Joints 5..n (1-based) are re-solved; the others stay fixed (0 if n < 5)."""
    return sum(1 << j for j in range(first, n))


# --------------------------------------------------------------------- candidates
@dataclass
class CandDraws:
    noise: np.ndarray      # [T][K][n] standard normals
    wb: np.ndarray         # [T][K] bool, candidate on the wrong branch
    out: np.ndarray        # [T][K] bool, one joint pushed outside its limits
    out_joint: np.ndarray  # [T][K] int
    out_up: np.ndarray     # [T][K] bool, above the upper limit (else below the lower)
    out_mag: np.ndarray    # [T][K] float, U(0.01, 0.2) beyond the limit


def draw_candidates(seed: int, T: int, K: int, n: int, p_wb: float, p_out: float) -> CandDraws:
    noise = normal(seed, S_NOISE, T * K * n).reshape(T, K, n)
    wb = uniform(seed, S_WB, T * K).reshape(T, K) < p_wb
    out = uniform(seed, S_OUT, T * K).reshape(T, K) < p_out
    oj = np.minimum((uniform(seed, S_OUTJ, T * K) * n).astype(np.int64), n - 1).reshape(T, K)
    up = uniform(seed, S_OUTSIGN, T * K).reshape(T, K) < 0.5
    mag = 0.01 + 0.19 * uniform(seed, S_OUTMAG, T * K).reshape(T, K)
    return CandDraws(noise, wb, out, oj, up, mag)


def draw_candidates_coherent(seed: int, T: int, K: int, n: int, p_wb: float, p_out: float,
                             rho: float = 0.98) -> CandDraws:
    """Lane-coherent draws, shaped like a generative IK model's K motion plans (lane k
    across the waypoints is one plan): the wrong-branch choice is made once per lane,
    and each lane's noise follows an AR(1) walk along the path, e_i = rho e_{i-1} +
    sqrt(1 - rho^2) z_i (standard normal at every waypoint, correlation rho between
    neighbours). Outliers stay independent per candidate."""
    z = normal(seed, S_NOISE, T * K * n).reshape(T, K, n)
    noise = np.empty_like(z)
    noise[0] = z[0]
    c = math.sqrt(1.0 - rho * rho)
    for i in range(1, T):
        noise[i] = rho * noise[i - 1] + c * z[i]
    wb_lane = uniform(seed, S_WB, K) < p_wb
    wb = np.broadcast_to(wb_lane[None, :], (T, K)).copy()
    out = uniform(seed, S_OUT, T * K).reshape(T, K) < p_out
    oj = np.minimum((uniform(seed, S_OUTJ, T * K) * n).astype(np.int64), n - 1).reshape(T, K)
    up = uniform(seed, S_OUTSIGN, T * K).reshape(T, K) < 0.5
    mag = 0.01 + 0.19 * uniform(seed, S_OUTMAG, T * K).reshape(T, K)
    return CandDraws(noise, wb, out, oj, up, mag)


def pad_k(K: int, mult: int = 32) -> int:
    return ((K + mult - 1) // mult) * mult


def assemble(truth: np.ndarray, q_wb: np.ndarray, draws: CandDraws, sigma: float,
             lo: np.ndarray, hi: np.ndarray, Kp: int | None = None) -> np.ndarray:
    """Candidate lattice [T][n][Kp] FP32 (k contiguous): each candidate is the true
    (or the wrong-branch) configuration plus N(0, sigma^2) per joint; an outlier has
    one joint set to limit +- U(0.01, 0.2). Rounded to FP32 once; lanes k >= K are 0."""
    T, K, n = draws.noise.shape
    Kp = pad_k(K) if Kp is None else Kp
    base = np.where(draws.wb[:, :, None], q_wb[:, None, :], truth[:, None, :])
    c = base + sigma * draws.noise
    ti, ki = np.nonzero(draws.out)
    jj = draws.out_joint[ti, ki]
    c[ti, ki, jj] = np.where(draws.out_up[ti, ki], hi[jj] + draws.out_mag[ti, ki],
                             lo[jj] - draws.out_mag[ti, ki])
    lattice = np.zeros((T, n, Kp), np.float32)
    lattice[:, :, :K] = np.transpose(c, (0, 2, 1)).astype(np.float32)
    return lattice


# --------------------------------------------------------------------- workloads
@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    T: int
    K: int
    sigma: float
    p_wb: float
    p_out: float
    lm_iters: int
    lambda0: float = 1e-3
    wrist: bool = False
    arm_seed: int = 1
    path_seed: int = 1
    cand_seed: int = 1


# The five workloads: plain (T50 K32), single request at scale (T300 K512),
# batched uneven launch, serving mix, and the 9-DoF near-singular stress case.
PLAIN = Workload("plain_t50_k32_n7", 7, 50, 32, 0.03, 0.20, 0.0, 10)
SINGLE = Workload("single_t300_k512_n7", 7, 300, 512, 0.05, 0.25, 0.05, 20,
                  arm_seed=2, path_seed=2, cand_seed=2)
STRESS = Workload("stress_t2000_k1024_n9", 9, 2000, 1024, 0.05, 0.25, 0.05, 20, wrist=True,
                  arm_seed=5, path_seed=5, cand_seed=5)


def batched_request(r: int) -> Workload:
    """Request r of the batched uneven launch: arm (r mod 8) of 8 seeded chains,
    T ~ U{50..1000}, K uniform in {128, 256, 512}, seed 3000 + r."""
    u = uniform(3000 + r, S_MIX, 2)
    T = 50 + min(int(u[0] * 951), 950)
    K = (128, 256, 512)[min(int(u[1] * 3), 2)]
    return Workload(f"batched_r{r}", 7, T, K, 0.05, 0.25, 0.05, 20,
                    arm_seed=100 + (r % 8), path_seed=3000 + r, cand_seed=3000 + r)


def serving_request(r: int, seed: int = 4000) -> Workload:
    """Request r of the serving mix: T = floor(exp U(ln 50, ln 2000)),
    K uniform in {128, 256, 512, 1024}, arm (r mod 8)."""
    u = uniform(seed + r, S_MIX, 2)
    T = int(math.floor(math.exp(math.log(50) + u[0] * (math.log(2000) - math.log(50)))))
    T = max(50, min(T, 2000))
    K = (128, 256, 512, 1024)[min(int(u[1] * 4), 3)]
    return Workload(f"serve_r{r}", 7, T, K, 0.05, 0.25, 0.05, 20,
                    arm_seed=100 + (r % 8), path_seed=seed + r, cand_seed=seed + r)


def poisson_arrivals(rate_hz: float, count: int, seed: int = 77) -> np.ndarray:
    """Arrival times (s) of an open-loop Poisson process (seeded exponential gaps)."""
    u = uniform(seed, S_MIX, count)
    return np.cumsum(-np.log1p(-u) / rate_hz)
