"""FP64 CPU oracle for the CppFlow planner core -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It loads ``liboracle_cppflow.so`` (plain C,
built with ``gcc -O2 -ffp-contract=off``) and marshals numpy arrays; every step
of the computation is in ``cppflow_oracle.c``. It shares no code with the CUDA
library: the two meet only through the seeded input arrays.

Paper sections cited below: §II Problem Specification, §III-B Global discrete
search, §III-C Levenberg-Marquardt for trajectory optimization (arXiv 2309.09102).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cppflow_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_cppflow.so")

MAXJ = 16
OUT, NEAR, POSE, NONFINITE, PAD = 1, 2, 4, 8, 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(_SRC[:-2] + ".h")
    ):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
             "-shared", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Robot(C.Structure):
    _fields_ = [("n", C.c_int32), ("pad_", C.c_int32)] + [
        (f, C.c_double * MAXJ) for f in ("a", "d", "alpha", "theta0", "lo", "hi")
    ]


class Params(C.Structure):
    _fields_ = [(f, C.c_double) for f in (
        "tau_pos", "tau_rot", "near_margin", "pen_limit", "pen_pose", "jump_max",
        "lambda0", "lambda_up", "lambda_down", "lambda_min", "lambda_max",
        "freeze_step", "freeze_cost")] + [("lm_iters", C.c_int32), ("free_mask", C.c_uint32)]


MAX_CAPS, MAX_PAIRS, MAX_BOXES = 12, 64, 8
COLLIDE = 32


class Capsule(C.Structure):
    _fields_ = [("frame", C.c_int32), ("pad_", C.c_int32), ("a", C.c_double * 3),
                ("b", C.c_double * 3), ("radius", C.c_double)]


class Cuboid(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("p", C.c_double * 3), ("half", C.c_double * 3)]


class Geometry(C.Structure):
    _fields_ = [("n_caps", C.c_int32), ("n_pairs", C.c_int32), ("n_boxes", C.c_int32),
                ("pad_", C.c_int32), ("caps", Capsule * MAX_CAPS),
                ("pairs", (C.c_int32 * 2) * MAX_PAIRS), ("boxes", Cuboid * MAX_BOXES)]


def make_geometry(geo) -> Geometry:
    """Oracle copy of a collision model (synth.Geometry)."""
    g = Geometry()
    g.n_caps, g.n_pairs, g.n_boxes = len(geo.cap_r), len(geo.pairs), len(geo.box_half)
    assert g.n_caps <= MAX_CAPS and g.n_pairs <= MAX_PAIRS and g.n_boxes <= MAX_BOXES
    for c in range(g.n_caps):
        g.caps[c].frame = int(geo.cap_frame[c])
        g.caps[c].a[:] = [float(x) for x in geo.cap_a[c]]
        g.caps[c].b[:] = [float(x) for x in geo.cap_b[c]]
        g.caps[c].radius = float(geo.cap_r[c])
    for k in range(g.n_pairs):
        g.pairs[k][0], g.pairs[k][1] = int(geo.pairs[k][0]), int(geo.pairs[k][1])
    for o in range(g.n_boxes):
        g.boxes[o].R[:] = [float(x) for x in np.asarray(geo.box_R[o]).ravel()]
        g.boxes[o].p[:] = [float(x) for x in geo.box_p[o]]
        g.boxes[o].half[:] = [float(x) for x in geo.box_half[o]]
    return g


class Report(C.Structure):
    _fields_ = [(f, C.c_double) for f in ("max_pos", "max_rot", "mjac", "sum_linf", "traj_len")] + [
        (f, C.c_int32) for f in ("n_pose_fail", "n_limit_fail", "n_jump_fail", "valid")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        sig = {
            "orc_fk": (None, [P, P, P, P]),
            "orc_fk_frames": (None, [P, P, P, P, P, P]),
            "orc_quat_to_R": (None, [P, P]),
            "orc_R_to_quat": (None, [P, P]),
            "orc_rot_angle": (C.c_double, [P, P]),
            "orc_fk_pose": (None, [P, P, C.c_int64, P]),
            "orc_mask": (None, [P, P, P, P, C.c_int, C.c_int, C.c_int, P, P, P]),
            "orc_dp_f32": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]),
            "orc_dp_f64": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, P]),
            "orc_dp_f32_ex": (C.c_int, [P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]),
            "orc_path_mjac_f32": (C.c_float, [P, C.c_int, C.c_int, C.c_int, P]),
            "orc_log_rot": (None, [P, P]),
            "orc_jacobian": (None, [P, P, P]),
            "orc_residual": (None, [P, P, P, P]),
            "orc_lm": (None, [P, P, P, P, C.c_int, P, P, P]),
            "orc_check": (None, [P, P, P, P, C.c_int, P, P]),
            "orc_plan": (C.c_int, [P, P, P, P, C.c_int, C.c_int, C.c_int, P, P, P, P, P]),
            "orc_block_tridiag_solve": (C.c_int, [C.c_int, C.c_int, P, P, P, P]),
            "orc_diff_step": (C.c_int, [P, P, C.c_int, C.c_double, P]),
            "orc_lm_smooth": (None, [P, P, P, P, C.c_int, C.c_int, C.c_double, P, P]),
            "orc_seg_seg_dist2": (C.c_double, [P, P, P, P, P, P]),
            "orc_seg_box_dist2": (C.c_double, [P, P, P, P]),
            "orc_capsules_world": (None, [P, P, P, P, P]),
            "orc_clearance": (None, [P, P, P, P, P]),
            "orc_mask_geo": (None, [P, P, P, C.c_double, P, P, C.c_int, C.c_int, C.c_int, P, P, P,
                                    P]),
            "orc_lane_mjac_f32": (None, [P, C.c_int, C.c_int, C.c_int, C.c_int, P]),
            "orc_batch_opt": (C.c_int, [P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]),
            "orc_collision_rows": (C.c_int, [P, P, P, C.c_double, C.c_double, P, P, C.c_int]),
            "orc_diff_step_geo": (C.c_int, [P, P, P, C.c_int, C.c_double, C.c_double, C.c_double,
                                            P, P]),
            "orc_lm_smooth_geo": (None, [P, P, P, P, P, C.c_int, C.c_int, C.c_double, C.c_double,
                                         C.c_double, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_robot(a, d, alpha, lo, hi, theta0=None) -> Robot:
    n = len(a)
    assert 1 <= n <= MAXJ
    r = Robot()
    r.n = n
    for name, v in (("a", a), ("d", d), ("alpha", alpha), ("lo", lo), ("hi", hi),
                    ("theta0", np.zeros(n) if theta0 is None else theta0)):
        arr = getattr(r, name)
        for j in range(n):
            arr[j] = float(v[j])
    return r


def make_params(**kw) -> Params:
    """Defaults: 1 mm / 0.1 deg pose threshold (Table I caption), 1.5 deg near-limit
    band and +10 / +100 node costs (§III-B), 7 deg discontinuity bound (§II)."""
    p = Params()
    d = dict(tau_pos=1e-3, tau_rot=math.radians(0.1), near_margin=math.radians(1.5),
             pen_limit=10.0, pen_pose=100.0, jump_max=math.radians(7.0), lambda0=1e-3,
             lambda_up=10.0, lambda_down=10.0, lambda_min=1e-12, lambda_max=1e12,
             freeze_step=1e-10, freeze_cost=1e-13, lm_iters=10, free_mask=0xFFFF)
    d.update(kw)
    for k, v in d.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- §II FK
def fk(robot: Robot, q) -> tuple[np.ndarray, np.ndarray]:
    q = _f64(q)
    R = np.zeros(9)
    p = np.zeros(3)
    lib().orc_fk(C.byref(robot), _p(q), _p(R), _p(p))
    return R.reshape(3, 3), p


def fk_frames(robot: Robot, q):
    q = _f64(q)
    z = np.zeros((MAXJ + 1, 3))
    o = np.zeros((MAXJ + 1, 3))
    R = np.zeros(9)
    p = np.zeros(3)
    lib().orc_fk_frames(C.byref(robot), _p(q), _p(z), _p(o), _p(R), _p(p))
    return z[: robot.n + 1], o[: robot.n + 1], R.reshape(3, 3), p


def fk_pose(robot: Robot, q) -> np.ndarray:
    """FP64 FK of q [N][n] -> poses [N][7] (x, y, z, qw, qx, qy, qz)."""
    q = _f64(q).reshape(-1, robot.n)
    out = np.zeros((q.shape[0], 7))
    lib().orc_fk_pose(C.byref(robot), _p(q), q.shape[0], _p(out))
    return out


def quat_to_R(qwxyz) -> np.ndarray:
    q = _f64(qwxyz)
    R = np.zeros(9)
    lib().orc_quat_to_R(_p(q), _p(R))
    return R.reshape(3, 3)


def R_to_quat(R) -> np.ndarray:
    R = _f64(R).reshape(9)
    q = np.zeros(4)
    lib().orc_R_to_quat(_p(R), _p(q))
    return q


def rot_angle(Rt, R) -> float:
    return lib().orc_rot_angle(_p(_f64(Rt).reshape(9)), _p(_f64(R).reshape(9)))


def log_rot(M) -> np.ndarray:
    w = np.zeros(3)
    lib().orc_log_rot(_p(_f64(M).reshape(9)), _p(w))
    return w


# ---------------------------------------------------------------- §II / §III-B mask
def mask(robot: Robot, params: Params, cand: np.ndarray, targets: np.ndarray, K: int,
         want_err: bool = True):
    cand = np.ascontiguousarray(cand, dtype=np.float32)
    T, n, Kp = cand.shape
    assert n == robot.n
    targets = _f64(targets).reshape(T, 7)
    m = np.zeros((T, Kp), np.uint8)
    pen = np.zeros((T, Kp), np.float32)
    err = np.zeros((T, Kp, 2)) if want_err else None
    lib().orc_mask(C.byref(robot), C.byref(params), _p(cand), _p(targets), T, K, Kp,
                   _p(m), _p(pen), _p(err))
    return m, pen, err


# ---------------------------------------------------------------- §III-B search
def dp_f32(cand: np.ndarray, pen: np.ndarray, K: int, objective: int = 0):
    """objective 0: summed per-step L-inf jump; 1: the paper's min-max (mjac) objective."""
    cand = np.ascontiguousarray(cand, dtype=np.float32)
    T, n, Kp = cand.shape
    pen = np.ascontiguousarray(pen, dtype=np.float32).reshape(T, Kp)
    sel = np.zeros(T, np.int32)
    best = np.zeros(1, np.float32)
    cT = np.zeros(Kp, np.float32)
    bp = np.zeros((T, Kp), np.uint16)
    st = lib().orc_dp_f32_ex(_p(cand), _p(pen), T, K, Kp, n, objective, _p(sel), _p(best),
                             _p(cT), _p(bp))
    return dict(status=st, sel=sel, best=best[0], cost_T=cT, bp=bp)


def path_mjac_f32(cand: np.ndarray, sel) -> float:
    cand = np.ascontiguousarray(cand, dtype=np.float32)
    T, n, Kp = cand.shape
    sel = np.ascontiguousarray(sel, dtype=np.int32)
    return float(lib().orc_path_mjac_f32(_p(cand), T, Kp, n, _p(sel)))


def dp_f64(cand: np.ndarray, pen: np.ndarray, K: int):
    cand = np.ascontiguousarray(cand, dtype=np.float32)
    T, n, Kp = cand.shape
    pen = np.ascontiguousarray(pen, dtype=np.float32).reshape(T, Kp)
    sel = np.zeros(T, np.int32)
    best = np.zeros(1, np.float64)
    st = lib().orc_dp_f64(_p(cand), _p(pen), T, K, Kp, n, _p(sel), _p(best))
    return dict(status=st, sel=sel, best=best[0])


# ---------------------------------------------------------------- §III-C LM
def jacobian(robot: Robot, q) -> np.ndarray:
    J = np.zeros(6 * robot.n)
    lib().orc_jacobian(C.byref(robot), _p(_f64(q)), _p(J))
    return J.reshape(6, robot.n)


def residual(robot: Robot, q, target7) -> np.ndarray:
    e = np.zeros(6)
    lib().orc_residual(C.byref(robot), _p(_f64(q)), _p(_f64(target7)), _p(e))
    return e


def lm(robot: Robot, params: Params, q_in, targets, want_hist: bool = False):
    q_in = _f64(q_in).reshape(-1, robot.n)
    T = q_in.shape[0]
    targets = _f64(targets).reshape(T, 7)
    q_out = np.zeros_like(q_in)
    hist = np.zeros((T, params.lm_iters + 1)) if want_hist else None
    iters = np.zeros(T, np.int32)
    lib().orc_lm(C.byref(robot), C.byref(params), _p(q_in), _p(targets), T, _p(q_out),
                 _p(hist), _p(iters))
    return q_out, hist, iters


# ---------------------------------------------------------------- collision distances
def seg_seg_dist2(a1, b1, a2, b2):
    """(squared distance, s, t) between segments a1-b1 and a2-b2."""
    v = [_f64(x).reshape(3) for x in (a1, b1, a2, b2)]
    s, t = np.zeros(1), np.zeros(1)
    d = lib().orc_seg_seg_dist2(_p(v[0]), _p(v[1]), _p(v[2]), _p(v[3]), _p(s), _p(t))
    return d, float(s[0]), float(t[0])


def seg_box_dist2(a, b, half):
    """(squared distance, t) between segment a-b and the box [-half, half]."""
    v = [_f64(x).reshape(3) for x in (a, b, half)]
    t = np.zeros(1)
    d = lib().orc_seg_box_dist2(_p(v[0]), _p(v[1]), _p(v[2]), _p(t))
    return d, float(t[0])


def capsules_world(robot: Robot, geo: Geometry, q):
    q = _f64(q).reshape(robot.n)
    A = np.zeros((MAX_CAPS, 3))
    B = np.zeros((MAX_CAPS, 3))
    lib().orc_capsules_world(C.byref(robot), C.byref(geo), _p(q), _p(A), _p(B))
    return A[:geo.n_caps], B[:geo.n_caps]


def clearance(robot: Robot, geo: Geometry, q):
    """(smallest self clearance, smallest obstacle clearance) of one configuration."""
    q = _f64(q).reshape(robot.n)
    sm, em = np.zeros(1), np.zeros(1)
    lib().orc_clearance(C.byref(robot), C.byref(geo), _p(q), _p(sm), _p(em))
    return float(sm[0]), float(em[0])


def mask_geo(robot: Robot, params: Params, geo: Geometry, pen_collide: float, cand: np.ndarray,
             targets: np.ndarray, K: int):
    """orc_mask_geo: (mask, pen, err, clearance)."""
    cand = np.ascontiguousarray(cand, np.float32)
    T, n, Kp = cand.shape
    targets = _f64(targets).reshape(T, 7)
    mask = np.zeros((T, Kp), np.uint8)
    pen = np.zeros((T, Kp), np.float32)
    err = np.zeros((T, Kp, 2))
    cl = np.zeros((T, Kp))
    lib().orc_mask_geo(C.byref(robot), C.byref(params), C.byref(geo), float(pen_collide), _p(cand),
                       _p(targets), T, K, Kp, _p(mask), _p(pen), _p(err), _p(cl))
    return mask, pen, err, cl


MAX_ROWS = MAX_PAIRS + MAX_CAPS * MAX_BOXES


def collision_rows(robot: Robot, geo: Geometry, q, d_safe: float, w: float):
    """Hinge residuals w (d_safe - d) of the pairs / capsule-box combinations closer
    than d_safe and their gradient rows: (res [m], J [m][n])."""
    q = _f64(q).reshape(robot.n)
    res = np.zeros(MAX_ROWS)
    J = np.zeros((MAX_ROWS, robot.n))
    m = lib().orc_collision_rows(C.byref(robot), C.byref(geo), _p(q), float(d_safe), float(w),
                                 _p(res), _p(J), MAX_ROWS)
    return res[:m].copy(), J[:m].copy()


def diff_step_geo(robot: Robot, geo: Geometry, q, lambda_d: float, d_safe: float, w: float):
    """Trajectory-length step with collision rows: (q', ok, rows)."""
    q = _f64(q).reshape(-1, robot.n)
    out = np.zeros_like(q)
    rows = np.zeros(1, np.int32)
    ok = lib().orc_diff_step_geo(C.byref(robot), C.byref(geo), _p(q), q.shape[0], float(lambda_d),
                                 float(d_safe), float(w), _p(out), _p(rows))
    return out, bool(ok), int(rows[0])


def lm_smooth_geo(robot: Robot, params: Params, geo: Geometry, q_in, targets, rounds: int,
                  lambda_d: float, d_safe: float, w: float):
    q_in = _f64(q_in).reshape(-1, robot.n)
    T = q_in.shape[0]
    targets = _f64(targets).reshape(T, 7)
    out = np.zeros_like(q_in)
    taken = np.zeros(1, np.int32)
    lib().orc_lm_smooth_geo(C.byref(robot), C.byref(params), C.byref(geo), _p(q_in), _p(targets), T,
                            int(rounds), float(lambda_d), float(d_safe), float(w), _p(out),
                            _p(taken))
    return out, int(taken[0])


# ---------------------------------------------------------------- §III-C trajectory length
def block_tridiag_solve(Dg, Off, b):
    """x = A^{-1} b for the SPD block-tridiagonal A with diagonal blocks Dg [T][n][n] and
    upper blocks Off [T-1][n][n] (block Cholesky). Returns (x, ok)."""
    Dg = _f64(Dg)
    T, n, _ = Dg.shape
    Off = _f64(Off).reshape(max(T - 1, 0), n, n) if T > 1 else np.zeros((1, n, n))
    b = _f64(b).reshape(T, n)
    x = np.zeros((T, n))
    ok = lib().orc_block_tridiag_solve(T, n, _p(Dg), _p(Off), _p(b), _p(x))
    return x, bool(ok)


def diff_step(robot: Robot, q, lambda_d: float):
    """One damped step on the differencing residual, clamped to the limits."""
    q = _f64(q).reshape(-1, robot.n)
    out = np.zeros_like(q)
    ok = lib().orc_diff_step(C.byref(robot), _p(q), q.shape[0], float(lambda_d), _p(out))
    return out, bool(ok)


def lm_smooth(robot: Robot, params: Params, q_in, targets, rounds: int, lambda_d: float):
    """Pose phases alternating with trajectory-length steps; returns (q, steps taken)."""
    q_in = _f64(q_in).reshape(-1, robot.n)
    T = q_in.shape[0]
    targets = _f64(targets).reshape(T, 7)
    out = np.zeros_like(q_in)
    taken = np.zeros(1, np.int32)
    lib().orc_lm_smooth(C.byref(robot), C.byref(params), _p(q_in), _p(targets), T, int(rounds),
                        float(lambda_d), _p(out), _p(taken))
    return out, int(taken[0])


# ---------------------------------------------------------------- cpf-BatchOpt
def lane_mjac_f32(cand: np.ndarray, K: int) -> np.ndarray:
    cand = np.ascontiguousarray(cand, np.float32)
    T, n, Kp = cand.shape
    out = np.zeros(K, np.float32)
    lib().orc_lane_mjac_f32(_p(cand), T, K, Kp, n, _p(out))
    return out


def batch_opt(robot: Robot, params: Params, cand: np.ndarray, targets: np.ndarray, K: int,
              lanes: int = 5):
    """The `lanes` smoothest lanes refined and checked: dict(sel, mjac, q, reports, best)."""
    cand = np.ascontiguousarray(cand, np.float32)
    T, n, Kp = cand.shape
    targets = _f64(targets).reshape(T, 7)
    sel = np.zeros(lanes, np.int32)
    mj = np.zeros(lanes, np.float32)
    q = np.zeros((lanes, T, n))
    reps = (Report * lanes)()
    best = lib().orc_batch_opt(C.byref(robot), C.byref(params), _p(cand), _p(targets), T, K, Kp,
                               lanes, _p(sel), _p(mj), _p(q), C.cast(reps, C.c_void_p))
    return dict(sel=sel, mjac=mj, q=q, reports=[r.as_dict() for r in reps], best=best)


# ---------------------------------------------------------------- §II report
def check(robot: Robot, params: Params, q, targets):
    q = _f64(q).reshape(-1, robot.n)
    T = q.shape[0]
    targets = _f64(targets).reshape(T, 7)
    err = np.zeros((T, 2))
    rep = Report()
    lib().orc_check(C.byref(robot), C.byref(params), _p(q), _p(targets), T, _p(err),
                    C.byref(rep))
    return err, rep.as_dict()


def plan(robot: Robot, params: Params, cand: np.ndarray, targets: np.ndarray, K: int):
    """Whole post-generation pipeline for one request: mask, FP32 search, LM, check."""
    cand = np.ascontiguousarray(cand, dtype=np.float32)
    T, n, Kp = cand.shape
    targets = _f64(targets).reshape(T, 7)
    sel = np.zeros(T, np.int32)
    best = np.zeros(1, np.float32)
    q_out = np.zeros((T, n))
    err = np.zeros((T, 2))
    rep = Report()
    st = lib().orc_plan(C.byref(robot), C.byref(params), _p(cand), _p(targets), T, K, Kp,
                        _p(sel), _p(best), _p(q_out), _p(err), C.byref(rep))
    return dict(status=st, sel=sel, best=best[0], q=q_out, err=err, report=rep.as_dict())
