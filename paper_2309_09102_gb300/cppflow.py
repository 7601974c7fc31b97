"""ctypes binding of the C ABI in ``include/cppflow.h`` (argument marshalling only).

Every call takes torch tensors that already live on the GPU (or raw device
pointers), passes their addresses and the current CUDA stream to the library,
and raises ``CppflowError`` on a non-OK status. All computation happens in the
library's CUDA kernels; if ``libcppflow_gb300.so`` has not been built, ``lib()``
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcppflow_gb300.so")
MAXJ = 16

OK, PENDING, ERR_INVALID_ARG, ERR_INFEASIBLE, ERR_OOM, ERR_BUDGET, ERR_TIMEOUT, ERR_CUDA, \
    ERR_NOT_FOUND, ERR_CANCELLED = range(10)
MASK_OUT, MASK_NEAR, MASK_POSE, MASK_NONFINITE, MASK_PAD = 1, 2, 4, 8, 16
STAGE_MASK, STAGE_LAYER_MIN, STAGE_DP_FORWARD, STAGE_BACKTRACK, STAGE_LM, STAGE_CHECK = \
    1, 2, 4, 8, 16, 32
STAGE_ALL = 63
DP_SUM, DP_MINMAX = 0, 1


class CppflowError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cppflow status {status}: {msg}")
        self.status = status


class Robot(C.Structure):
    _fields_ = [("n", C.c_int32), ("reserved", C.c_int32)] + [
        (f, C.c_double * MAXJ) for f in ("a", "d", "alpha", "theta0", "lo", "hi")]


class Params(C.Structure):
    _fields_ = [(f, C.c_double) for f in (
        "tau_pos", "tau_rot", "near_margin", "pen_limit", "pen_pose", "jump_max", "lambda0",
        "lambda_up", "lambda_down", "lambda_min", "lambda_max", "freeze_step", "freeze_cost")] + [
        ("lm_iters", C.c_int32), ("free_mask", C.c_uint32), ("lm_fp64", C.c_int32),
        ("dp_objective", C.c_int32), ("smooth_rounds", C.c_int32), ("reserved_", C.c_int32),
        ("smooth_lambda", C.c_double), ("pen_collide", C.c_double), ("coll_margin", C.c_double),
        ("coll_weight", C.c_double)]


class Report(C.Structure):
    _fields_ = [(f, C.c_double) for f in ("max_pos", "max_rot", "mjac", "sum_linf", "traj_len")] + [
        (f, C.c_int32) for f in ("n_pose_fail", "n_limit_fail", "n_jump_fail", "valid")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


MAX_CAPSULES, MAX_PAIRS, MAX_BOXES = 12, 64, 8
MASK_COLLIDE = 32


class Capsule(C.Structure):
    _fields_ = [("frame", C.c_int32), ("reserved", C.c_int32), ("a", C.c_double * 3),
                ("b", C.c_double * 3), ("radius", C.c_double)]


class Cuboid(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("p", C.c_double * 3), ("half", C.c_double * 3)]


class Geometry(C.Structure):
    _fields_ = [("n_caps", C.c_int32), ("n_pairs", C.c_int32), ("n_boxes", C.c_int32),
                ("reserved", C.c_int32), ("caps", Capsule * MAX_CAPSULES),
                ("pairs", (C.c_int32 * 2) * MAX_PAIRS), ("boxes", Cuboid * MAX_BOXES)]


def geometry_from(geo) -> Geometry:
    """cpp_geometry_t of a collision model given as arrays (synth.Geometry fields)."""
    g = Geometry()
    g.n_caps, g.n_pairs, g.n_boxes = len(geo.cap_r), len(geo.pairs), len(geo.box_half)
    if g.n_caps > MAX_CAPSULES or g.n_pairs > MAX_PAIRS or g.n_boxes > MAX_BOXES:
        raise ValueError("collision model larger than the library's limits")
    for c in range(g.n_caps):
        g.caps[c].frame = int(geo.cap_frame[c])
        g.caps[c].a[:] = [float(x) for x in geo.cap_a[c]]
        g.caps[c].b[:] = [float(x) for x in geo.cap_b[c]]
        g.caps[c].radius = float(geo.cap_r[c])
    for k in range(g.n_pairs):
        g.pairs[k][0], g.pairs[k][1] = int(geo.pairs[k][0]), int(geo.pairs[k][1])
    for o in range(g.n_boxes):
        g.boxes[o].R[:] = [float(x) for row in geo.box_R[o] for x in row]
        g.boxes[o].p[:] = [float(x) for x in geo.box_p[o]]
        g.boxes[o].half[:] = [float(x) for x in geo.box_half[o]]
    return g


class PlanDesc(C.Structure):
    _fields_ = [("T", C.c_int32), ("K", C.c_int32), ("Kp", C.c_int32), ("robot", C.c_int32),
                ("cand", C.c_void_p), ("targets", C.c_void_p), ("sel", C.c_void_p),
                ("q_out", C.c_void_p), ("pose_err", C.c_void_p), ("report", C.c_void_p),
                ("best_cost", C.c_void_p), ("geometry", C.c_void_p)]


REPORT_BYTES = C.sizeof(Report)
REQ_BORROW = 1
REQ_ANYTIME = 2


class TuneResult(C.Structure):
    _fields_ = [("alpha", C.c_double), ("cands_per_cta", C.c_int32), ("heavy", C.c_int32),
                ("forward_launches", C.c_int32), ("timed", C.c_int32), ("from_table", C.c_int32),
                ("dp_ms", C.c_float), ("dp_ms_unsplit", C.c_float),
                ("mask_tasks_per_warp", C.c_int32), ("mask_ms", C.c_float),
                ("mask_ms_default", C.c_float), ("cluster_min_kp", C.c_int32),
                ("budget_ms", C.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class ServerConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_slots", C.c_int32), ("max_batch", C.c_int32),
                ("max_inflight", C.c_int32), ("hbm_budget_bytes", C.c_size_t),
                ("pinned_bytes", C.c_size_t), ("params", Params), ("latency_requests", C.c_int32),
                ("reserved_", C.c_int32), ("search_budget_ms", C.c_double)]


class PlanReq(C.Structure):
    _fields_ = [("robot", C.c_void_p), ("T", C.c_int32), ("K", C.c_int32), ("Kp", C.c_int32),
                ("flags", C.c_int32), ("cand", C.c_void_p), ("targets", C.c_void_p),
                ("geometry", C.c_void_p), ("anytime_rounds", C.c_int32), ("reserved", C.c_int32)]


class PlanResult(C.Structure):
    _fields_ = [("sel", C.c_void_p), ("q", C.c_void_p), ("pose_err", C.c_void_p),
                ("report", C.c_void_p), ("best_cost", C.c_void_p), ("latency_ms", C.c_double),
                ("dev_status", C.c_int32), ("rounds", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("submitted", "completed", "failed", "cancelled",
                                           "batches", "sum_batch")] + [
        (f, C.c_int32) for f in ("max_batch_seen", "resident", "queued", "reserved")] + [
        ("hbm_used", C.c_size_t), ("hbm_high_water", C.c_size_t)] + [
        (f, C.c_uint64) for f in ("improve_batches", "improve_rounds", "published")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Counters(C.Structure):
    _fields_ = [("lm_waypoints", C.c_uint64), ("lm_iterations", C.c_uint64)]


PROBE_FP32 = 0
PROBE_FP64 = 1

_lib = None
_P = C.c_void_p
_SIGS = {
    "cpp_last_error": (C.c_char_p, []),
    "cpp_status_string": (C.c_char_p, [C.c_int]),
    "cpp_version": (C.c_int32, []),
    "cpp_params_default": (None, [_P]),
    "cpp_fk_batch": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P]),
    "cpp_fk_pose_f64": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "cpp_mask": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, _P, _P]),
    "cpp_dp_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32]),
    "cpp_mask_geo": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P,
                               _P, _P, _P]),
    "cpp_plan_geo": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_size_t,
                               _P, _P, _P, _P, _P, _P, _P]),
    "cpp_mask_range": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P,
                                 _P, _P, _P]),
    "cpp_dp_search_ex": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P,
                                   C.c_size_t, _P, _P, _P, _P, _P, _P]),
    "cpp_dp_search": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, C.c_size_t,
                                _P, _P, _P, _P, _P]),
    "cpp_lm_refine": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P, _P, _P, _P]),
    "cpp_smooth_step": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P, _P]),
    "cpp_smooth_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32]),
    "cpp_smooth_step_geo": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, _P, C.c_size_t, _P, _P]),
    "cpp_check": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P, _P, _P]),
    "cpp_plan_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "cpp_plan": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_size_t,
                           _P, _P, _P, _P, _P, _P, _P]),
    "cpp_batch_opt_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "cpp_batch_opt": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P,
                                C.c_size_t, _P, _P, _P, _P, _P, _P, _P, _P]),
    "cpp_plan_batch_workspace_size": (C.c_size_t, [_P, C.c_int32, _P, C.c_int32]),
    "cpp_plan_batch": (C.c_int, [_P, C.c_int32, _P, _P, C.c_int32, _P, C.c_size_t, _P, _P]),
    "cpp_batch_create": (C.c_int, [_P, C.c_int32, _P, _P, C.c_int32, _P, C.c_size_t, _P, _P,
                                   C.POINTER(C.c_void_p)]),
    "cpp_batch_run": (C.c_int, [_P, C.c_uint32, _P]),
    "cpp_batch_launches": (C.c_int32, [_P, C.c_uint32]),
    "cpp_batch_destroy": (None, [_P]),
    "cpp_batch_set_split": (C.c_int, [_P, C.c_double, C.c_int32, _P]),
    "cpp_batch_set_budget": (C.c_int, [_P, C.c_double, _P]),
    "cpp_batch_set_mask_tasks": (C.c_int, [_P, C.c_int32]),
    "cpp_wait_selftest": (C.c_int, [C.c_int64, C.c_int32, _P, _P]),
    "cpp_batch_set_cluster_min_kp": (C.c_int, [_P, C.c_int32, _P]),
    "cpp_batch_tune": (C.c_int, [_P, C.c_char_p, _P, _P]),
    "cpp_batch_capture": (C.c_int, [_P, C.c_uint32, _P]),
    "cpp_batch_replay": (C.c_int, [_P, _P]),
    "cpp_server_config_default": (None, [_P]),
    "cpp_server_create": (C.c_int, [_P, C.POINTER(C.c_void_p)]),
    "cpp_plan_submit": (C.c_int, [_P, _P, C.POINTER(C.c_uint64)]),
    "cpp_plan_poll": (C.c_int, [_P, C.c_uint64, _P]),
    "cpp_plan_wait": (C.c_int, [_P, C.c_uint64, _P, C.c_int64]),
    "cpp_plan_cancel": (C.c_int, [_P, C.c_uint64]),
    "cpp_plan_peek": (C.c_int, [_P, C.c_uint64, _P]),
    "cpp_server_get_stats": (C.c_int, [_P, _P]),
    "cpp_server_destroy": (None, [_P]),
    "cpp_plan_host_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "cpp_plan_host": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_size_t,
                                _P, _P, _P, _P, _P, _P]),
    "cpp_peak_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, _P, C.POINTER(C.c_double), _P]),
    "cpp_counters_reset": (C.c_int, [_P]),
    "cpp_counters_read": (C.c_int, [_P]),
    "cpp_jacobian_f64": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
}


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().cpp_last_error().decode()


def _check(status: int, what: str):
    if status != OK:
        raise CppflowError(status, f"{what}: {last_error()}")


def ptr(t) -> int | None:
    """Device address of a tensor (None stays NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def stream_handle(stream=None) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


# ------------------------------------------------------------------ structs
def make_robot(a, d, alpha, lo, hi, theta0=None) -> Robot:
    n = len(a)
    if not 1 <= n <= MAXJ:
        raise ValueError(f"n = {n} outside [1, {MAXJ}]")
    r = Robot()
    r.n = n
    th0 = [0.0] * n if theta0 is None else theta0
    for name, v in (("a", a), ("d", d), ("alpha", alpha), ("lo", lo), ("hi", hi), ("theta0", th0)):
        arr = getattr(r, name)
        for j in range(n):
            arr[j] = float(v[j])
    return r


def robot_from_arm(arm) -> Robot:
    return make_robot(arm.a, arm.d, arm.alpha, arm.lo, arm.hi, arm.theta0)


def make_params(**kw) -> Params:
    p = Params()
    lib().cpp_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def wait_selftest(limit_ns: int, cluster_scope: bool, dev_status, stream=None):
    """A bounded device wait that nothing completes: CPP_ERR_TIMEOUT lands in dev_status."""
    _check(lib().cpp_wait_selftest(int(limit_ns), 1 if cluster_scope else 0, ptr(dev_status),
                                   stream_handle(stream)), "cpp_wait_selftest")


# ------------------------------------------------------------------ stage calls
def fk_batch(robot: Robot, q, R, p, stream=None):
    """q [n][N] FP32 -> R [9][N], p [3][N] FP32 (device tensors)."""
    _check(lib().cpp_fk_batch(C.byref(robot), ptr(q), q.shape[-1], ptr(R), ptr(p),
                              stream_handle(stream)), "cpp_fk_batch")


def fk_pose_f64(robot: Robot, q, pose, stream=None):
    """q [N][n] FP64 -> pose [N][7] FP64 (device tensors)."""
    _check(lib().cpp_fk_pose_f64(C.byref(robot), ptr(q), q.numel() // robot.n, ptr(pose),
                                 stream_handle(stream)), "cpp_fk_pose_f64")


def mask(robot: Robot, params: Params, cand, targets, K: int, mask_out, pen, err=None,
         dev_status=None, stream=None):
    T, n, Kp = cand.shape
    _check(lib().cpp_mask(C.byref(robot), C.byref(params), ptr(cand), ptr(targets), T, K, Kp,
                          ptr(mask_out), ptr(pen), ptr(err), ptr(dev_status),
                          stream_handle(stream)), "cpp_mask")


def mask_geo(robot: Robot, params: Params, geometry: Geometry | None, cand, targets, K: int,
             mask_out, pen, err=None, clearance=None, dev_status=None, stream=None):
    """cpp_mask with a collision model (COLLIDE bit, collision cost, clearances)."""
    T, n, Kp = cand.shape
    g = C.byref(geometry) if geometry is not None else None
    _check(lib().cpp_mask_geo(C.byref(robot), C.byref(params), g, ptr(cand), ptr(targets), T, K,
                              Kp, ptr(mask_out), ptr(pen), ptr(err), ptr(clearance),
                              ptr(dev_status), stream_handle(stream)), "cpp_mask_geo")


def mask_range(robot: Robot, params: Params, cand, targets, K: int, k_begin: int, mask_out, pen,
               err=None, dev_status=None, stream=None):
    """cpp_mask on lanes [k_begin, K) only (appended candidates)."""
    T, n, Kp = cand.shape
    _check(lib().cpp_mask_range(C.byref(robot), C.byref(params), ptr(cand), ptr(targets), T, K, Kp,
                                k_begin, ptr(mask_out), ptr(pen), ptr(err), ptr(dev_status),
                                stream_handle(stream)), "cpp_mask_range")


def dp_workspace_size(T: int, Kp: int) -> int:
    return lib().cpp_dp_workspace_size(T, Kp)


def dp_search(cand, pen, K: int, workspace, sel, best_cost, q_seed=None, dev_status=None,
              stream=None, ws_bytes: int | None = None):
    T, n, Kp = cand.shape
    nbytes = ws_bytes if ws_bytes is not None else workspace.numel() * workspace.element_size()
    _check(lib().cpp_dp_search(ptr(cand), ptr(pen), T, K, Kp, n, ptr(workspace), nbytes,
                               ptr(sel), ptr(best_cost), ptr(q_seed), ptr(dev_status),
                               stream_handle(stream)), "cpp_dp_search")


def dp_search_ex(cand, pen, K: int, objective: int, workspace, sel, best_cost, q_seed=None,
                 search_mjac=None, dev_status=None, stream=None):
    T, n, Kp = cand.shape
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().cpp_dp_search_ex(ptr(cand), ptr(pen), T, K, Kp, n, objective, ptr(workspace),
                                  nbytes, ptr(sel), ptr(best_cost), ptr(q_seed), ptr(search_mjac),
                                  ptr(dev_status), stream_handle(stream)), "cpp_dp_search_ex")


def lm_refine(robot: Robot, params: Params, q_in, targets, q_out, pose_err=None, dev_status=None,
              stream=None):
    T = q_in.shape[0]
    _check(lib().cpp_lm_refine(C.byref(robot), C.byref(params), ptr(q_in), ptr(targets), T,
                               ptr(q_out), ptr(pose_err), ptr(dev_status),
                               stream_handle(stream)), "cpp_lm_refine")


def smooth_step(robot: Robot, params: Params, q, targets, dev_status=None, stream=None):
    """One trajectory-length step on q [T][n] FP32 in place (taken only when every
    waypoint is within tau)."""
    T = q.shape[0]
    _check(lib().cpp_smooth_step(C.byref(robot), C.byref(params), ptr(q), ptr(targets), T,
                                 ptr(dev_status), stream_handle(stream)), "cpp_smooth_step")


def smooth_workspace_size(T: int, n: int) -> int:
    return lib().cpp_smooth_workspace_size(T, n)


def smooth_step_geo(robot: Robot, params: Params, geometry: Geometry | None, q, targets, workspace,
                    dev_status=None, stream=None):
    """The trajectory-length step with collision rows, on q [T][n] FP32 in place."""
    T = q.shape[0]
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    g = C.byref(geometry) if geometry is not None else None
    _check(lib().cpp_smooth_step_geo(C.byref(robot), C.byref(params), g, ptr(q), ptr(targets), T,
                                     ptr(workspace), nbytes, ptr(dev_status),
                                     stream_handle(stream)), "cpp_smooth_step_geo")


def check(robot: Robot, params: Params, q, targets, pose_err=None, report=None, stream=None):
    T = q.shape[0]
    _check(lib().cpp_check(C.byref(robot), C.byref(params), ptr(q), ptr(targets), T,
                           ptr(pose_err), ptr(report), stream_handle(stream)), "cpp_check")


def plan_workspace_size(T: int, K: int, Kp: int, n: int) -> int:
    return lib().cpp_plan_workspace_size(T, K, Kp, n)


def plan(robot: Robot, params: Params, cand, targets, K: int, workspace, sel, best_cost, q_out,
         pose_err=None, report=None, dev_status=None, stream=None):
    T, n, Kp = cand.shape
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().cpp_plan(C.byref(robot), C.byref(params), ptr(cand), ptr(targets), T, K, Kp,
                          ptr(workspace), nbytes, ptr(sel), ptr(best_cost), ptr(q_out),
                          ptr(pose_err), ptr(report), ptr(dev_status), stream_handle(stream)),
           "cpp_plan")


def plan_host_workspace_size(T: int, K: int, Kp: int, n: int) -> int:
    return lib().cpp_plan_host_workspace_size(T, K, Kp, n)


def plan_host(robot: Robot, params: Params, cand, targets, K: int, workspace, sel=None,
              best_cost=None, q_out=None, pose_err=None, report=None, stream=None) -> int:
    """cpp_plan_host: HOST numpy inputs cand [T][n][Kp] FP32 and targets [T][7] FP64 (pinned
    memory makes the copies DMA), DEVICE workspace; outputs into HOST numpy arrays (or None,
    report: a Report). Synchronous. Returns the plan's status (OK, INFEASIBLE, TIMEOUT);
    raises for invalid arguments and CUDA failures."""
    T, n, Kp = cand.shape
    nbytes = workspace.numel() * workspace.element_size()
    host = lambda a: None if a is None else a.ctypes.data
    st = lib().cpp_plan_host(C.byref(robot), C.byref(params), host(cand), host(targets), T, K, Kp,
                             ptr(workspace), nbytes, host(sel), host(best_cost), host(q_out),
                             host(pose_err), C.addressof(report) if report is not None else None,
                             stream_handle(stream))
    if st in (OK, ERR_INFEASIBLE, ERR_TIMEOUT):
        return st
    raise CppflowError(st, f"cpp_plan_host: {last_error()}")


def peak_probe(kind: int, blocks_per_sm: int, iters: int, sink, stream=None) -> float:
    """Enqueue one throughput-probe launch; returns the lane operations (FP32) or flops
    (FP64) it performs."""
    ops = C.c_double()
    _check(lib().cpp_peak_probe(kind, blocks_per_sm, int(iters), ptr(sink), C.byref(ops),
                                stream_handle(stream)), "cpp_peak_probe")
    return ops.value


def counters_reset(stream=None):
    _check(lib().cpp_counters_reset(stream_handle(stream)), "cpp_counters_reset")


def counters_read() -> dict:
    c = Counters()
    _check(lib().cpp_counters_read(C.byref(c)), "cpp_counters_read")
    return {"lm_waypoints": c.lm_waypoints, "lm_iterations": c.lm_iterations}


def jacobian_f64(robot: Robot, q, J, stream=None):
    """q [N][n] FP64 -> J [N][6][n] FP64 (device tensors)."""
    _check(lib().cpp_jacobian_f64(C.byref(robot), ptr(q), q.numel() // robot.n, ptr(J),
                                  stream_handle(stream)), "cpp_jacobian_f64")


def plan_geo(robot: Robot, params: Params, geometry: Geometry | None, cand, targets, K: int,
             workspace, sel, best_cost, q_out, pose_err=None, report=None, dev_status=None,
             stream=None):
    T, n, Kp = cand.shape
    nbytes = workspace.numel() * workspace.element_size()
    g = C.byref(geometry) if geometry is not None else None
    _check(lib().cpp_plan_geo(C.byref(robot), C.byref(params), g, ptr(cand), ptr(targets), T, K,
                              Kp, ptr(workspace), nbytes, ptr(sel), ptr(best_cost), ptr(q_out),
                              ptr(pose_err), ptr(report), ptr(dev_status), stream_handle(stream)),
           "cpp_plan_geo")


def batch_opt_workspace_size(T: int, K: int, n: int, lanes: int) -> int:
    return lib().cpp_batch_opt_workspace_size(T, K, n, lanes)


def batch_opt(robot: Robot, params: Params, cand, targets, K: int, lanes: int, workspace, lane_sel,
              lane_mjac, q_out, reports, best, pose_err=None, dev_status=None, stream=None):
    """cpf-BatchOpt: the `lanes` smoothest candidate lanes refined and checked (device
    tensors: lane_sel [lanes] i32, lane_mjac [lanes] f32, q_out [lanes][T][n] f32,
    reports [lanes * REPORT_BYTES] u8, best [1] i32)."""
    T, n, Kp = cand.shape
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().cpp_batch_opt(C.byref(robot), C.byref(params), ptr(cand), ptr(targets), T, K, Kp,
                               lanes, ptr(workspace), nbytes, ptr(lane_sel), ptr(lane_mjac),
                               ptr(q_out), ptr(pose_err), ptr(reports), ptr(best),
                               ptr(dev_status), stream_handle(stream)), "cpp_batch_opt")


def plan_batch_workspace_size(descs, robots) -> int:
    D = (PlanDesc * len(descs))(*descs)
    R = (Robot * len(robots))(*robots)
    return lib().cpp_plan_batch_workspace_size(D, len(descs), R, len(robots))


def plan_batch(robots, params: Params, descs, workspace, dev_status=None, stream=None):
    D = (PlanDesc * len(descs))(*descs)
    R = (Robot * len(robots))(*robots)
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().cpp_plan_batch(R, len(robots), C.byref(params), D, len(descs), ptr(workspace),
                                nbytes, ptr(dev_status), stream_handle(stream)), "cpp_plan_batch")


class Batch:
    """A prepared batch (cpp_batch_create); run() enqueues any subset of stages."""

    def __init__(self, robots, params: Params, descs, workspace, dev_status=None, stream=None):
        D = (PlanDesc * len(descs))(*descs)
        R = (Robot * len(robots))(*robots)
        h = C.c_void_p()
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().cpp_batch_create(R, len(robots), C.byref(params), D, len(descs),
                                      ptr(workspace), nbytes, ptr(dev_status),
                                      stream_handle(stream), C.byref(h)), "cpp_batch_create")
        self.handle = h
        self.count = len(descs)

    def run(self, stages: int = STAGE_ALL, stream=None):
        _check(lib().cpp_batch_run(self.handle, stages, stream_handle(stream)), "cpp_batch_run")

    def launches(self, stages: int = STAGE_ALL) -> int:
        return lib().cpp_batch_launches(self.handle, stages)

    def set_split(self, alpha: float, cands_per_cta: int = 0, stream=None):
        _check(lib().cpp_batch_set_split(self.handle, float(alpha), int(cands_per_cta),
                                         stream_handle(stream)), "cpp_batch_set_split")

    def set_budget(self, budget_ms: float, stream=None):
        _check(lib().cpp_batch_set_budget(self.handle, float(budget_ms), stream_handle(stream)),
               "cpp_batch_set_budget")

    def set_cluster_min_kp(self, min_kp: int, stream=None):
        _check(lib().cpp_batch_set_cluster_min_kp(self.handle, int(min_kp), stream_handle(stream)),
               "cpp_batch_set_cluster_min_kp")

    def set_mask_tasks(self, tasks_per_warp: int):
        _check(lib().cpp_batch_set_mask_tasks(self.handle, int(tasks_per_warp)),
               "cpp_batch_set_mask_tasks")

    def tune(self, table_path: str | None = None, stream=None) -> dict:
        r = TuneResult()
        path = table_path.encode() if table_path else None
        _check(lib().cpp_batch_tune(self.handle, path, stream_handle(stream), C.byref(r)),
               "cpp_batch_tune")
        return r.as_dict()

    def capture(self, stages: int = STAGE_ALL, stream=None):
        _check(lib().cpp_batch_capture(self.handle, stages, stream_handle(stream)),
               "cpp_batch_capture")

    def replay(self, stream=None):
        _check(lib().cpp_batch_replay(self.handle, stream_handle(stream)), "cpp_batch_replay")

    def close(self):
        if self.handle:
            lib().cpp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """cpp_server_* with host numpy buffers. submit() returns a ticket; poll()/wait()
    return (status, result dict) once the plan is done."""

    def __init__(self, params: Params | None = None, device: int = 0, hbm_budget: int | None = None,
                 max_slots: int | None = None, max_batch: int | None = None,
                 max_inflight: int | None = None, pinned_bytes: int | None = None,
                 latency_requests: int | None = None, search_budget_ms: float | None = None):
        cfg = ServerConfig()
        lib().cpp_server_config_default(C.byref(cfg))
        cfg.device = device
        if params is not None:
            cfg.params = params
        for name, v in (("hbm_budget_bytes", hbm_budget), ("max_slots", max_slots),
                        ("max_batch", max_batch), ("max_inflight", max_inflight),
                        ("pinned_bytes", pinned_bytes), ("latency_requests", latency_requests),
                        ("search_budget_ms", search_budget_ms)):
            if v is not None:
                setattr(cfg, name, v)
        h = C.c_void_p()
        _check(lib().cpp_server_create(C.byref(cfg), C.byref(h)), "cpp_server_create")
        self.handle = h
        self._live = {}  # ticket -> (robot, inputs kept alive, shape)

    def submit(self, robot: Robot, cand, targets, K: int, borrow: bool = False,
               geometry: Geometry | None = None, anytime_rounds: int | None = None) -> int:
        """anytime_rounds: an anytime request with that many improvement rounds."""
        import numpy as np
        cand = np.ascontiguousarray(cand, dtype=np.float32)
        targets = np.ascontiguousarray(targets, dtype=np.float64)
        T, n, Kp = cand.shape
        flags = (REQ_BORROW if borrow else 0) | (REQ_ANYTIME if anytime_rounds is not None else 0)
        req = PlanReq(C.addressof(robot), T, K, Kp, flags, cand.ctypes.data, targets.ctypes.data,
                      C.addressof(geometry) if geometry is not None else None,
                      int(anytime_rounds or 0), 0)
        t = C.c_uint64()
        _check(lib().cpp_plan_submit(self.handle, C.byref(req), C.byref(t)), "cpp_plan_submit")
        self._live[t.value] = (robot, (cand, targets) if borrow else None, (T, n))
        return t.value

    def peek(self, ticket: int):
        """The best-so-far result of an anytime request, without collecting it:
        (status, result dict) -- status PENDING (and None) while none is published."""
        return self._result(ticket, lib().cpp_plan_peek, keep=True)

    def _result(self, ticket: int, fn, *extra, keep: bool = False):
        import numpy as np
        if ticket not in self._live:  # unknown here: let the library answer (NOT_FOUND)
            _check(fn(self.handle, ticket, None, *extra), "cpp_plan_poll")
        robot, _, (T, n) = self._live[ticket]
        sel = np.zeros(T, np.int32)
        q = np.zeros((T, n), np.float32)
        err = np.zeros((T, 2), np.float64)
        rep = Report()
        best = np.zeros(1, np.float32)
        res = PlanResult(sel.ctypes.data, q.ctypes.data, err.ctypes.data, C.addressof(rep),
                         best.ctypes.data, 0.0, 0, 0)
        st = fn(self.handle, ticket, C.byref(res), *extra)
        if st == PENDING:
            return st, None
        if not keep:
            self._live.pop(ticket, None)
        if st == ERR_NOT_FOUND:
            raise CppflowError(st, last_error())
        return st, dict(sel=sel, q=q, err=err, report=rep.as_dict(), best=float(best[0]),
                        latency_ms=res.latency_ms, dev_status=res.dev_status, rounds=res.rounds)

    def poll(self, ticket: int):
        return self._result(ticket, lib().cpp_plan_poll)

    def wait(self, ticket: int, timeout_us: int = -1):
        return self._result(ticket, lib().cpp_plan_wait, timeout_us)

    def cancel(self, ticket: int) -> int:
        return lib().cpp_plan_cancel(self.handle, ticket)

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().cpp_server_get_stats(self.handle, C.byref(s)), "cpp_server_get_stats")
        return s.as_dict()

    def close(self):
        if self.handle:
            lib().cpp_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def report_from_bytes(buf: bytes) -> dict:
    r = Report.from_buffer_copy(buf)
    return r.as_dict()


DEG = math.pi / 180.0
