"""Helpers for the GPU parity tests: move oracle-built problems to the device and
run the C-ABI stages on them."""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import oracle
from paper_2309_09102_gb300 import cppflow


def torch():
    import torch as _t
    return _t


DEV = "cuda:0"

# Tolerances. FK: FP32 rounding (unit round-off 6e-8) accumulates through at most 16
# links of at most 0.4 m each, a few 1e-6 m / rad, so 1e-5 bounds the FP32 pose error
# against FP64 with a margin of a few:
FK_TOL = 1e-5           # m / rad, FP32 FK vs FP64 oracle
GUARD = 1e-5            # pose errors within this of a threshold are excluded from bit checks
JUMP_TOL = 1e-4         # rad, max joint jump of the refined trajectory vs the oracle's
TAU_POS, TAU_ROT = 1e-3, math.radians(0.1)


def params_pair(**kw):
    """The same settings as an oracle.Params and a cppflow.Params."""
    op = oracle.make_params(**{k: v for k, v in kw.items()
                               if k not in ("lm_fp64", "dp_objective", "smooth_rounds", "smooth_lambda",
                                            "pen_collide", "coll_margin", "coll_weight")})
    cp = cppflow.make_params(**kw)
    return op, cp


def dev(a, dtype=None):
    t = torch().from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


@dataclass
class GpuMask:
    mask: np.ndarray
    pen: np.ndarray
    err: np.ndarray


def run_mask(robot, params, cand, targets, K) -> GpuMask:
    T, n, Kp = cand.shape
    tt = torch()
    m = tt.empty(T, Kp, dtype=tt.uint8, device=DEV)
    p = tt.empty(T, Kp, dtype=tt.float32, device=DEV)
    e = tt.empty(T, Kp, 2, dtype=tt.float32, device=DEV)
    cppflow.mask(robot, params, dev(cand), dev(targets), K, m, p, e)
    tt.cuda.synchronize()
    return GpuMask(m.cpu().numpy(), p.cpu().numpy(), e.cpu().numpy())


def run_dp(cand, pen, K):
    T, n, Kp = cand.shape
    tt = torch()
    ws = tt.empty(cppflow.dp_workspace_size(T, Kp), dtype=tt.uint8, device=DEV)
    sel = tt.empty(T, dtype=tt.int32, device=DEV)
    best = tt.empty(1, dtype=tt.float32, device=DEV)
    seed = tt.empty(T, n, dtype=tt.float32, device=DEV)
    st = tt.zeros(1, dtype=tt.int32, device=DEV)
    cppflow.dp_search(dev(cand), dev(pen), K, ws, sel, best, seed, st)
    tt.cuda.synchronize()
    return dict(sel=sel.cpu().numpy(), best=np.float32(best.item()), seed=seed.cpu().numpy(),
                status=int(st.item()))


def run_dp_ex(cand, pen, K, objective):
    T, n, Kp = cand.shape
    tt = torch()
    ws = tt.empty(cppflow.dp_workspace_size(T, Kp), dtype=tt.uint8, device=DEV)
    sel = tt.empty(T, dtype=tt.int32, device=DEV)
    best = tt.empty(1, dtype=tt.float32, device=DEV)
    mj = tt.empty(1, dtype=tt.float32, device=DEV)
    st = tt.zeros(1, dtype=tt.int32, device=DEV)
    cppflow.dp_search_ex(dev(cand), dev(pen), K, objective, ws, sel, best, None, mj, st)
    tt.cuda.synchronize()
    return dict(sel=sel.cpu().numpy(), best=np.float32(best.item()), mjac=np.float32(mj.item()),
                status=int(st.item()))


def run_lm(robot, params, q_in, targets):
    T, n = q_in.shape
    tt = torch()
    qo = tt.empty(T, n, dtype=tt.float32, device=DEV)
    pe = tt.empty(T, 2, dtype=tt.float64, device=DEV)
    st = tt.zeros(1, dtype=tt.int32, device=DEV)
    cppflow.lm_refine(robot, params, dev(q_in.astype(np.float32)), dev(targets), qo, pe, st)
    tt.cuda.synchronize()
    return qo.cpu().numpy(), pe.cpu().numpy()


def run_plan(robot, params, cand, targets, K):
    T, n, Kp = cand.shape
    tt = torch()
    ws = tt.empty(cppflow.plan_workspace_size(T, K, Kp, n), dtype=tt.uint8, device=DEV)
    sel = tt.empty(T, dtype=tt.int32, device=DEV)
    best = tt.empty(1, dtype=tt.float32, device=DEV)
    q = tt.empty(T, n, dtype=tt.float32, device=DEV)
    pe = tt.empty(T, 2, dtype=tt.float64, device=DEV)
    rep = tt.zeros(cppflow.REPORT_BYTES, dtype=tt.uint8, device=DEV)
    st = tt.zeros(1, dtype=tt.int32, device=DEV)
    cppflow.plan(robot, params, dev(cand), dev(targets), K, ws, sel, best, q, pe, rep, st)
    tt.cuda.synchronize()
    return dict(sel=sel.cpu().numpy(), best=np.float32(best.item()), q=q.cpu().numpy(),
                err=pe.cpu().numpy(), report=cppflow.report_from_bytes(rep.cpu().numpy().tobytes()),
                status=int(st.item()))


def path_cost_f32(cand, pen, K, sel):
    """FP32 cost of a given selection, summed in the search's association with the
    per-waypoint relative node costs (an independent restatement for property checks)."""
    f32 = np.float32
    m = pen[:, :K].min(axis=1)
    m = np.where(np.isinf(m), f32(0), m).astype(np.float32)
    r = (pen - m[:, None]).astype(np.float32)
    T = cand.shape[0]
    c = r[0, sel[0]]
    for i in range(1, T):
        d = np.abs(cand[i, :, sel[i]] - cand[i - 1, :, sel[i - 1]]).astype(np.float32).max()
        c = f32(f32(c + f32(d)) + r[i, sel[i]])
    return c
