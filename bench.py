"""Benchmark of the GB300 planner core on the T = 300, K = 512, 7-DoF workload (the
single-request-at-scale configuration).

The headline `value` is plans/s of the batched path with its inputs resident in HBM:
one step = one pass of the whole path (FK + masks, search, backtracking, LM, FP64
check) over one batch of B synthetic requests of that shape. `e2e` is the same metric
served end to end through the serving API (cpp_plan_submit / cpp_plan_wait): host
inputs copied in, continuous batching, results copied out, all inside the timed
region. Beside them, on rank 0:
  * the plain per-request GPU path (cpp_plan one request at a time, one stream),
  * the roofline of the search kernel (FP32 lane operations) and of the LM kernel
    (FP64 flops) against peaks measured in the same run by the library's
    throughput probe,
  * SM clocks during the timed region (nvidia-smi),
  * the serving mix under open-loop Poisson arrivals at 100, 1000 and 5000 req/s:
    served (continuous batching) and plain (the same arrival trace, in real time,
    one request at a time through cpp_plan_host) -- plans/s, p50 / p99 latency,
  * the batched uneven workload (tuned schedule, CUDA graph), the collision-aware
    workload, the 9-DoF T = 2000, K = 1024 precision case with both LM precisions,
  * the CPU-oracle leg: the FP64 oracle timed on the host's cores on a bounded
    sample of the workload (the same inputs as the GPU's first requests), with the
    GPU results of those requests and of the precision case compared against it.
``--impl reference`` times the CPU oracle alone as the reference arm.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl cuda|reference]
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import queue
import tempfile
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

# The server runs its launches on up to 16 streams, each forking its search groups onto
# side streams. CUDA maps streams onto 8 hardware queues by default, and work in one
# queue runs in order, so launches of unrelated streams wait on each other. 32 queues
# remove most of that (set before the first CUDA call; a value set by the caller wins).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2309_09102_gb300 import synth  # noqa: E402

METRIC = "served plans/s & p99 latency at \u22641mm/\u22640.1\u00b0 vs plain per-request GPU path"
VALUE_IS = ("plans/s of the batched path, inputs resident in HBM (T=300 K=512 7-DoF, valid at "
            "<=1mm/<=0.1deg); e2e = the same through the serving API from host memory; the "
            "served-vs-plain comparison under Poisson arrivals is in serving_mix")
# DRAM bytes (read + write) of one dp3_forward_kernel launch on this workload (304 requests,
# T = 300, K = 512, n = 7), from one ncu capture of the kernel build it names
# (profiles/dp3_forward_single_t300_k512_b304.md). Set to None whenever the kernel changes.
DP3_TRAFFIC_BYTES = 1.496150e9 + 91.826176e6


def lm_flops_per_iter(n: int) -> int:
    """FP64 flops of one LM iteration of one waypoint (FP32 Jacobian mode): J^T J lower
    triangle 6 n (n + 1), J^T e 12 n, lambda on the diagonal n, Cholesky sum_j [2 j + 2 +
    (n - 1 - j)(2 j + 1)], two triangular solves 2 n^2, the step n, the trial cost 12
    (691 at n = 7). FP32 work (chains, Jacobian columns) is not counted."""
    chol = sum(2 * j + 2 + (n - 1 - j) * (2 * j + 1) for j in range(n))
    return 6 * n * (n + 1) + 12 * n + n + chol + 2 * n * n + n + 12


def workload_requests(B: int, rank: int):
    """B requests shaped like the single-request-at-scale workload; arm r mod 8 of 8
    seeded chains, distinct paths and candidates per request (and per rank)."""
    base = synth.SINGLE
    out = []
    for r in range(B):
        g = rank * B + r
        out.append(synth.Workload(f"{base.name}_r{g}", base.n, base.T, base.K, base.sigma,
                                  base.p_wb, base.p_out, base.lm_iters, base.lambda0,
                                  arm_seed=100 + (g % 8), path_seed=7000 + g, cand_seed=9000 + g))
    return out


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, device_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.dev = device_index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_problem(w: synth.Workload):
    import oracle
    arm = synth.draw_arm(w.arm_seed, w.n, w.wrist)
    rob = oracle.make_robot(arm.a, arm.d, arm.alpha, arm.lo, arm.hi, arm.theta0)
    truth = synth.draw_truth(w.path_seed, w.n, w.T, w.wrist)
    targets = oracle.fk_pose(rob, truth)
    P_wb = oracle.make_params(lm_iters=30, free_mask=synth.wrong_branch_free_mask(w.n))
    q_wb, _, _ = oracle.lm(rob, P_wb, synth.wrong_branch_start(truth), targets)
    draws = synth.draw_candidates(w.cand_seed, w.T, w.K, w.n, w.p_wb, w.p_out)
    cand = synth.assemble(truth, q_wb, draws, w.sigma, arm.lo, arm.hi)
    return rob, targets, cand


def cpu_oracle_run(reqs, threads: int, steps: int = 1, probs=None):
    """Time the oracle (mask, FP32 search, LM, check) on `reqs`, one request per thread
    (the C oracle releases the GIL), `steps` times. probs: the inputs (robot, targets,
    lattice) per request, else built with the oracle. Returns (plans/s, valid, seconds,
    results of the last step)."""
    import oracle
    oracle.build()
    if probs is None:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            probs = list(ex.map(oracle_problem, reqs))
    P = oracle.make_params(lm_iters=reqs[0].lm_iters, lambda0=reqs[0].lambda0)

    def one(i):
        rob, targets, cand = probs[i]
        return oracle.plan(rob, P, cand, targets, reqs[i].K)

    t0 = time.perf_counter()
    valid = 0
    outs = []
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for _ in range(steps):
            outs = list(ex.map(one, range(len(probs))))
            valid += sum(o["report"]["valid"] for o in outs)
    dt = time.perf_counter() - t0
    return len(probs) * steps / dt, valid, dt, outs


def oracle_leg(arms, reqs, cand_h, targets_h, gpu, stress, per_core: int = 4) -> dict:
    """The CPU-oracle leg (rank 0 at N = 1). (1) The FP64 oracle plans the first
    cores * per_core requests of the batch on the GPU's own inputs, one request per host
    thread on every core, timed: the CPU baseline. Its results are compared with the
    GPU's for the same requests: search indices, refined joints, mjac. (2) The precision
    case: the oracle's LM from the GPU search's seed, compared with both GPU LM modes."""
    import oracle
    cores = os.cpu_count() or 1
    S = cores
    m = min(len(reqs), S * per_core)
    probs = []
    for r in range(m):
        a = arms[reqs[r].arm_seed - 100]
        probs.append((oracle.make_robot(a.a, a.d, a.alpha, a.lo, a.hi, a.theta0),
                      targets_h[r].numpy(), cand_h[r].numpy()))
    value, valid, dt, outs = cpu_oracle_run(reqs[:m], S, probs=probs)
    same_sel = sum(int(np.array_equal(o["sel"], gpu["sel"][r])) for r, o in enumerate(outs))
    dq = max(float(np.abs(gpu["q"][r].astype(np.float64) - o["q"]).max()) for r, o in enumerate(outs))
    dmjac = max(abs(gpu["mjac"][r] - o["report"]["mjac"]) for r, o in enumerate(outs))
    base = {"value": round(value, 3), "unit": "plans/s", "cores": S, "host_cpu_count": cores,
            "kind": "oracle",
            "sample": f"{m} requests of T=300 K=512 n=7 (the GPU batch's first {m}, same inputs; "
                      f"mask + FP32 search + FP64 LM + check) on {S} threads, {dt:.1f} s wall "
                      f"(~{dt * S:.0f} s of CPU work)",
            "valid": int(valid),
            "vs_gpu": {"requests": m, "identical_search_indices": f"{same_sel}/{m}",
                       "max_abs_q_diff_rad": dq, "max_abs_mjac_diff_rad": dmjac,
                       "gpu_max_pos_err_m": max(gpu["max_pos"][:m]),
                       "gpu_max_rot_err_deg": math.degrees(max(gpu["max_rot"][:m]))}}
    st = None
    if stress is not None:
        rob = oracle.make_robot(*stress["arm"])
        P = oracle.make_params(lm_iters=stress["lm_iters"], lambda0=stress["lambda0"])
        t0 = time.perf_counter()
        q_o, _, iters = oracle.lm(rob, P, stress["seed"], stress["targets"])
        t_lm = time.perf_counter() - t0
        err_o, rep_o = oracle.check(rob, P, q_o, stress["targets"])
        st = {"oracle_lm_s": round(t_lm, 2), "oracle_max_pos_m": float(err_o[:, 0].max()),
              "oracle_max_rot_deg": math.degrees(float(err_o[:, 1].max())),
              "oracle_mjac_rad": float(rep_o["mjac"]), "oracle_valid": int(rep_o["valid"]),
              "oracle_mean_lm_iters": round(float(iters.mean()), 2)}
        for name, q in stress["q"].items():
            st[name] = {"max_abs_q_diff_rad": float(np.abs(q.astype(np.float64) - q_o).max()),
                        "abs_mjac_diff_rad": abs(stress["mjac"][name] - float(rep_o["mjac"]))}
    return {"cpu_baseline": base, "stress_vs_oracle": st}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    S = cores
    reqs = workload_requests(S, 0)
    cpu_oracle_run(reqs[:1], 1)  # warm the library
    value, valid, dt, _ = cpu_oracle_run(reqs, S, steps=args.steps)
    line = {"metric": METRIC, "value": round(value, 3), "unit": "plans/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * dt / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": synth.SINGLE.name, "T": 300, "K": 512, "n": 7,
                       "requests_per_step": S},
            "cpu_baseline": {"value": round(value, 3), "unit": "plans/s", "cores": S,
                             "host_cpu_count": cores, "kind": "oracle",
                             "sample": f"{S} requests per step, one per thread"},
            "e2e": {"value": round(value, 3), "unit": "plans/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- serving mix
def serving_pool(cppflow, torch, dev, pool_size: int):
    """pool_size distinct requests of the serving mix (T = floor(exp U(ln 50, ln 2000)),
    K in {128, 256, 512, 1024}, 7-DoF arms r mod 8): target poses by the library's FP64
    FK and wrong-branch solutions by its FP64 LM on the GPU, random draws and assembly
    on the host threads, every lattice in one pinned host buffer."""
    n = 7
    arms = [synth.draw_arm(100 + k, n) for k in range(8)]
    robots = [cppflow.robot_from_arm(a) for a in arms]
    P_wb = cppflow.make_params(lm_iters=30, lm_fp64=1, free_mask=synth.wrong_branch_free_mask(n))
    ws = [synth.serving_request(r) for r in range(pool_size)]
    threads = os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        truths = list(ex.map(lambda w: synth.draw_truth(w.path_seed, n, w.T), ws))
    targets, qwb = [], []
    for w, truth in zip(ws, truths):
        rob = robots[w.arm_seed - 100]
        tgt = torch.empty(w.T, 7, dtype=torch.float64, device=dev)
        cppflow.fk_pose_f64(rob, torch.from_numpy(truth).to(dev), tgt)
        q = torch.empty(w.T, n, dtype=torch.float32, device=dev)
        cppflow.lm_refine(rob, P_wb, torch.from_numpy(
            synth.wrong_branch_start(truth).astype(np.float32)).to(dev), tgt, q)
        targets.append(tgt)
        qwb.append(q)
    torch.cuda.synchronize()
    sizes = [w.T * n * synth.pad_k(w.K) for w in ws]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    big = torch.empty(int(offs[-1]), dtype=torch.float32, pin_memory=True)
    bnp = big.numpy()
    tsz = [w.T * 7 for w in ws]
    toffs = np.concatenate([[0], np.cumsum(tsz)])
    tbig = torch.empty(int(toffs[-1]), dtype=torch.float64, pin_memory=True)
    tnp = tbig.numpy()
    qwb_h = [q.cpu().numpy().astype(np.float64) for q in qwb]
    for r in range(pool_size):
        tnp[toffs[r]:toffs[r + 1]] = targets[r].cpu().numpy().ravel()

    def fill(r):
        w = ws[r]
        arm = arms[w.arm_seed - 100]
        d = synth.draw_candidates(w.cand_seed, w.T, w.K, n, w.p_wb, w.p_out)
        lat = synth.assemble(truths[r], qwb_h[r], d, w.sigma, arm.lo, arm.hi, synth.pad_k(w.K))
        bnp[offs[r]:offs[r + 1]] = lat.ravel()

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(fill, range(pool_size)))
    pool = []
    for r, w in enumerate(ws):
        Kp = synth.pad_k(w.K)
        pool.append((w, robots[w.arm_seed - 100], bnp[offs[r]:offs[r + 1]].reshape(w.T, n, Kp),
                     tnp[toffs[r]:toffs[r + 1]].reshape(w.T, 7)))
    return pool, (big, tbig)


def _pct(v, q):
    v = sorted(v)
    return round(1000 * v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))], 3)


def serving_mix(cppflow, torch, dev, rates, pool_size: int, seconds: float, min_requests: int,
                plain_max: int):
    """Open-loop Poisson arrivals of the serving mix at each rate, drawn with replacement
    from a pool of distinct requests. Per rate, max(`seconds` of arrivals, `min_requests`)
    requests are reported after a warm-up of 10 % more.
    served: real-time submission to cpp_plan_submit (borrowed pinned inputs) while a
    second client thread collects the results in submission order (cpp_plan_wait),
    latency = arrival -> completion seen by the server; the p50 of the first and the
    last third of the reported requests show whether the server keeps up (a server
    that falls behind sees its latency grow over the window).
    plain: the same arrival trace in real time through cpp_plan_host, one request at a
    time on one stream (inputs copied in, results copied out, the next request starts
    when the previous one is done), latency = arrival -> completion, over the trace's
    first `plain_max` reported requests (a saturated plain path falls further behind
    with every request, so a longer trace only lengthens its queue).
    plans/s = reported requests / (last completion - first reported arrival)."""
    pool, keep = serving_pool(cppflow, torch, dev, pool_size)
    n = 7
    P = cppflow.make_params()
    T_max = max(w.T for w, *_ in pool)
    Kp_max = max(synth.pad_k(w.K) for w, *_ in pool)
    ws = torch.empty(cppflow.plan_host_workspace_size(T_max, Kp_max, Kp_max, n), dtype=torch.uint8,
                     device=dev)
    sel_h = torch.empty(T_max, dtype=torch.int32, pin_memory=True).numpy()
    q_h = torch.empty(T_max * n, dtype=torch.float32, pin_memory=True).numpy()
    rep_h = cppflow.Report()
    pstream = torch.cuda.Stream()
    # warm the plain path: one request of every K in the pool (each K takes its own
    # kernel instances, which CUDA loads on their first launch); repeated before each
    # plain timing, after the served run's teardown, so no one-time cost of the
    # device or driver falls inside the plain window
    first_of_k = {}
    for item in pool:
        first_of_k.setdefault(item[0].K, item)

    def warm_plain():
        for w, rob, ch, th in first_of_k.values():
            cppflow.plan_host(rob, P, ch, th, w.K, ws, sel_h[:w.T], None, q_h[:w.T * n], None,
                              rep_h, stream=pstream)
        torch.cuda.synchronize()

    warm_plain()
    # Warm the served path: CUDA loads a kernel on its first launch, which would stall
    # the server's worker the first time each search form and size appears. The whole
    # pool at once (every throughput form) and a few requests one by one (the latency
    # forms) load them before any measured window.
    with cppflow.Server(P, device=dev.index or 0, hbm_budget=40 << 30, max_batch=512,
                        max_inflight=16) as srv:
        for tk in [srv.submit(rob, ch, th, w.K, borrow=True) for w, rob, ch, th in pool]:
            srv.wait(tk)
        for w, rob, ch, th in pool[:64]:
            srv.wait(srv.submit(rob, ch, th, w.K, borrow=True))
    out = {"pool_requests": pool_size}
    for rate in rates:
        target = int(max(min_requests, math.ceil(rate * seconds)))
        count = int(math.ceil(target / 0.9))
        drop = count - target
        ptarget = min(target, plain_max)
        pcount = drop + ptarget
        arr = synth.poisson_arrivals(rate, count, seed=int(rate))
        pick = (synth.uniform(991 + int(rate), synth.S_MIX, count) * len(pool)).astype(int)
        # served: real-time open-loop submission (Python's cyclic collector is run before and
        # paused during the loop, so no collection pause delays the arrivals)
        gc.collect()
        gc.disable()
        with cppflow.Server(P, device=dev.index or 0, hbm_budget=40 << 30, max_batch=512,
                            max_inflight=16) as srv:
            done, ok = [0.0] * count, [False] * count
            handoff = queue.SimpleQueue()

            def collector():
                while (item := handoff.get()) is not None:
                    i, tk, sub = item
                    stt, res = srv.wait(tk)
                    done[i] = sub + res["latency_ms"] / 1000.0
                    ok[i] = stt == cppflow.OK and bool(res["report"]["valid"])

            coll = threading.Thread(target=collector)
            coll.start()
            t0 = time.perf_counter()
            for i, (a, k) in enumerate(zip(arr, pick)):
                now = time.perf_counter() - t0
                if a > now:
                    time.sleep(a - now)
                w, rob, ch, th = pool[k]
                sub = time.perf_counter() - t0
                handoff.put((i, srv.submit(rob, ch, th, w.K, borrow=True), sub))
            handoff.put(None)
            coll.join()
            valid = sum(ok[drop:])
            ss = srv.stats()
        gc.enable()
        slat = [d - a for d, a in zip(done[drop:], arr[drop:])]
        sspan = max(done[drop:]) - arr[drop]
        third = max(1, target // 3)
        # plain: the same trace through one stream, one request at a time
        warm_plain()
        gc.collect()
        gc.disable()
        pdone, pvalid = [], 0
        t0 = time.perf_counter()
        for i, (a, k) in enumerate(zip(arr[:pcount], pick[:pcount])):
            now = time.perf_counter() - t0
            if a > now:
                time.sleep(a - now)
            w, rob, ch, th = pool[k]
            st = cppflow.plan_host(rob, P, ch, th, w.K, ws, sel_h[:w.T], None, q_h[:w.T * n], None,
                                   rep_h, stream=pstream)
            pdone.append(time.perf_counter() - t0)
            if i >= drop:
                pvalid += int(st == cppflow.OK and rep_h.valid)
        gc.enable()
        plat = [d - a for d, a in zip(pdone[drop:], arr[drop:pcount])]
        pspan = max(pdone[drop:]) - arr[drop]
        out[str(int(rate))] = {
            "requests": count, "reported": target,
            "offered_per_s": round(target / (arr[-1] - arr[drop]), 1),
            "served": {"plans_per_s": round(target / sspan, 1), "p50_ms": _pct(slat, 0.5),
                       "p99_ms": _pct(slat, 0.99),
                       "p50_first_third_ms": _pct(slat[:third], 0.5),
                       "p50_last_third_ms": _pct(slat[-third:], 0.5),
                       "valid": f"{valid}/{target}",
                       "mean_batch": round(ss["sum_batch"] / max(1, ss["batches"]), 2),
                       "batches": ss["batches"], "max_batch": ss["max_batch_seen"],
                       "hbm_high_water_bytes": ss["hbm_high_water"]},
            "plain": {"plans_per_s": round(ptarget / pspan, 1), "p50_ms": _pct(plat, 0.5),
                      "p99_ms": _pct(plat, 0.99), "reported": ptarget,
                      "valid": f"{pvalid}/{ptarget}"}}
    del keep
    return out


# ----------------------------------------------------------------------------- GPU arm
def build_inputs(cppflow, torch, dev, reqs, want_truth: bool = False):
    """Pinned host lattices and FP64 targets of the given requests (each with its own
    T, K and n): random draws on the host, target poses by the library's FP64 FK,
    wrong-branch solutions by its FP64 LM restricted to the wrist joints.
    Returns (arms, robots, cand_h, targets_h); arm a of robots is seed 100 + a."""
    n = reqs[0].n
    arms = [synth.draw_arm(100 + k, n) for k in range(8)]
    robots = [cppflow.robot_from_arm(a) for a in arms]
    P_wb = cppflow.make_params(lm_iters=30, lm_fp64=1, free_mask=synth.wrong_branch_free_mask(n))

    def draws_of(w):
        truth = synth.draw_truth(w.path_seed, w.n, w.T)
        return truth, synth.draw_candidates(w.cand_seed, w.T, w.K, w.n, w.p_wb, w.p_out)

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        drawn = list(ex.map(draws_of, reqs))
    cand_h, targets_h = [], []
    truths = []
    for r, w in enumerate(reqs):
        truth, draws = drawn[r]
        truths.append(truth)
        rob = robots[w.arm_seed - 100]
        tq = torch.from_numpy(truth).to(dev)
        tgt = torch.empty(w.T, 7, dtype=torch.float64, device=dev)
        cppflow.fk_pose_f64(rob, tq, tgt)
        q0 = torch.from_numpy(synth.wrong_branch_start(truth).astype(np.float32)).to(dev)
        qwb = torch.empty(w.T, w.n, dtype=torch.float32, device=dev)
        cppflow.lm_refine(rob, P_wb, q0, tgt, qwb)
        torch.cuda.synchronize()
        arm = arms[w.arm_seed - 100]
        cand = synth.assemble(truth, qwb.cpu().numpy().astype(np.float64), draws, w.sigma,
                              arm.lo, arm.hi, synth.pad_k(w.K))
        cand_h.append(torch.from_numpy(cand).pin_memory())
        targets_h.append(tgt.cpu().pin_memory())
    if want_truth:
        return arms, robots, cand_h, targets_h, truths
    return arms, robots, cand_h, targets_h


def stress_leg(cppflow, torch, dev):
    """The stress / precision workload: a 9-DoF chain with a spherical wrist, T = 2000,
    K = 1024, the true path through near-singular wrist poses (joint 6 within 0.02 rad
    of 0). One request through cpp_plan with the FP32-Jacobian LM (FP64 normal equations
    and Cholesky, the default) and again with the all-FP64 LM: plan time, per-path pose
    errors (FP64 check) and joint jumps of each, and the smallest singular value of the
    library's FP64 Jacobian along the refined path. Returns (report, data for the
    comparison with the oracle in the CPU-oracle leg)."""
    w = synth.STRESS
    arm = synth.draw_arm(w.arm_seed, w.n, w.wrist)
    rob = cppflow.robot_from_arm(arm)
    truth = synth.draw_truth(w.path_seed, w.n, w.T, w.wrist)
    tgt = torch.empty(w.T, 7, dtype=torch.float64, device=dev)
    cppflow.fk_pose_f64(rob, torch.from_numpy(truth).to(dev), tgt)
    P_wb = cppflow.make_params(lm_iters=30, lm_fp64=1, free_mask=synth.wrong_branch_free_mask(w.n))
    qwb = torch.empty(w.T, w.n, dtype=torch.float32, device=dev)
    cppflow.lm_refine(rob, P_wb, torch.from_numpy(synth.wrong_branch_start(truth).astype(np.float32)).to(dev),
                      tgt, qwb)
    torch.cuda.synchronize()
    draws = synth.draw_candidates(w.cand_seed, w.T, w.K, w.n, w.p_wb, w.p_out)
    cand = synth.assemble(truth, qwb.cpu().numpy().astype(np.float64), draws, w.sigma,
                          arm.lo, arm.hi, synth.pad_k(w.K))
    cd = torch.from_numpy(cand).to(dev)
    T, n, Kp = cand.shape
    st = torch.cuda.current_stream()
    out = {"workload": f"stress: {n}-DoF spherical wrist, T={T}, K={w.K}, joint 6 within 0.02 rad "
                       "of 0 along the true path; one request, cpp_plan"}
    qs, mj = {}, {}
    sel_h = None
    for mode, name in ((0, "fp32_jacobian_lm"), (1, "all_fp64_lm")):
        P = cppflow.make_params(lm_iters=w.lm_iters, lambda0=w.lambda0, lm_fp64=mode)
        ws = torch.empty(cppflow.plan_workspace_size(T, w.K, Kp, n), dtype=torch.uint8, device=dev)
        sel = torch.empty(T, dtype=torch.int32, device=dev)
        best = torch.empty(1, device=dev)
        q = torch.empty(T, n, device=dev)
        err = torch.empty(T, 2, dtype=torch.float64, device=dev)
        rep = torch.zeros(cppflow.REPORT_BYTES, dtype=torch.uint8, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        times = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record(st)
            cppflow.plan(rob, P, cd, tgt, w.K, ws, sel, best, q, err, rep, status, stream=st)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        r = cppflow.report_from_bytes(rep.cpu().numpy().tobytes())
        qs[name] = q.cpu().numpy()
        mj[name] = float(r["mjac"])
        sel_h = sel.cpu().numpy()
        # smallest singular value of the FP64 geometric Jacobian at every refined waypoint
        J = torch.empty(T, 6, n, dtype=torch.float64, device=dev)
        cppflow.jacobian_f64(rob, q.to(torch.float64).contiguous(), J)
        sv = np.linalg.svd(J.cpu().numpy(), compute_uv=False)[:, -1]
        out[name] = {"plan_ms": round(min(times[1:]), 3), "valid": int(r["valid"]),
                     "max_pos_m": float(r["max_pos"]), "max_rot_deg": math.degrees(r["max_rot"]),
                     "mjac_rad": float(r["mjac"]), "sum_linf_rad": float(r["sum_linf"]),
                     "status": int(status.item()),
                     "sigma_min_J": {"min": float(sv.min()), "median": float(np.median(sv)),
                                     "argmin_waypoint": int(sv.argmin())}}
    out["max_abs_q_diff_between_modes_rad"] = float(np.abs(qs["fp32_jacobian_lm"].astype(np.float64)
                                                           - qs["all_fp64_lm"]).max())
    data = {"arm": (arm.a, arm.d, arm.alpha, arm.lo, arm.hi, arm.theta0),
            "seed": cand[np.arange(T), :, sel_h].astype(np.float64),
            "targets": tgt.cpu().numpy(), "lm_iters": w.lm_iters, "lambda0": w.lambda0,
            "q": qs, "mjac": mj}
    return out, data


def path_clearance(cppflow, torch, dev, robot, geometry, q, params):
    """Smallest clearance of each configuration of q [T][n] under a collision model,
    from the library's collision mask (the configurations as one-lane lattices)."""
    T, n = q.shape
    cand = torch.zeros(T, n, 4, dtype=torch.float32, device=dev)
    cand[:, :, 0] = torch.as_tensor(q, dtype=torch.float32, device=dev)
    tg = torch.zeros(T, 7, dtype=torch.float64, device=dev)
    tg[:, 3] = 1.0
    m = torch.empty(T, 4, dtype=torch.uint8, device=dev)
    p = torch.empty(T, 4, dtype=torch.float32, device=dev)
    c = torch.empty(T, 4, dtype=torch.float32, device=dev)
    cppflow.mask_geo(robot, params, geometry, cand, tg, 1, m, p, None, c)
    return c[:, 0].cpu().numpy()


def collision_leg(cppflow, torch, dev, nreq: int, boxes: int = 4, rounds: int = 3) -> dict:
    """Collision-aware planning on the T = 300, K = 512 workload: per request link
    capsules (radius 2 cm) and `boxes` cuboids that the true path clears by 5 cm
    (drawn, then kept when the library's clearance along the true path allows),
    the collision cost in the search and `rounds` trajectory-length steps with the
    collision rows between pose phases. Reports plans/s, validity and the smallest
    clearance of the refined paths, beside the same run without collision rows."""
    reqs = workload_requests(nreq, 0)
    arms, robots, cand_h, targets_h, truths = build_inputs(cppflow, torch, dev, reqs, want_truth=True)
    T, K, n = synth.SINGLE.T, synth.SINGLE.K, synth.SINGLE.n
    Kp = synth.pad_k(K)
    P0 = cppflow.make_params(lm_iters=20)
    geos, kept = [], []
    for r, w in enumerate(reqs):
        arm = arms[w.arm_seed - 100]
        caps = synth.link_capsules(arm, radius=0.02)
        # self-collision pairs only where the true path itself keeps 1 cm between them
        self_cl = path_clearance(cppflow, torch, dev, robots[w.arm_seed - 100],
                                 cppflow.geometry_from(caps), truths[r], P0)
        if self_cl.min() < 0.01:
            caps = synth.Geometry(caps.cap_frame, caps.cap_a, caps.cap_b, caps.cap_r, caps.pairs[:0],
                                  caps.box_R, caps.box_p, caps.box_half)
        pool = synth.with_boxes(caps, 60000 + r, 16)
        good = []
        for b in range(16):
            one = synth.Geometry(caps.cap_frame, caps.cap_a, caps.cap_b, caps.cap_r, caps.pairs[:0],
                                 pool.box_R[b:b + 1], pool.box_p[b:b + 1], pool.box_half[b:b + 1])
            cl = path_clearance(cppflow, torch, dev, robots[w.arm_seed - 100],
                                cppflow.geometry_from(one), truths[r], P0)
            if cl.min() >= 0.05:
                good.append(b)
            if len(good) == boxes:
                break
        kept.append(len(good))
        geo = synth.Geometry(caps.cap_frame, caps.cap_a, caps.cap_b, caps.cap_r, caps.pairs,
                             pool.box_R[good], pool.box_p[good], pool.box_half[good])
        geos.append(cppflow.geometry_from(geo))
    cand_d = [c.to(dev) for c in cand_h]
    targ_d = [t.to(dev) for t in targets_h]
    out = {"workload": f"collision-aware: {nreq} requests T={T} K={K} n={n}, link capsules r = 2 cm "
                       f"(pairs >= 2 links apart), up to {boxes} boxes clearing the true path by 5 cm",
           "boxes_per_request": round(float(np.mean(kept)), 2)}
    for label, P in (("with_collision_rows", cppflow.make_params(lm_iters=20, smooth_rounds=rounds)),
                     ("without_collision_rows", cppflow.make_params(lm_iters=20, smooth_rounds=rounds,
                                                                    coll_weight=0.0))):
        outs, descs = [], []
        for r in range(nreq):
            o = dict(sel=torch.empty(T, dtype=torch.int32, device=dev),
                     q=torch.empty(T, n, dtype=torch.float32, device=dev),
                     err=torch.empty(T, 2, dtype=torch.float64, device=dev),
                     rep=torch.zeros(cppflow.REPORT_BYTES, dtype=torch.uint8, device=dev),
                     best=torch.empty(1, dtype=torch.float32, device=dev))
            outs.append(o)
            d = cppflow.PlanDesc(T, K, Kp, reqs[r].arm_seed - 100, cand_d[r].data_ptr(),
                                 targ_d[r].data_ptr(), o["sel"].data_ptr(), o["q"].data_ptr(),
                                 o["err"].data_ptr(), o["rep"].data_ptr(), o["best"].data_ptr())
            d.geometry = cppflow.C.addressof(geos[r])
            descs.append(d)
        ws = torch.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=torch.uint8, device=dev)
        st = torch.zeros(nreq, dtype=torch.int32, device=dev)
        s0 = torch.cuda.Stream()
        batch = cppflow.Batch(robots, P, descs, ws, st, s0)
        for _ in range(2):
            batch.run(cppflow.STAGE_ALL, s0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s0)
        for _ in range(3):
            batch.run(cppflow.STAGE_ALL, s0)
        e1.record(s0)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        reps = [cppflow.report_from_bytes(o["rep"].cpu().numpy().tobytes()) for o in outs]
        clear = [float(path_clearance(cppflow, torch, dev, robots[reqs[r].arm_seed - 100], geos[r],
                                      outs[r]["q"].cpu().numpy(), P0).min()) for r in range(nreq)]
        out[label] = {"ms_per_batch": round(ms, 3), "plans_per_s": round(nreq / (ms / 1e3), 1),
                      "valid_plans": f"{sum(int(x['valid']) for x in reps)}/{nreq}",
                      "collision_free_paths": f"{sum(int(c >= 0) for c in clear)}/{nreq}",
                      "min_clearance_m": round(min(clear), 4),
                      "median_path_clearance_m": round(float(np.median(clear)), 4),
                      "mean_mjac_rad": round(float(np.mean([x["mjac"] for x in reps])), 4),
                      "dev_status_nonzero": int((st != 0).sum())}
        batch.close()
    return out


def uneven_batch(cppflow, torch, dev, nreq: int) -> dict:
    """The batched uneven launch: nreq requests (T ~ U{50..1000}, K in {128, 256, 512},
    7-DoF arms from 8 seeded chains) in one prepared batch, its search schedule
    tuned on the batch, all stages captured into one CUDA graph and replayed;
    inputs resident in HBM. Reported beside the headline, not as it."""
    reqs = [synth.batched_request(r) for r in range(nreq)]
    _, robots, cand_h, targets_h = build_inputs(cppflow, torch, dev, reqs)
    P = cppflow.make_params(lm_iters=20, lambda0=1e-3)
    keep, descs = [], []
    for r, w in enumerate(reqs):
        o = dict(cand=cand_h[r].to(dev), targets=targets_h[r].to(dev),
                 sel=torch.empty(w.T, dtype=torch.int32, device=dev),
                 q=torch.empty(w.T, w.n, dtype=torch.float32, device=dev),
                 err=torch.empty(w.T, 2, dtype=torch.float64, device=dev),
                 rep=torch.zeros(cppflow.REPORT_BYTES, dtype=torch.uint8, device=dev),
                 best=torch.empty(1, dtype=torch.float32, device=dev))
        keep.append(o)
        descs.append(cppflow.PlanDesc(w.T, w.K, synth.pad_k(w.K), w.arm_seed - 100,
                                      o["cand"].data_ptr(), o["targets"].data_ptr(),
                                      o["sel"].data_ptr(), o["q"].data_ptr(), o["err"].data_ptr(),
                                      o["rep"].data_ptr(), o["best"].data_ptr()))
    del cand_h
    ws = torch.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=torch.uint8, device=dev)
    status = torch.zeros(nreq, dtype=torch.int32, device=dev)
    st = torch.cuda.Stream()
    batch = cppflow.Batch(robots, P, descs, ws, status, st)

    def time_runs(fn, reps=5):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    batch.set_split(0.0, 0, st)
    unsplit_ms = time_runs(lambda: batch.run(cppflow.STAGE_ALL, st))
    t0 = time.perf_counter()
    tune = batch.tune(None, st)
    tune_s = time.perf_counter() - t0
    batch.capture(cppflow.STAGE_ALL, st)
    graph_ms = time_runs(lambda: batch.replay(st))
    torch.cuda.synchronize()
    reps = [cppflow.report_from_bytes(o["rep"].cpu().numpy().tobytes()) for o in keep]
    out = {"workload": f"batched uneven: {nreq} requests, T ~ U{{50..1000}}, K in {{128, 256, 512}}, "
                       "7-DoF, inputs resident",
           "plans_per_s": round(nreq / (graph_ms / 1e3), 1), "ms_per_batch": round(graph_ms, 3),
           "launches": batch.launches(cppflow.STAGE_ALL),
           "unsplit_ms_per_batch": round(unsplit_ms, 3),
           "tuned": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in tune.items()},
           "tune_s": round(tune_s, 2),
           "valid_plans": f"{sum(int(r['valid']) for r in reps)}/{nreq}",
           "dev_status_nonzero": int((status != 0).sum())}
    batch.close()
    return out


def measure_peaks(cppflow, torch, dev) -> dict:
    """FP32 lane-operation and FP64 flop rates of the library's throughput probe
    (cpp_peak_probe: 4 blocks of 256 threads per SM, 8 independent chains per thread):
    each probe sized to about 25 ms, best of 6 launches timed with CUDA events on the
    launching stream, SM clocks sampled meanwhile."""
    st = torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    out = {}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.2)
    for kind, name in ((cppflow.PROBE_FP32, "fp32_lane_ops_per_s"),
                       (cppflow.PROBE_FP64, "fp64_flops_per_s")):
        iters, best = 1024, 0.0
        for rep in range(8):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ops = cppflow.peak_probe(kind, 4, iters, sink, st)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if rep < 2:  # size the probe to about 25 ms
                iters = int(min(1e9, max(1024, iters * 25.0 / max(ms, 1e-3))))
                continue
            best = max(best, ops / (ms / 1e3))
        out[name] = best
    out["clocks"] = clocks.stop()
    return out


def run_cuda(args, rank: int, world: int, dist):
    import torch

    from paper_2309_09102_gb300 import cppflow

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cppflow.lib()
    B = args.batch
    reqs = workload_requests(B, rank)
    n, T, K = synth.SINGLE.n, synth.SINGLE.T, synth.SINGLE.K
    Kp = synth.pad_k(K)

    # ---- inputs: random draws on the host, target FK and wrong-branch re-solve on the GPU
    arms, robots, cand_h, targets_h = build_inputs(cppflow, torch, dev, reqs)
    P = cppflow.make_params(lm_iters=synth.SINGLE.lm_iters, lambda0=synth.SINGLE.lambda0)

    # ---- device buffers and the prepared batch
    cand_d = [c.to(dev) for c in cand_h]
    targ_d = [t.to(dev) for t in targets_h]
    sel = torch.empty(B, T, dtype=torch.int32, device=dev)
    q_out = torch.empty(B, T, n, dtype=torch.float32, device=dev)
    err = torch.empty(B, T, 2, dtype=torch.float64, device=dev)
    rep = torch.zeros(B, cppflow.REPORT_BYTES, dtype=torch.uint8, device=dev)
    best = torch.empty(B, dtype=torch.float32, device=dev)
    status = torch.zeros(B, dtype=torch.int32, device=dev)
    descs = [cppflow.PlanDesc(T, K, Kp, reqs[r].arm_seed - 100, cand_d[r].data_ptr(),
                              targ_d[r].data_ptr(), sel[r].data_ptr(), q_out[r].data_ptr(),
                              err[r].data_ptr(), rep[r].data_ptr(), best[r].data_ptr())
             for r in range(B)]
    ws = torch.empty(cppflow.plan_batch_workspace_size(descs, robots), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    batch = cppflow.Batch(robots, P, descs, ws, status, stream)
    # the library's autotuner, once, before the warm-up (a user's setup step): the search
    # split and the mask stage's tasks per warp for this batch
    tuned = batch.tune(None, stream)
    launches_per_step = batch.launches(cppflow.STAGE_ALL)

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- warm-up
    for _ in range(args.warmup):
        batch.run(cppflow.STAGE_ALL, stream)
    torch.cuda.synchronize()

    # ---- measured peaks (rank 0 runs the probe; its figures enter the rooflines it prints)
    peaks = measure_peaks(cppflow, torch, dev) if rank == 0 else None

    # ---- timed region: device-resident batched path, the stages bracketed by events
    stages = [cppflow.STAGE_MASK | cppflow.STAGE_LAYER_MIN, cppflow.STAGE_DP_FORWARD,
              cppflow.STAGE_BACKTRACK, cppflow.STAGE_LM, cppflow.STAGE_CHECK]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
          for _ in range(args.steps)]
    cppflow.counters_reset(stream)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        ev[s][0].record(stream)
        for k, stg in enumerate(stages):
            batch.run(stg, stream)
            ev[s][k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    counters = cppflow.counters_read()
    total_ms = ev[0][0].elapsed_time(ev[-1][-1])
    stage_ms = [[ev[s][k].elapsed_time(ev[s][k + 1]) for s in range(args.steps)]
                for k in range(len(stages))]
    pre_ms, dp_ms, bt_ms, lm_ms, chk_ms = stage_ms
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * B * args.steps / (total_ms / 1000.0)

    # ---- results valid?
    st = status.cpu().numpy()
    reps = [cppflow.report_from_bytes(rep[r].cpu().numpy().tobytes()) for r in range(B)]
    gpu_res = {"sel": sel.cpu().numpy(), "q": q_out.cpu().numpy(),
               "mjac": [r["mjac"] for r in reps], "max_pos": [r["max_pos"] for r in reps],
               "max_rot": [r["max_rot"] for r in reps]}
    valid = sum(int(r["valid"]) for r in reps)
    max_pos = max(r["max_pos"] for r in reps)
    max_rot = max(r["max_rot"] for r in reps)

    # ---- plain per-request path (one request at a time, one stream)
    n_plain = min(B, args.plain)
    pws = torch.empty(cppflow.plan_workspace_size(T, K, Kp, n), dtype=torch.uint8, device=dev)
    psel = torch.empty(T, dtype=torch.int32, device=dev)
    pbest = torch.empty(1, dtype=torch.float32, device=dev)
    pq = torch.empty(T, n, dtype=torch.float32, device=dev)
    perr = torch.empty(T, 2, dtype=torch.float64, device=dev)
    prep = torch.zeros(cppflow.REPORT_BYTES, dtype=torch.uint8, device=dev)
    pst = torch.zeros(1, dtype=torch.int32, device=dev)
    for r in range(min(2, n_plain)):
        cppflow.plan(robots[reqs[r].arm_seed - 100], P, cand_d[r], targ_d[r], K, pws, psel, pbest,
                     pq, perr, prep, pst, stream)
    torch.cuda.synchronize()
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n_plain)]
    for r in range(n_plain):
        pev[r][0].record(stream)
        cppflow.plan(robots[reqs[r].arm_seed - 100], P, cand_d[r], targ_d[r], K, pws, psel, pbest,
                     pq, perr, prep, pst, stream)
        pev[r][1].record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in pev)
    plain_total = pev[0][0].elapsed_time(pev[-1][1])
    plain = {"value": round(n_plain / (plain_total / 1000.0), 3), "unit": "plans/s",
             "p50_ms": round(lat[len(lat) // 2], 3),
             "p99_ms": round(lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)], 3),
             "requests": n_plain}

    # ---- end to end through the serving API: host inputs in, results in host memory out
    h2d = sum(c.numel() * 4 + t.numel() * 8 for c, t in zip(cand_h, targets_h))
    d2h_per_req = T * 4 + T * n * 4 + T * 16 + cppflow.REPORT_BYTES + 4
    cand_np = [c.numpy() for c in cand_h]     # pinned host memory, borrowed by the server
    targ_np = [t.numpy() for t in targets_h]
    e2e_steps = max(40, min(args.steps, 80))  # fill and drain of the pipeline amortised
    lat = []
    e2e_valid = 0

    def submit_step(srv):
        return [srv.submit(robots[reqs[r].arm_seed - 100], cand_np[r], targ_np[r], K, borrow=True)
                for r in range(B)]

    # The client keeps `serve_depth` steps in flight (it submits step s + depth - 1 before
    # it waits for the results of step s), as a serving front end would; every step's H2D
    # copies, batching, kernels and D2H copies lie inside the timed region.
    depth = max(1, args.serve_depth)
    gc.collect()
    gc.disable()  # no collection pause inside the timed client loop
    with cppflow.Server(P, device=local, hbm_budget=(depth + 1) * int(B * 6.5e6) + (256 << 20),
                        max_batch=args.serve_batch, max_inflight=args.serve_inflight,
                        pinned_bytes=64 << 20) as srv:
        for tk in submit_step(srv):              # one closed step warms the server up
            srv.wait(tk)
        t0 = time.perf_counter()
        pending = [submit_step(srv) for _ in range(min(depth - 1, e2e_steps))]
        for s_i in range(e2e_steps):
            if s_i + depth - 1 < e2e_steps:
                pending.append(submit_step(srv))
            outs = [srv.wait(tk) for tk in pending.pop(0)]
            lat += [o[1]["latency_ms"] for o in outs]
            e2e_valid += sum(int(o[1]["report"]["valid"]) for o in outs)
        e2e_total = time.perf_counter() - t0
        sstats = srv.stats()
    gc.enable()
    lat.sort()
    e2e = {"value": round(world * B * e2e_steps / e2e_total, 3), "unit": "plans/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(B * d2h_per_req),
           "path": "cpp_plan_submit (pinned host inputs, borrowed) -> continuous batching -> "
                   f"cpp_plan_wait (results in host memory); client keeps {depth} steps in flight",
           "server": {"max_batch": args.serve_batch, "max_inflight": args.serve_inflight},
           "steps_in_flight": depth,
           "p50_ms": round(lat[len(lat) // 2], 3),
           "p99_ms": round(lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)], 3),
           "valid_plans": f"{e2e_valid}/{B * e2e_steps}",
           "batches_per_step": round(sstats["batches"] / (e2e_steps + 1), 2), "steps": e2e_steps}

    # ---- rooflines: the search kernel (dominant) and the LM kernel, against the peaks
    # measured above by the library's throughput probe
    edges = B * (T - 1) * K * K
    ops_per_edge = 2 * n + 1
    dp_s = statistics.mean(dp_ms) / 1000.0
    achieved = edges * ops_per_edge / dp_s
    if peaks is not None:
        peak, basis = peaks["fp32_lane_ops_per_s"], (
            "measured: cpp_peak_probe FP32 add + max chains, best of 6 launches in this run "
            f"(SM clock median {peaks['clocks'].get('sm_mhz')} MHz during the probe)")
    else:
        peak, basis = 152 * 128 * 2070e6, "derived: 152 SMs x 128 FP32 lanes x 2070 MHz"
    roof = {"bound": "alu", "kernel": "dp3_forward_kernel", "achieved": round(achieved / 1e12, 3),
            "peak": round(peak / 1e12, 3), "unit": "T FP32 lane-ops/s",
            "frac": round(achieved / peak, 4),
            "traffic": DP3_TRAFFIC_BYTES if (B, T, K, n) == (304, 300, 512, 7) else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "algorithmic_bytes": B * T * Kp * (4 * n + 4) + B * T * synth.pad_k(K, 8) * 2,
            "ops": f"{ops_per_edge} FP32 ALU ops per edge (n sub, n-1 abs-max, add, min) x "
                   f"{edges:.4g} edges per launch",
            "peak_basis": basis, "kernel_ms": round(statistics.mean(dp_ms), 4),
            "edges_per_s": round(edges / dp_s, 1)}
    lm_iters_launch = counters["lm_iterations"] / args.steps
    lm_wp_launch = counters["lm_waypoints"] / args.steps
    lm_s = statistics.mean(lm_ms) / 1000.0
    lm_achieved = lm_iters_launch * lm_flops_per_iter(n) / lm_s
    roof_lm = None
    if peaks is not None:
        roof_lm = {"bound": "fp64", "kernel": "lm_kernel", "achieved": round(lm_achieved / 1e12, 4),
                   "peak": round(peaks["fp64_flops_per_s"] / 1e12, 4), "unit": "TFLOP/s (FP64)",
                   "frac": round(lm_achieved / peaks["fp64_flops_per_s"], 4),
                   "ops": f"{lm_flops_per_iter(n)} FP64 flops per waypoint-iteration x "
                          f"{lm_iters_launch:.0f} iterations per launch (library counters: "
                          f"{lm_wp_launch:.0f} waypoints, "
                          f"{lm_iters_launch / max(1.0, lm_wp_launch):.2f} iterations each)",
                   "peak_basis": "measured: cpp_peak_probe FP64 fma chains, best of 6 launches "
                                 "in this run",
                   "kernel_ms": round(statistics.mean(lm_ms), 4)}

    uneven = uneven_batch(cppflow, torch, dev, args.uneven) if args.uneven and rank == 0 else None
    coll = collision_leg(cppflow, torch, dev, args.collision) if args.collision and rank == 0 else None
    stress, stress_data = stress_leg(cppflow, torch, dev) if args.stress and rank == 0 else (None, None)
    mix = None
    if args.serve_rates and rank == 0:
        mix = serving_mix(cppflow, torch, dev, [float(x) for x in args.serve_rates.split(",")],
                          args.mix_pool, args.mix_seconds, args.mix_min, args.mix_plain_max)
    orc = None
    if rank == 0 and world == 1 and not args.no_cpu:
        orc = oracle_leg(arms, reqs, cand_h, targets_h, gpu_res, stress_data)
        if stress is not None and orc["stress_vs_oracle"] is not None:
            stress["vs_oracle"] = orc["stress_vs_oracle"]
    line = {"metric": METRIC, "value": round(value, 3), "unit": "plans/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": synth.SINGLE.name, "T": T, "K": K, "n": n,
                       "requests_per_step": B, "per_gpu_requests": B,
                       "l2": f"inputs larger than L2 ({B * T * n * Kp * 4 / 1e6:.0f} MB lattice per step)",
                       "lm_iters": P.lm_iters, "parallelism": f"replicas x{world}",
                       "tuned": {"heavy": tuned["heavy"], "alpha": round(tuned["alpha"], 4),
                                 "mask_tasks_per_warp": tuned["mask_tasks_per_warp"]}},
            "value_is": VALUE_IS,
            "stage_ms": {"mask_and_layer_min": round(statistics.mean(pre_ms), 4),
                         "dp_forward": round(statistics.mean(dp_ms), 4),
                         "backtrack": round(statistics.mean(bt_ms), 4),
                         "lm": round(statistics.mean(lm_ms), 4),
                         "check": round(statistics.mean(chk_ms), 4)},
            "plain_per_request": plain,
            "valid_plans": f"{valid}/{B}", "max_pos_err_m": max_pos, "max_rot_err_rad": max_rot,
            "dev_status_nonzero": int((st != 0).sum()),
            "roofline": roof, "roofline_lm": roof_lm, "peaks_measured": (
                None if peaks is None else
                {"fp32_lane_ops_per_s": peaks["fp32_lane_ops_per_s"],
                 "fp64_flops_per_s": peaks["fp64_flops_per_s"], "clocks": peaks["clocks"]}),
            "e2e": e2e, "clocks": clk,
            "gpu_launches": launches_per_step * args.steps}
    if uneven is not None:
        line["batched_uneven"] = uneven
    if coll is not None:
        line["collision_aware"] = coll
    if stress is not None:
        line["stress_precision"] = stress
    if mix is not None:
        line["serving_mix"] = {"workload": "serving mix: T = floor(exp U(ln 50, ln 2000)), "
                                           "K in {128, 256, 512, 1024}, 7-DoF, open-loop Poisson "
                                           "arrivals; served = cpp_plan_submit (continuous "
                                           "batching), plain = the same trace through "
                                           "cpp_plan_host one request at a time; host copies "
                                           "inside both latencies; first 10 % dropped",
                               "rates": mix}
    if orc is not None:
        line["cpu_baseline"] = orc["cpu_baseline"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=304)
    ap.add_argument("--plain", type=int, default=32, help="requests timed on the plain path")
    ap.add_argument("--serve-batch", type=int, default=38, help="server: requests per launch")
    ap.add_argument("--serve-inflight", type=int, default=16, help="server: launches in flight")
    ap.add_argument("--serve-depth", type=int, default=3,
                    help="e2e client: steps of requests in flight")
    ap.add_argument("--uneven", type=int, default=256,
                    help="requests of the batched uneven leg (0: skip)")
    ap.add_argument("--collision", type=int, default=304,
                    help="requests of the collision-aware leg (0: skip)")
    ap.add_argument("--stress", type=int, default=1,
                    help="run the 9-DoF T=2000 K=1024 precision leg (0: skip)")
    ap.add_argument("--serve-rates", default="100,1000,5000", help="Poisson rates (req/s) of the "
                    "serving mix, comma separated; empty to skip")
    ap.add_argument("--mix-pool", type=int, default=512, help="distinct requests in the mix pool")
    ap.add_argument("--mix-seconds", type=float, default=10.0,
                    help="seconds of reported arrivals per rate (at least --mix-min requests)")
    ap.add_argument("--mix-min", type=int, default=1000)
    ap.add_argument("--mix-plain-max", type=int, default=10000,
                    help="reported requests of the plain arm per rate (a prefix of the trace)")
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "cuda":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "cuda" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group(backend)
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_cuda(args, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
