// lm.cu -- Levenberg-Marquardt refinement of the searched trajectory (paper
// §III-C) and the FP64 trajectory check (§II constraints and metrics).
//
// The pose residual of waypoint i depends on q_i only, so its Jacobian is block
// diagonal and every waypoint is an independent damped n x n problem. One
// thread owns one waypoint (32 waypoints per warp):
//   * the DH chain runs in FP32 (or FP64 in the all-FP64 mode) and records the
//     frames (z_j, o_j); column j of the geometric Jacobian is
//     [z_j x (p_e - o_j); z_j],
//   * J^T J + lambda I and J^T e are accumulated in FP64 registers one Jacobian
//     row at a time (products of FP32 values are exact in FP64),
//   * the Cholesky factorisation and both triangular solves run in FP64 registers,
//   * the trial q' = clamp(q + delta, lo, hi) is accepted iff F(q') < F(q)
//     (F = |e|^2 / 2 summed in FP64), with lambda / 10 or * 10.
// Why a thread and not a warp per waypoint: GB300 issues FP64 at about two lanes
// per clock per SM, so an FP64 warp instruction costs the same ~16 cycles
// whether one lane or 32 do useful work. Spreading one waypoint's n x n algebra
// over a warp leaves most lanes of every FP64 instruction idle; a thread per
// waypoint fills all 32.
// The joint state is held in FP64; q_out is its FP32 rounding.
#include <type_traits>

#include "collide.cuh"
#include "internal.h"

namespace cppflow {

constexpr int kLmThreads = 32;   // one warp per block: a lone request spreads over T / 32 SMs
constexpr int kChkThreads = 64;
constexpr int kChkCluster = 8;   // CTAs per request in the check

struct LmArgs {
  double lambda0, lambda_up, lambda_down, lambda_min, lambda_max, freeze_step, freeze_cost;
  int iters;
  uint32_t free_mask;
  int want_err;  // write the FP64 pose error of q_out (skipped when a check follows)
  int from_out;  // start from q_out (a later pose phase of the alternation) instead of q_in
};

struct CheckArgs {
  double tau_pos, tau_rot, jump_max;
};



// Work counters of the LM stage (cpp_counters_read): one atomic add per warp.
__device__ cpp_counters_t g_lm_counters;

__device__ __forceinline__ float to_angle(double q, const RobotF& rb, int j) {
  return (float)q + rb.th0[j];
}
__device__ __forceinline__ double to_angle(double q, const RobotD& rb, int j) {
  return q + rb.th0[j];
}

template <class F>
struct RobotFor;
template <>
struct RobotFor<float> {
  __device__ static const RobotF& get(const RobotF& f, const RobotD&) { return f; }
};
template <>
struct RobotFor<double> {
  __device__ static const RobotD& get(const RobotF&, const RobotD& d) { return d; }
};

// FK of q; e = [p_t - p; log(R_t R^T)]; returns F = |e|^2 / 2 summed in FP64.
// With FRAMES the frames (z_j, o_j) before each joint and the end position are kept.
template <int NJ, bool FRAMES, class F, class RB>
__device__ __forceinline__ double lm_eval(const RB& rb, int n, const double* q, const F Rt[9],
                                          const F pt[3], F e[6], F (*z)[3], F (*o)[3], F* pe) {
  constexpr int MJ = NJ ? NJ : kMaxJ;
  F R[9], p[3];
  pose_identity(R, p);
#pragma unroll
  for (int j = 0; j < MJ; ++j) {
    if (!NJ && j >= n) break;
    if (FRAMES) {
      z[j][0] = R[2]; z[j][1] = R[5]; z[j][2] = R[8];
      o[j][0] = p[0]; o[j][1] = p[1]; o[j][2] = p[2];
    }
    F s, c;
    sincos_t(to_angle(q[j], rb, j), &s, &c);
    dh_step(R, p, c, s, (F)rb.ca[j], (F)rb.sa[j], (F)rb.a[j], (F)rb.d[j]);
  }
  if (FRAMES) { pe[0] = p[0]; pe[1] = p[1]; pe[2] = p[2]; }
  e[0] = pt[0] - p[0]; e[1] = pt[1] - p[1]; e[2] = pt[2] - p[2];
  F M[9];  // M = R_t R^T
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      M[3 * a + b] = Rt[3 * a] * R[3 * b] + Rt[3 * a + 1] * R[3 * b + 1] + Rt[3 * a + 2] * R[3 * b + 2];
  log_rot<F>(M, e + 3, F(1e-6), sizeof(F) == 4 ? F(1e-3) : F(1e-6));
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) s += (double)e[k] * (double)e[k];
  return 0.5 * s;
}

__global__ void __launch_bounds__(32) robot_views_kernel(const cpp_robot_t* robots, RobotViews* views) {
  __shared__ RobotF rf;
  __shared__ RobotD rd;
  stage_robot(robots[blockIdx.x], 0.0, &rf, &rd);
  __syncthreads();
  if (threadIdx.x == 0) {
    views[blockIdx.x].f = rf;
    views[blockIdx.x].d = rd;
  }
}

// One LM refinement kernel for single requests and batches. Each lane carries
// the state of one waypoint (q, the target, F, lambda, the iteration count) and
// every trip of the loop runs one iteration of its waypoint, so the lanes of a
// warp advance together whatever waypoints they hold. A single request gives
// each lane one waypoint (one warp per 32 waypoints). A batch runs a persistent
// grid of one-warp blocks whose lanes take waypoints from a counter over the
// batch's waypoints (prefix sums over its requests) as their previous ones
// finish, so a warp no longer waits for its slowest waypoint and no second wave
// of blocks follows the first. The arithmetic of every waypoint is the same in
// both, so a request's result does not depend on its batch.
template <int NJ, class F, class Src>
__global__ void __launch_bounds__(kLmThreads) lm_kernel(const __grid_constant__ Src src,
                                                         const LmArgs a) {
  pdl_trigger();
  pdl_wait();
  constexpr int MJ = NJ ? NJ : kMaxJ;
  constexpr int MT = MJ * (MJ + 1) / 2;  // packed lower triangle
  constexpr bool DYN = std::is_same<Src, BatchSrc>::value;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  __shared__ RobotF srf;
  __shared__ RobotD srd;
  // J^T J (packed lower triangle) and J^T e of each lane's current q, kept across
  // rejected steps: a rejected step leaves q, and so J and e, unchanged, and the
  // next iteration only needs the factorisation with the larger lambda
  __shared__ double sA[MT * kLmThreads], sg[MJ * kLmThreads];
  if (!DYN) {
    stage_robot(src.rob(src.req(0).robot), 0.0, &srf, &srd);
    __syncthreads();
  }

  // state of the lane's waypoint
  bool have = false, exhausted = false, cached = false;
  const Req* rq = nullptr;
  const RobotF* rfp = &srf;
  const RobotD* rdp = &srd;
  int i = 0, it = 0;
  F Rt[9], pt[3];
  double q[MJ];
  double Fc = 0.0, lam = 0.0;
  unsigned worked = 0, waypoints = 0;  // counters of this lane

  auto start = [&](int r, int w) {  // take waypoint w of request r
    rq = &src.req(r);
    if constexpr (DYN) {
      rfp = &src.lm.views[rq->robot].f;
      rdp = &src.lm.views[rq->robot].d;
    }
    i = w;
    const int n = NJ ? NJ : rdp->n;
    double R[9];
    const double* t7 = rq->targets + 7 * (size_t)i;
    quat_to_rot(t7 + 3, R);
#pragma unroll
    for (int k = 0; k < 9; ++k) Rt[k] = (F)R[k];
    pt[0] = (F)t7[0]; pt[1] = (F)t7[1]; pt[2] = (F)t7[2];
    const float* q_src = a.from_out ? rq->q_out : rq->q_in;
#pragma unroll
    for (int j = 0; j < MJ; ++j) q[j] = (NJ || j < n) ? (double)q_src[(size_t)i * n + j] : 0.0;
    F e[6];
    Fc = lm_eval<NJ, false, F>(RobotFor<F>::get(*rfp, *rdp), n, q, Rt, pt, e, nullptr, nullptr,
                               nullptr);
    lam = a.lambda0;
    it = 0;
    have = true;
    cached = false;
    ++waypoints;
  };

  auto finish = [&]() {  // deliver the waypoint's result
    const RobotD& rd = *rdp;
    const int n = NJ ? NJ : rd.n;
#pragma unroll
    for (int j = 0; j < MJ; ++j)
      if (NJ || j < n) rq->q_out[(size_t)i * n + j] = (float)q[j];
    if (a.want_err && rq->pose_err) {
      // FP64 pose error of the delivered (FP32-rounded) configuration
      double qq[kMaxJ], R[9], p[3], RtD[9];
      for (int j = 0; j < n; ++j) qq[j] = (double)(float)q[j];
      fk_f64(rd, qq, R, p);
      const double* t7 = rq->targets + 7 * (size_t)i;
      quat_to_rot(t7 + 3, RtD);
      const double dx = p[0] - t7[0], dy = p[1] - t7[1], dz = p[2] - t7[2];
      rq->pose_err[2 * (size_t)i] = sqrt(dx * dx + dy * dy + dz * dz);
      rq->pose_err[2 * (size_t)i + 1] = geodesic<double>(RtD, R);
    }
    have = false;
  };

  if (!DYN) {  // a single request: one waypoint per lane
    const int w = blockIdx.x * kLmThreads + lane;
    if (w < src.req(0).T) start(0, w);
    exhausted = true;
  }

  for (;;) {
    if constexpr (DYN) if (!exhausted) {
      const LmAux& aux = src.lm;
      // lanes without a waypoint take the next ones of the batch (one atomic per warp)
      const unsigned need = __ballot_sync(FULL, !have);
      if (need) {
        const int leader = __ffs(need) - 1, cnt = __popc(need);
        int base = 0;
        if (lane == leader) base = atomicAdd(aux.counter, cnt);
        base = __shfl_sync(FULL, base, leader);
        if (!have) {
          const int w = base + __popc(need & ((1u << lane) - 1u));
          if (w < aux.total) {
            int lo = 0, hi = aux.nreq - 1;  // request r with wp_begin[r] <= w < wp_begin[r + 1]
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (aux.wp_begin[mid] <= w) lo = mid; else hi = mid - 1;
            }
            start(lo, w - aux.wp_begin[lo]);
          }
        }
        if (base + cnt >= aux.total) exhausted = true;  // base and cnt are the same in every lane
      }
    }
    if (!__any_sync(FULL, have)) break;
    if (!have) continue;

    // one LM iteration of the lane's waypoint
    const auto& rb = RobotFor<F>::get(*rfp, *rdp);
    const RobotD& rd = *rdp;
    const int n = NJ ? NJ : rd.n;
    if (it >= a.iters || Fc < a.freeze_cost) { finish(); continue; }
    ++worked;
    double A[MT], g[MJ];
    if (cached) {
#pragma unroll
      for (int t = 0; t < MT; ++t) A[t] = sA[t * kLmThreads + lane];
#pragma unroll
      for (int j = 0; j < MJ; ++j) g[j] = sg[j * kLmThreads + lane];
    } else {
    F e[6];
    F z[MJ][3], o[MJ][3], pe[3];
    lm_eval<NJ, true, F>(rb, n, q, Rt, pt, e, z, o, pe);
    // J^T J (packed lower triangle) and J^T e, one Jacobian row at a time
#pragma unroll
    for (int t = 0; t < MT; ++t) A[t] = 0.0;
#pragma unroll
    for (int j = 0; j < MJ; ++j) g[j] = 0.0;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double Jr[MJ];
#pragma unroll
      for (int j = 0; j < MJ; ++j) {
        F v = F(0);
        if ((NJ || j < n) && ((a.free_mask >> j) & 1u)) {
          const F dx = pe[0] - o[j][0], dy = pe[1] - o[j][1], dz = pe[2] - o[j][2];
          v = r == 0 ? z[j][1] * dz - z[j][2] * dy
            : r == 1 ? z[j][2] * dx - z[j][0] * dz
            : r == 2 ? z[j][0] * dy - z[j][1] * dx
            : z[j][r - 3];
        }
        Jr[j] = (double)v;
      }
      const double er = (double)e[r];
#pragma unroll
      for (int x = 0; x < MJ; ++x) {
        g[x] += Jr[x] * er;
#pragma unroll
        for (int y = 0; y <= x; ++y) A[x * (x + 1) / 2 + y] += Jr[x] * Jr[y];
      }
    }
#pragma unroll
    for (int t = 0; t < MT; ++t) sA[t * kLmThreads + lane] = A[t];
#pragma unroll
    for (int j = 0; j < MJ; ++j) sg[j * kLmThreads + lane] = g[j];
    cached = true;
    }
    // Cholesky of J^T J + lam I, left-looking, in place: L_jj = sqrt(A_jj + lam - sum L_jm^2),
    // L_xj = (A_xj - sum L_xm L_jm) / L_jj. Only 1 / L_jj is used (the off-diagonal
    // entries and both solves multiply by it), so each pivot takes one reciprocal
    // square root (rsqrt, within 1 ulp) where a square root and a division would
    // take two FP64 sequences on GB300's narrow FP64 pipe.
    bool ok = true;
    double inv[MJ];
#pragma unroll
    for (int j = 0; j < MJ; ++j) {
      if (!NJ && j >= n) { inv[j] = 0.0; continue; }
      double d = A[j * (j + 1) / 2 + j] + lam;
#pragma unroll
      for (int m = 0; m < j; ++m) d -= A[j * (j + 1) / 2 + m] * A[j * (j + 1) / 2 + m];
      ok = ok && (d > 0.0) && isfinite(d);
      inv[j] = rsqrt(d);
#pragma unroll
      for (int x = j + 1; x < MJ; ++x) {
        if (!NJ && x >= n) break;
        double t = A[x * (x + 1) / 2 + j];
#pragma unroll
        for (int m = 0; m < j; ++m) t -= A[x * (x + 1) / 2 + m] * A[j * (j + 1) / 2 + m];
        A[x * (x + 1) / 2 + j] = t * inv[j];
      }
    }
    if (!ok) {
      lam = fmin(lam * a.lambda_up, a.lambda_max);
      ++it;
      continue;
    }
    // L y = g, then L^T x = y (x overwrites g)
#pragma unroll
    for (int x = 0; x < MJ; ++x) {
      if (!NJ && x >= n) break;
      double t = g[x];
#pragma unroll
      for (int m = 0; m < x; ++m) t -= A[x * (x + 1) / 2 + m] * g[m];
      g[x] = t * inv[x];
    }
#pragma unroll
    for (int x = MJ - 1; x >= 0; --x) {
      if (!NJ && x >= n) continue;
      double t = g[x];
#pragma unroll
      for (int m = x + 1; m < MJ; ++m) {
        if (!NJ && m >= n) break;
        t -= A[m * (m + 1) / 2 + x] * g[m];
      }
      g[x] = t * inv[x];
    }
    double mx = 0.0;
#pragma unroll
    for (int j = 0; j < MJ; ++j)
      if (NJ || j < n) mx = fmax(mx, fabs(g[j]));
    if (mx < a.freeze_step) { finish(); continue; }
    double qt[MJ];
#pragma unroll
    for (int j = 0; j < MJ; ++j) {
      double v = q[j] + g[j];
      if (NJ || j < n) {
        if (v < rd.lo[j]) v = rd.lo[j];
        if (v > rd.hi[j]) v = rd.hi[j];
      }
      qt[j] = v;
    }
    F et[6];
    const double Ft = lm_eval<NJ, false, F>(rb, n, qt, Rt, pt, et, nullptr, nullptr, nullptr);
    if (Ft < Fc) {
#pragma unroll
      for (int j = 0; j < MJ; ++j) q[j] = qt[j];
      Fc = Ft;
      lam = fmax(lam / a.lambda_down, a.lambda_min);
      cached = false;  // q moved: J and e change
    } else {
      lam = fmin(lam * a.lambda_up, a.lambda_max);
    }
    ++it;
  }
  {  // work counters: one atomic add per warp
    const unsigned sw = __reduce_add_sync(FULL, worked), sp = __reduce_add_sync(FULL, waypoints);
    if (lane == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&g_lm_counters.lm_iterations),
                (unsigned long long)sw);
      atomicAdd(reinterpret_cast<unsigned long long*>(&g_lm_counters.lm_waypoints),
                (unsigned long long)sp);
    }
  }
}

// ------------------------------------------------------------------ FP64 check
// Waypoints are split over kChkCluster groups of 64 threads: group c takes
// waypoints c * 64 + t + 512 k. Each group reduces its two warps in a fixed
// order into one partial, and the 8 partials combine in group order. The FP64
// FK of a waypoint costs a few hundred FP64 operations and GB300 issues FP64 at
// two lanes per clock per SM, so a lone request (or a small batch) runs the
// groups as the CTAs of a thread-block cluster on 8 SMs, the partials combined
// through distributed shared memory (CL = true); a large batch runs them as
// the warps of one 512-thread CTA per request (CL = false). Both orders are the
// same, so a request's report is the same alone and in any batch.
template <bool CL, class Src>
__global__ void __launch_bounds__(CL ? kChkThreads : kChkThreads * kChkCluster)
    check_kernel(const __grid_constant__ Src src, const CheckArgs a) {
  pdl_trigger();
  pdl_wait();
  constexpr int NWARP = (CL ? kChkThreads : kChkThreads * kChkCluster) / 32;
  const Req& rq = src.req(CL ? blockIdx.x / kChkCluster : blockIdx.x);
  const uint32_t crank = CL ? cluster_rank() : 0;
  __shared__ RobotD rd;
  __shared__ double red[5][NWARP];
  __shared__ int redi[3][NWARP];
  __shared__ double part[CL ? 1 : kChkCluster][5];  // group partials
  __shared__ int parti[CL ? 1 : kChkCluster][3];
  stage_robot(src.rob(rq.robot), 0.0, nullptr, &rd);
  __syncthreads();
  const int n = rd.n, T = rq.T, tid = threadIdx.x;
  const int group = CL ? (int)crank : tid / kChkThreads, gt = CL ? tid : tid % kChkThreads;
  double mpos = 0, mrot = 0, mjac = 0, slinf = 0, tlen = 0;
  int npose = 0, nlim = 0, njump = 0;
  for (int i = group * kChkThreads + gt; i < T; i += kChkCluster * kChkThreads) {
    double q[kMaxJ], R[9], p[3], Rt[9];
    for (int j = 0; j < n; ++j) q[j] = (double)rq.q_out[(size_t)i * n + j];
    fk_f64(rd, q, R, p);
    const double* t7 = rq.targets + 7 * (size_t)i;
    quat_to_rot(t7 + 3, Rt);
    const double dx = p[0] - t7[0], dy = p[1] - t7[1], dz = p[2] - t7[2];
    const double pos = sqrt(dx * dx + dy * dy + dz * dz);
    const double rot = geodesic<double>(Rt, R);
    if (rq.pose_err) {
      rq.pose_err[2 * (size_t)i] = pos;
      rq.pose_err[2 * (size_t)i + 1] = rot;
    }
    mpos = fmax(mpos, pos);
    mrot = fmax(mrot, rot);
    if (!(pos <= a.tau_pos && rot <= a.tau_rot)) ++npose;
    bool out = false;
    for (int j = 0; j < n; ++j)
      if (!(q[j] >= rd.lo[j] && q[j] <= rd.hi[j])) out = true;
    nlim += out;
    if (i + 1 < T) {
      double linf = 0.0;
      for (int j = 0; j < n; ++j) {
        const double dj = fabs((double)rq.q_out[(size_t)(i + 1) * n + j] - q[j]);
        linf = fmax(linf, dj);
        tlen += dj;
      }
      mjac = fmax(mjac, linf);
      slinf += linf;
      if (linf > a.jump_max) ++njump;
    }
  }
  // fixed-order reduction: warps by shuffles, a group's two warps in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mpos = fmax(mpos, __shfl_xor_sync(0xffffffffu, mpos, o));
    mrot = fmax(mrot, __shfl_xor_sync(0xffffffffu, mrot, o));
    mjac = fmax(mjac, __shfl_xor_sync(0xffffffffu, mjac, o));
    slinf += __shfl_xor_sync(0xffffffffu, slinf, o);
    tlen += __shfl_xor_sync(0xffffffffu, tlen, o);
    npose += __shfl_xor_sync(0xffffffffu, npose, o);
    nlim += __shfl_xor_sync(0xffffffffu, nlim, o);
    njump += __shfl_xor_sync(0xffffffffu, njump, o);
  }
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) {
    red[0][warp] = mpos; red[1][warp] = mrot; red[2][warp] = mjac;
    red[3][warp] = slinf; red[4][warp] = tlen;
    redi[0][warp] = npose; redi[1][warp] = nlim; redi[2][warp] = njump;
  }
  __syncthreads();
  constexpr int WPG = kChkThreads / 32;  // warps per group
  if (gt == 0) {
    const int w0 = CL ? 0 : group * WPG, slot = CL ? 0 : group;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int c[3] = {0, 0, 0};
    for (int w = w0; w < w0 + WPG; ++w) {
      for (int k = 0; k < 3; ++k) v[k] = fmax(v[k], red[k][w]);
      v[3] += red[3][w];
      v[4] += red[4][w];
      for (int k = 0; k < 3; ++k) c[k] += redi[k][w];
    }
    for (int k = 0; k < 5; ++k) part[slot][k] = v[k];
    for (int k = 0; k < 3; ++k) parti[slot][k] = c[k];
  }
  if (CL)
    cluster_barrier();  // every CTA's partial is visible to CTA 0
  else
    __syncthreads();
  if (crank == 0 && tid == 0 && rq.report) {
    cpp_report_t r;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int c[3] = {0, 0, 0};
    for (int g = 0; g < kChkCluster; ++g) {
      for (int k = 0; k < 5; ++k) {
        const double x = CL ? ld_peer_f64(map_peer(smem_u32(&part[0][k]), (uint32_t)g)) : part[g][k];
        v[k] = k < 3 ? fmax(v[k], x) : v[k] + x;
      }
      for (int k = 0; k < 3; ++k)
        c[k] += CL ? ld_peer_s32(map_peer(smem_u32(&parti[0][k]), (uint32_t)g)) : parti[g][k];
    }
    r.max_pos = v[0]; r.max_rot = v[1]; r.mjac = v[2]; r.sum_linf = v[3]; r.traj_len = v[4];
    r.n_pose_fail = c[0]; r.n_limit_fail = c[1]; r.n_jump_fail = c[2];
    r.valid = (r.n_pose_fail == 0 && r.n_limit_fail == 0 && r.n_jump_fail == 0) ? 1 : 0;
    *rq.report = r;
  }
  if (CL) cluster_barrier();  // no CTA leaves before CTA 0 has read its partial
}

// ------------------------------------------------------------------ trajectory-length step
// §III-C non-stationary objective: pose-only LM phases alternate with single
// steps on the differencing residual r_diff = [q_{i+1} - q_i] (requests with a
// collision model add its rows: smooth_geo_kernel below). A step is taken only when every waypoint is
// within tau_pos / tau_rot (FP64 FK of q_out). It is the damped least-squares
// step delta = -(J^T J + lambda_d I)^{-1} J^T r_diff; J^T J is block tridiagonal
// with blocks (c_i + lambda_d) I on the diagonal (c_i = 1 at the ends, 2 inside)
// and -I beside it. Blocks that are multiples of I never mix joints, so the
// block Thomas recursion is exactly n scalar recursions, one per lane:
//   s_0 = a_0,  s_i = a_i - 1 / s_{i-1};   y_0 = b_0,  y_i = b_i + y_{i-1} / s_{i-1}
//   delta_{T-1} = y_{T-1} / s_{T-1},       delta_i = (y_i + delta_{i+1}) / s_i
// with b_i = (q_{i+1} - q_i) - (q_i - q_{i-1}) (absent terms 0), then
// q' = clamp(q + delta, lo, hi), stored in FP32. One warp per request; FP64;
// 1 / s_i and y_i are kept in shared memory ((n + 1) T doubles).
struct SmoothArgs {
  double tau_pos, tau_rot, lambda_d;
  double coll_margin, coll_weight;  // collision rows: w (margin - d) where d < margin
};

// The trajectory-length step of one request with scalar-identity blocks: lane j
// (< n) runs the Thomas recursion of joint j over T in FP64 (inv_s: [T] 1 / s_i,
// the same in every lane; y: [T][n]) and stores clamp(q + delta) in FP32.
__device__ __forceinline__ void scalar_thomas(const Req& rq, const RobotD& rd, double lambda_d,
                                              double* inv_s, double* y, int lane) {
  const int n = rd.n, T = rq.T;
  if (lane >= n) return;
  const int j = lane;
  float* qc = rq.q_out + j;   // column j, stride n
  double qp = 0.0, qi = (double)qc[0], ip = 0.0, yp = 0.0;
  for (int i = 0; i < T; ++i) {
    const double qn = i + 1 < T ? (double)qc[(size_t)(i + 1) * n] : 0.0;
    const double c = (i > 0 ? 1.0 : 0.0) + (i + 1 < T ? 1.0 : 0.0);
    const double b = (i + 1 < T ? qn - qi : 0.0) - (i > 0 ? qi - qp : 0.0);
    const double s = c + lambda_d - (i > 0 ? ip : 0.0);
    const double yi = b + (i > 0 ? yp * ip : 0.0);
    ip = 1.0 / s;
    yp = yi;
    if (j == 0) inv_s[i] = ip;  // the same in every lane
    y[(size_t)i * n + j] = yi;
    qp = qi;
    qi = qn;
  }
  __syncwarp((1u << n) - 1u);
  double d = 0.0;
  const double lo = rd.lo[j], hi = rd.hi[j];
  for (int i = T - 1; i >= 0; --i) {
    d = (y[(size_t)i * n + j] + (i + 1 < T ? d : 0.0)) * inv_s[i];
    const double v = fmin(fmax((double)qc[(size_t)i * n] + d, lo), hi);
    qc[(size_t)i * n] = (float)v;
  }
}

template <class Src>
__global__ void __launch_bounds__(32) smooth_kernel(const __grid_constant__ Src src,
                                                     const SmoothArgs a) {
  const Req& rq = src.req(blockIdx.x);
  if (src.geom(rq) && rq.smooth_ws) return;  // smooth_geo_kernel's request
  extern __shared__ double sm_s[];
  __shared__ RobotD rd;
  stage_robot(src.rob(rq.robot), 0.0, nullptr, &rd);
  __syncthreads();
  const int n = rd.n, T = rq.T, lane = threadIdx.x;
  bool ok = true;
  for (int i = lane; i < T; i += 32) {
    double q[kMaxJ], R[9], p[3], Rt[9];
    for (int j = 0; j < n; ++j) q[j] = (double)rq.q_out[(size_t)i * n + j];
    fk_f64(rd, q, R, p);
    const double* t7 = rq.targets + 7 * (size_t)i;
    quat_to_rot(t7 + 3, Rt);
    const double dx = p[0] - t7[0], dy = p[1] - t7[1], dz = p[2] - t7[2];
    const double pos = sqrt(dx * dx + dy * dy + dz * dz);
    const double rot = geodesic<double>(Rt, R);
    ok = ok && pos <= a.tau_pos && rot <= a.tau_rot;
  }
  if (!__all_sync(0xffffffffu, ok) || T < 2) return;
  scalar_thomas(rq, rd, a.lambda_d, sm_s, sm_s + T, lane);
}

size_t smooth_smem_bytes(int T, int n) { return (size_t)T * (n + 1) * sizeof(double); }

// The trajectory-length step with the collision rows of r_diff (§III-C), for a
// request with a collision model. Rows: for every listed pair and every
// capsule-box combination with clearance d < margin, the hinge w (margin - d),
// whose gradient follows the envelope theorem, -w n . (dx_u/dq - dx_v/dq) with n
// the unit vector between the closest points and dx/dq_j = z_j x (x - o_j) for
// a point on a frame that joint j moves (the box point fixed); rows whose closest
// points are within 1e-6 m (touching or interpenetrating: no direction) are
// skipped. Each row touches one waypoint, so it adds g g^T to that waypoint's
// diagonal block and g r to its right-hand side: the normal equations stay block tridiagonal, now with
// full n x n diagonal blocks D_i = (c_i + lambda_d) I + G_i and -I beside them.
// One block of 4 warps per request:
//   phase 1, threads over waypoints: the FP64 gate (every waypoint within tau),
//     FP32 FK with frames and capsules, the rows, G_i and J^T r in FP64 to scratch;
//   phase 2, warp 0, the block Thomas recursion over T in FP64:
//     S_0 = D_0, S_i = D_i - S_{i-1}^{-1};  y_0 = b_0, y_i = b_i + S_{i-1}^{-1} y_{i-1}
//     (S_i^{-1} by Gauss-Jordan elimination without pivoting, which is stable for
//     a symmetric positive definite S_i and has its pivots positive; the lanes
//     share the n^2 entries, so a pivot costs one reciprocal and one update per
//     entry on the serial path), then x_{T-1} = S^{-1} y,
//     x_i = S_i^{-1} (y_i + x_{i+1}) (lane c: component c), q' = clamp(q + x) in FP32.
//     The blocks of step i + 1 are loaded during step i.
constexpr float kMinDir = 1e-6f;  // m: closest points nearer than this give no direction
constexpr int kSmoothGeoThreads = 128;
constexpr int kGjPerLane = (kMaxJ * kMaxJ + 31) / 32;  // matrix entries per lane

template <class Src>
__global__ void __launch_bounds__(kSmoothGeoThreads) smooth_geo_kernel(const __grid_constant__ Src src,
                                                         const SmoothArgs a) {
  const Req& rq = src.req(blockIdx.x);
  const GeoF* gsrc = src.geom(rq);
  if (!gsrc || !rq.smooth_ws) return;
  __shared__ RobotF rf;
  __shared__ RobotD rd;
  __shared__ GeoF g;
  __shared__ double Sb[2][kMaxJ * kMaxJ];  // S_i, inverted in place; S_{i-1}^{-1}
  __shared__ double yb[2][kMaxJ], xs[kMaxJ];
  stage_robot(src.rob(rq.robot), 0.0, &rf, &rd);
  {
    const uint32_t* from = reinterpret_cast<const uint32_t*>(gsrc);
    uint32_t* to = reinterpret_cast<uint32_t*>(&g);
    for (int w = threadIdx.x; w < (int)(sizeof(GeoF) / 4); w += kSmoothGeoThreads) to[w] = from[w];
  }
  __syncthreads();
  const int n = rd.n, T = rq.T, tid = threadIdx.x, lane = tid & 31, NP = n * (n + 1) / 2;
  double* Gh = rq.smooth_ws;                       // [T][NP + n]
  double* Wg = Gh + (size_t)T * (NP + n);          // [T][n * n]
  double* Yg = Wg + (size_t)T * n * n;             // [T][n]
  const float margin = (float)a.coll_margin, wt = (float)a.coll_weight;

  bool ok = true, any_rows = false;
  for (int i = tid; i < T; i += kSmoothGeoThreads) {
    double qd[kMaxJ], R[9], p[3], Rt[9];
    float qf[kMaxJ];
    for (int j = 0; j < n; ++j) { qf[j] = rq.q_out[(size_t)i * n + j]; qd[j] = (double)qf[j]; }
    fk_f64(rd, qd, R, p);
    const double* t7 = rq.targets + 7 * (size_t)i;
    quat_to_rot(t7 + 3, Rt);
    const double dx = p[0] - t7[0], dy = p[1] - t7[1], dz = p[2] - t7[2];
    ok = ok && sqrt(dx * dx + dy * dy + dz * dz) <= a.tau_pos && geodesic<double>(Rt, R) <= a.tau_rot;
    // FP32 frames and capsules
    float Rf[9], pf[3], z[kMaxJ][3], o[kMaxJ][3], cA[kMaxCaps][3], cB[kMaxCaps][3];
    pose_identity(Rf, pf);
    place_caps(g, 0, Rf, pf, cA, cB);
    for (int j = 0; j < n; ++j) {
      z[j][0] = Rf[2]; z[j][1] = Rf[5]; z[j][2] = Rf[8];
      o[j][0] = pf[0]; o[j][1] = pf[1]; o[j][2] = pf[2];
      float sj, cj;
      sincosf(qf[j] + rf.th0[j], &sj, &cj);
      dh_step(Rf, pf, cj, sj, rf.ca[j], rf.sa[j], rf.a[j], rf.d[j]);
      place_caps(g, j + 1, Rf, pf, cA, cB);
    }
    double G[kMaxJ * (kMaxJ + 1) / 2], h[kMaxJ];
    for (int k = 0; k < NP; ++k) G[k] = 0.0;
    for (int k = 0; k < n; ++k) h[k] = 0.0;
    // one row: residual res, unit direction nv, points xu (frame fu) minus xv (frame fv, or -1)
    auto add_row = [&](float res, const float nv[3], const float xu[3], int fu, const float xv[3],
                       int fv) {
      float row[kMaxJ];
      for (int j = 0; j < n; ++j) {
        float v = 0.f;
        if (fu > j) {
          const float rx = xu[0] - o[j][0], ry = xu[1] - o[j][1], rz = xu[2] - o[j][2];
          v += nv[0] * (z[j][1] * rz - z[j][2] * ry) + nv[1] * (z[j][2] * rx - z[j][0] * rz) +
               nv[2] * (z[j][0] * ry - z[j][1] * rx);
        }
        if (fv > j) {
          const float rx = xv[0] - o[j][0], ry = xv[1] - o[j][1], rz = xv[2] - o[j][2];
          v -= nv[0] * (z[j][1] * rz - z[j][2] * ry) + nv[1] * (z[j][2] * rx - z[j][0] * rz) +
               nv[2] * (z[j][0] * ry - z[j][1] * rx);
        }
        row[j] = -wt * v;
      }
      int k = 0;
      for (int r = 0; r < n; ++r) {
        h[r] += (double)row[r] * (double)res;
        for (int c = 0; c <= r; ++c) G[k++] += (double)row[r] * (double)row[c];
      }
    };
    for (int k = 0; k < g.n_pairs; ++k) {
      const int u = g.pu[k], v = g.pv[k];
      if (!aabb_meet(cA[u], cB[u], g.r[u] + margin, cA[v], cB[v], g.r[v] + 1e-5f)) continue;
      float su, tv;
      const float dist = sqrtf(seg_seg_d2_st(cA[u], cB[u], cA[v], cB[v], su, tv));
      const float d = dist - g.r[u] - g.r[v];
      if (!(d < margin) || dist <= kMinDir) continue;
      float xu[3], xv[3], nv[3];
      for (int c = 0; c < 3; ++c) {
        xu[c] = cA[u][c] + su * (cB[u][c] - cA[u][c]);
        xv[c] = cA[v][c] + tv * (cB[v][c] - cA[v][c]);
        nv[c] = (xu[c] - xv[c]) / dist;
      }
      // frame of a capsule: the f with frame_begin[f] <= c < frame_begin[f + 1]
      int fu = 0, fv = 0;
      while (g.frame_begin[fu + 1] <= u) ++fu;
      while (g.frame_begin[fv + 1] <= v) ++fv;
      add_row(wt * (margin - d), nv, xu, fu, xv, fv);
      any_rows = true;
    }
    for (int ob = 0; ob < g.n_boxes; ++ob) {
      for (int c = 0; c < g.n_caps; ++c) {
        float mc[3];
        for (int q = 0; q < 3; ++q) mc[q] = 0.5f * (cA[c][q] + cB[c][q]);
        if (!spheres_meet(mc, g.bound[c], g.p[ob], g.box_bound[ob], margin)) continue;
        float ab[3], bb[3];
        to_box(g, ob, cA[c], ab);
        to_box(g, ob, cB[c], bb);
        if (!aabb_box_meet(ab, bb, g.r[c] + margin + 1e-5f, g.h[ob])) continue;
        float t;
        const float dist = sqrtf(seg_box_d2_t(ab, bb, g.h[ob], t));
        const float d = dist - g.r[c];
        if (!(d < margin) || dist <= kMinDir) continue;
        float nb[3], nv[3], x[3];
        for (int q = 0; q < 3; ++q) {
          const float xb = ab[q] + t * (bb[q] - ab[q]);
          const float pb = fminf(fmaxf(xb, -g.h[ob][q]), g.h[ob][q]);
          nb[q] = (xb - pb) / dist;
        }
        for (int q = 0; q < 3; ++q) {  // back to the world: (R^T)^T n
          nv[q] = g.Rt[ob][q] * nb[0] + g.Rt[ob][3 + q] * nb[1] + g.Rt[ob][6 + q] * nb[2];
          x[q] = cA[c][q] + t * (cB[c][q] - cA[c][q]);
        }
        int fc = 0;
        while (g.frame_begin[fc + 1] <= c) ++fc;
        add_row(wt * (margin - d), nv, x, fc, x, -1);
        any_rows = true;
      }
    }
    double* dst = Gh + (size_t)i * (NP + n);
    for (int k = 0; k < NP; ++k) dst[k] = G[k];
    for (int k = 0; k < n; ++k) dst[NP + k] = h[k];
  }
  ok = __syncthreads_and(ok);
  any_rows = __syncthreads_or(any_rows);  // also orders the scratch stores before phase 2
  if (!ok || T < 2 || tid >= 32) return;
  if (!any_rows) {  // no active row: the scalar-identity step
    scalar_thomas(rq, rd, a.lambda_d, Wg, Wg + T, lane);
    return;
  }

  const float* qc = rq.q_out;
  const int nn = n * n;
  // lane's entries e = lane + 32 m of an n x n block, and the packed index of G
  int gidx[kGjPerLane];
#pragma unroll
  for (int m = 0; m < kGjPerLane; ++m) {
    const int e = lane + 32 * m, r = e / n, c = e - (e / n) * n;
    const int hi = r > c ? r : c, lo = r > c ? c : r;
    gidx[m] = e < nn ? hi * (hi + 1) / 2 + lo : 0;
  }
  double gn[kGjPerLane], hn = 0.0, qm = 0.0, q0 = 0.0, q1 = 0.0;  // step i + 1's inputs
  auto load_step = [&](int i) {
    const double* Gi = Gh + (size_t)i * (NP + n);
#pragma unroll
    for (int m = 0; m < kGjPerLane; ++m) gn[m] = lane + 32 * m < nn ? Gi[gidx[m]] : 0.0;
    if (lane < n) {
      hn = Gi[NP + lane];
      q0 = (double)qc[(size_t)i * n + lane];
      qm = i > 0 ? (double)qc[(size_t)(i - 1) * n + lane] : 0.0;
      q1 = i + 1 < T ? (double)qc[(size_t)(i + 1) * n + lane] : 0.0;
    }
  };
  load_step(0);
  for (int i = 0; i < T; ++i) {
    double* S = Sb[i & 1];
    const double* Wp = Sb[(i + 1) & 1];
    const double* yprev = yb[(i + 1) & 1];
    double* ycur = yb[i & 1];
    const double diag = (i > 0 ? 1.0 : 0.0) + (i + 1 < T ? 1.0 : 0.0) + a.lambda_d;
#pragma unroll
    for (int m = 0; m < kGjPerLane; ++m) {
      const int e = lane + 32 * m;
      if (e >= nn) break;
      double v = gn[m] + (e % (n + 1) == 0 ? diag : 0.0);
      if (i > 0) v -= Wp[e];
      S[e] = v;
    }
    if (lane < n) {
      const int c = lane;
      double b = -hn;
      if (i + 1 < T) b += q1 - q0;
      if (i > 0) b -= q0 - qm;
      if (i > 0)
        for (int k = 0; k < n; ++k) b += Wp[c * n + k] * yprev[k];
      ycur[c] = b;
    }
    if (i + 1 < T) load_step(i + 1);
    __syncwarp();
    // S <- S^{-1}: pivot j scales row j by 1/p, column j by -1/p, and takes
    // S[r][j] S[j][c] / p from the other entries
    for (int j = 0; j < n; ++j) {
      const double pv = S[j * n + j];
      if (!(pv > 0.0)) return;  // warp-uniform: leave q unchanged
      const double ip = 1.0 / pv;
      double nv[kGjPerLane];
#pragma unroll
      for (int m = 0; m < kGjPerLane; ++m) {
        const int e = lane + 32 * m;
        if (e >= nn) break;
        const int r = e / n, c = e - r * n;
        const double v = S[e];
        if (r == j)
          nv[m] = c == j ? ip : v * ip;
        else if (c == j)
          nv[m] = -v * ip;
        else
          nv[m] = fma(-(S[r * n + j] * ip), S[j * n + c], v);
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < kGjPerLane; ++m) {
        const int e = lane + 32 * m;
        if (e >= nn) break;
        S[e] = nv[m];
      }
      __syncwarp();
    }
    double* Wi = Wg + (size_t)i * nn;
#pragma unroll
    for (int m = 0; m < kGjPerLane; ++m) {
      const int e = lane + 32 * m;
      if (e >= nn) break;
      Wi[e] = S[e];
    }
    if (lane < n) Yg[(size_t)i * n + lane] = ycur[lane];
    __syncwarp();
  }
  // x_i = S_i^{-1} (y_i + x_{i+1}): lane c takes row c; step i - 1's row is loaded
  // during step i
  double wr[kMaxJ], yr[kMaxJ];
  auto load_back = [&](int i) {
#pragma unroll
    for (int k = 0; k < kMaxJ; ++k) {
      wr[k] = lane < n && k < n ? Wg[(size_t)i * nn + lane * n + k] : 0.0;
      yr[k] = k < n ? Yg[(size_t)i * n + k] : 0.0;
    }
  };
  load_back(T - 1);
  for (int i = T - 1; i >= 0; --i) {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxJ; ++k)
      if (k < n) v += wr[k] * (yr[k] + (i + 1 < T ? xs[k] : 0.0));
    if (i > 0) load_back(i - 1);
    __syncwarp();
    if (lane < n) {
      const int c = lane;
      xs[c] = v;
      const double qn = fmin(fmax((double)qc[(size_t)i * n + c] + v, rd.lo[c]), rd.hi[c]);
      rq.q_out[(size_t)i * n + c] = (float)qn;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ launchers
static LmArgs make_lm_args(const cpp_params_t& P, bool want_err, bool from_out) {
  LmArgs a;
  a.want_err = want_err ? 1 : 0;
  a.from_out = from_out ? 1 : 0;
  a.lambda0 = P.lambda0; a.lambda_up = P.lambda_up; a.lambda_down = P.lambda_down;
  a.lambda_min = P.lambda_min; a.lambda_max = P.lambda_max;
  a.freeze_step = P.freeze_step; a.freeze_cost = P.freeze_cost;
  a.iters = P.lm_iters; a.free_mask = P.free_mask;
  return a;
}

// Resident one-warp blocks of an LM kernel per SM (asked once per instantiation).
template <class KernelT>
static int lm_blocks_per_sm(KernelT kernel) {
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kLmThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    v = 0;
  }
  return v > 0 ? v : 1;
}

// A single request: one warp per 32 waypoints. A batch: a persistent grid of as
// many one-warp blocks as the device holds at once (no more than the waypoints
// need), the work counter zeroed first.
template <int NJ, class F, class Src>
static cudaError_t launch_lm_kernel(const Src& s, int max_T, const LmArgs& a, cudaStream_t st) {
  auto kernel = lm_kernel<NJ, F, Src>;
  if constexpr (std::is_same<Src, BatchSrc>::value) {
    if (!s.lm.counter || !s.lm.views || !s.lm.wp_begin) return cudaErrorInvalidValue;
    if (s.lm.total < 1) return cudaSuccess;
    static const int per_sm = lm_blocks_per_sm(kernel);
    const long long want = ((long long)s.lm.total + kLmThreads - 1) / kLmThreads;
    const int blocks = (int)std::min<long long>(want, (long long)per_sm * device_sm_count());
    cudaError_t e = cudaMemsetAsync(s.lm.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kernel<<<blocks, kLmThreads, 0, st>>>(s, a);
  } else {
    return launch_k(kernel, dim3((unsigned)((max_T + kLmThreads - 1) / kLmThreads)), dim3(kLmThreads),
                    0, st, 1, kPdl<Src>, s, a);
  }
  return cudaGetLastError();
}

template <int NJ, class Src>
static cudaError_t launch_lm_nj(const Src& s, int max_T, const LmArgs& a, bool fp64, cudaStream_t st) {
  return fp64 ? launch_lm_kernel<NJ, double>(s, max_T, a, st) : launch_lm_kernel<NJ, float>(s, max_T, a, st);
}

template <class Src>
static cudaError_t launch_lm_phase(const Src& s, int n, int nreq, int max_T, const cpp_params_t& P,
                                   bool want_err, bool from_out, cudaStream_t st) {
  (void)nreq;
  const LmArgs a = make_lm_args(P, want_err, from_out);
  const bool fp64 = P.lm_fp64 != 0;
  switch (n) {
    case 6: return launch_lm_nj<6>(s, max_T, a, fp64, st);
    case 7: return launch_lm_nj<7>(s, max_T, a, fp64, st);
    case 9: return launch_lm_nj<9>(s, max_T, a, fp64, st);
    default: return launch_lm_nj<0>(s, max_T, a, fp64, st);
  }
}

cudaError_t launch_robot_views(const cpp_robot_t* robots, int n, RobotViews* views,
                               cudaStream_t st) {
  if (n < 1) return cudaSuccess;
  robot_views_kernel<<<n, 32, 0, st>>>(robots, views);
  return cudaGetLastError();
}

template <class Src>
static cudaError_t launch_smooth_t(const Src& s, int n, int nreq, int max_T, const cpp_params_t& P,
                                   bool any_geo, cudaStream_t st) {
  const SmoothArgs a{P.tau_pos, P.tau_rot, P.smooth_lambda, P.coll_margin, P.coll_weight};
  if (any_geo) {
    smooth_geo_kernel<Src><<<nreq, kSmoothGeoThreads, 0, st>>>(s, a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = smooth_smem_bytes(max_T, n);
  if (smem > 48u * 1024u) {
    const cudaError_t e = cudaFuncSetAttribute(smooth_kernel<Src>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  smooth_kernel<Src><<<nreq, 32, smem, st>>>(s, a);
  return cudaGetLastError();
}

// The refinement of §III-C: a pose phase, then smooth_rounds times a
// trajectory-length step (taken per request only when its waypoints are all
// within tau) followed by another pose phase.
template <class Src>
static cudaError_t launch_lm_t(const Src& s, int n, int nreq, int max_T, const cpp_params_t& P,
                               bool want_err, bool any_geo, cudaStream_t st) {
  const int rounds = P.smooth_rounds > 0 ? P.smooth_rounds : 0;
  cudaError_t e = launch_lm_phase(s, n, nreq, max_T, P, want_err && rounds == 0, false, st);
  for (int k = 0; k < rounds && e == cudaSuccess; ++k) {
    if ((e = launch_smooth_t(s, n, nreq, max_T, P, any_geo, st)) != cudaSuccess) break;
    e = launch_lm_phase(s, n, nreq, max_T, P, want_err && k + 1 == rounds, true, st);
  }
  return e;
}

cudaError_t launch_lm(const SingleSrc& s, const cpp_params_t& P, bool want_err, cudaStream_t st) {
  return launch_lm_t(s, s.r.n, 1, s.r.T, P, want_err, s.has_geo && s.r.smooth_ws, st);
}
cudaError_t launch_lm_batch(const BatchSrc& s, int n, int nreq, int max_T, const cpp_params_t& P,
                            cudaStream_t st) {
  return launch_lm_t(s, n, nreq, max_T, P, false, false, st);
}
cudaError_t launch_lm_batch_geo(const BatchSrc& s, int n, int nreq, int max_T,
                                const cpp_params_t& P, bool any_geo, cudaStream_t st) {
  return launch_lm_t(s, n, nreq, max_T, P, false, any_geo, st);
}
template <class Src>
static cudaError_t launch_check_t(const Src& s, int nreq, const cpp_params_t& P, cudaStream_t st);

cudaError_t launch_improve_batch(const BatchSrc& s, int n, int nreq, int max_T,
                                 const cpp_params_t& P, bool any_geo, cudaStream_t st) {
  cudaError_t e = launch_smooth_t(s, n, nreq, max_T, P, any_geo, st);
  if (e == cudaSuccess) e = launch_lm_phase(s, n, nreq, max_T, P, false, true, st);
  if (e == cudaSuccess) e = launch_check_t(s, nreq, P, st);
  return e;
}
cudaError_t launch_smooth(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st) {
  return launch_smooth_t(s, s.r.n, 1, s.r.T, P, s.has_geo && s.r.smooth_ws, st);
}
int lm_launches(const cpp_params_t& P, bool any_geo) {
  return 1 + (any_geo ? 3 : 2) * (P.smooth_rounds > 0 ? P.smooth_rounds : 0);
}

// A batch whose clusters would not fit on the GPU at once runs one CTA per request.
template <class Src>
static cudaError_t launch_check_t(const Src& s, int nreq, const cpp_params_t& P, cudaStream_t st) {
  CheckArgs a{P.tau_pos, P.tau_rot, P.jump_max};
  if (nreq * kChkCluster > device_sm_count()) {
    check_kernel<false, Src><<<nreq, kChkThreads * kChkCluster, 0, st>>>(s, a);
    return cudaGetLastError();
  }
  return launch_k(check_kernel<true, Src>, dim3((unsigned)(nreq * kChkCluster)), dim3(kChkThreads), 0,
                  st, kChkCluster, kPdl<Src>, s, a);
}
cudaError_t launch_check(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st) {
  return launch_check_t(s, 1, P, st);
}
cudaError_t launch_check_batch(const BatchSrc& s, int nreq, const cpp_params_t& P,
                               cudaStream_t st) {
  return launch_check_t(s, nreq, P, st);
}

}  // namespace cppflow

extern "C" {

cpp_status cpp_counters_reset(cpp_stream_t stream) {
  const cpp_counters_t zero = {0, 0};
  const cudaError_t e = cudaMemcpyToSymbolAsync(cppflow::g_lm_counters, &zero, sizeof(zero), 0,
                                                cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e == cudaSuccess) {
    // the source is a stack variable: wait until the copy has read it
    const cudaError_t w = cudaStreamSynchronize((cudaStream_t)stream);
    if (w == cudaSuccess) return CPP_OK;
    cppflow::set_last_error(cudaGetErrorString(w));
    return CPP_ERR_CUDA;
  }
  cppflow::set_last_error(cudaGetErrorString(e));
  return CPP_ERR_CUDA;
}

cpp_status cpp_counters_read(cpp_counters_t* out) {
  if (!out) {
    cppflow::set_last_error("cpp_counters_read: out is NULL");
    return CPP_ERR_INVALID_ARG;
  }
  const cudaError_t e = cudaMemcpyFromSymbol(out, cppflow::g_lm_counters, sizeof(*out));
  if (e != cudaSuccess) {
    cppflow::set_last_error(cudaGetErrorString(e));
    return CPP_ERR_CUDA;
  }
  return CPP_OK;
}

}  // extern "C"
