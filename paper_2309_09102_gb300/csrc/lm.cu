// lm.cu -- Levenberg-Marquardt refinement of the searched trajectory (paper
// §III-C) and the FP64 trajectory check (§II constraints and metrics).
//
// The pose residual of waypoint i depends on q_i only, so its Jacobian is block
// diagonal and every waypoint is an independent damped n x n problem. One warp
// owns one waypoint:
//   * every lane runs the same DH chain (FP32, or FP64 in the all-FP64 mode);
//     lane j keeps the frame (z_j, o_j) it needs for Jacobian column j,
//   * lane j forms column j = [z_j x (p_e - o_j); z_j] of the geometric Jacobian,
//   * the n(n+1)/2 entries of J^T J and the n entries of J^T e are spread over
//     the lanes (columns fetched with per-lane shuffles) and accumulated in FP64,
//   * the Cholesky factorisation and both triangular solves run in FP64 in a
//     per-warp shared-memory tile, lanes parallel over rows,
//   * the trial q' = clamp(q + delta, lo, hi) is accepted iff F(q') < F(q)
//     (F = |e|^2 / 2 accumulated in FP64), with lambda / 10 or * 10.
// The joint state is held in FP64; q_out is its FP32 rounding.
#include "internal.h"

namespace cppflow {

constexpr int kLmWarps = 4;
constexpr int kLmThreads = 32 * kLmWarps;
constexpr int kChkThreads = 256;

struct LmArgs {
  double lambda0, lambda_up, lambda_down, lambda_min, lambda_max, freeze_step, freeze_cost;
  int iters;
  uint32_t free_mask;
  int want_err;  // write the FP64 pose error of q_out (skipped when a check follows)
};

struct CheckArgs {
  double tau_pos, tau_rot, jump_max;
};

// ------------------------------------------------------------------ chain evaluation
__device__ __forceinline__ float to_angle(double q, const RobotF& rb, int j) {
  return (float)q + rb.th0[j];
}
__device__ __forceinline__ double to_angle(double q, const RobotD& rb, int j) {
  return q + rb.th0[j];
}

// FK of q on every lane; lane j records (z_j, o_j); returns e = [p_t - p; log(R_t R^T)]
// and F = |e|^2 / 2 (FP64 sum).
template <class F, class RB>
__device__ __forceinline__ double chain_eval(const RB& rb, const double* q, int lane,
                                             const F Rt[9], const F pt[3], F z[3], F o[3],
                                             F e[6]) {
  F R[9], p[3];
  pose_identity(R, p);
#pragma unroll
  for (int j = 0; j < kMaxJ; ++j) {
    if (j >= rb.n) break;
    if (lane == j) {
      z[0] = R[2]; z[1] = R[5]; z[2] = R[8];
      o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
    }
    F s, c;
    sincos_t(to_angle(q[j], rb, j), &s, &c);
    dh_step(R, p, c, s, (F)rb.ca[j], (F)rb.sa[j], (F)rb.a[j], (F)rb.d[j]);
  }
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

template <class F, class Src>
__global__ void __launch_bounds__(kLmThreads) lm_kernel(const __grid_constant__ Src src,
                                                         const LmArgs a) {
  const Req& rq = src.req(blockIdx.y);
  __shared__ RobotF rf;
  __shared__ RobotD rd;
  __shared__ double sA[kLmWarps][kMaxJ * kMaxJ];
  __shared__ double sg[kLmWarps][kMaxJ];
  stage_robot(src.rob(rq.robot), 0.0, &rf, &rd);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kLmWarps + warp;
  if (i >= rq.T) return;
  const auto& rb = RobotFor<F>::get(rf, rd);
  const int n = rd.n;
  double* A = sA[warp];
  double* g = sg[warp];

  F Rt[9], pt[3];
  {
    double R[9];
    const double* t7 = rq.targets + 7 * (size_t)i;
    quat_to_rot(t7 + 3, R);
#pragma unroll
    for (int k = 0; k < 9; ++k) Rt[k] = (F)R[k];
    pt[0] = (F)t7[0]; pt[1] = (F)t7[1]; pt[2] = (F)t7[2];
  }
  double q[kMaxJ];
#pragma unroll
  for (int j = 0; j < kMaxJ; ++j) q[j] = j < n ? (double)rq.q_in[(size_t)i * n + j] : 0.0;

  F z[3] = {F(0), F(0), F(0)}, o[3] = {F(0), F(0), F(0)}, e[6];
  double Fc = chain_eval<F>(rb, q, lane, Rt, pt, z, o, e);
  double lam = a.lambda0;
  const int NT = n * (n + 1) / 2;

  for (int it = 0; it < a.iters; ++it) {
    if (Fc < a.freeze_cost) break;
    // Jacobian column of this lane
    F Jc[6];
    {
      F pe[3];
      // p_e = p_t - e_pos
      pe[0] = pt[0] - e[0]; pe[1] = pt[1] - e[1]; pe[2] = pt[2] - e[2];
      const bool on = lane < n && ((a.free_mask >> lane) & 1u);
      const F dx = pe[0] - o[0], dy = pe[1] - o[1], dz = pe[2] - o[2];
      Jc[0] = on ? z[1] * dz - z[2] * dy : F(0);
      Jc[1] = on ? z[2] * dx - z[0] * dz : F(0);
      Jc[2] = on ? z[0] * dy - z[1] * dx : F(0);
      Jc[3] = on ? z[0] : F(0);
      Jc[4] = on ? z[1] : F(0);
      Jc[5] = on ? z[2] : F(0);
    }
    // normal equations: entries (a >= b) of J^T J + lam I, then J^T e
    for (int t0 = 0; t0 < NT + n; t0 += 32) {
      const int t = t0 + lane;
      int ra = 0, cb = 0;
      if (t < NT) {
        while ((ra + 1) * (ra + 2) / 2 <= t) ++ra;
        cb = t - ra * (ra + 1) / 2;
      } else if (t < NT + n) {
        ra = t - NT;
        cb = ra;
      }
      F ja[6], jb[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        ja[r] = __shfl_sync(0xffffffffu, Jc[r], ra);
        jb[r] = __shfl_sync(0xffffffffu, Jc[r], cb);
      }
      double s = 0.0;
      if (t < NT) {
#pragma unroll
        for (int r = 0; r < 6; ++r) s += (double)ja[r] * (double)jb[r];
        if (ra == cb) s += lam;
        A[ra * kMaxJ + cb] = s;
      } else if (t < NT + n) {
#pragma unroll
        for (int r = 0; r < 6; ++r) s += (double)ja[r] * (double)e[r];
        g[ra] = s;
      }
    }
    __syncwarp();
    // Cholesky A = L L^T (lower triangle, in place), lanes own rows
    bool ok = true;
    for (int k = 0; k < n; ++k) {
      const double piv = A[k * kMaxJ + k];
      if (!(piv > 0.0) || !isfinite(piv)) { ok = false; break; }
      const double lkk = sqrt(piv);
      __syncwarp();
      if (lane == k) A[k * kMaxJ + k] = lkk;
      if (lane > k && lane < n) A[lane * kMaxJ + k] = A[lane * kMaxJ + k] / lkk;
      __syncwarp();
      if (lane > k && lane < n) {
        const double lak = A[lane * kMaxJ + k];
        for (int b = k + 1; b <= lane; ++b) A[lane * kMaxJ + b] -= lak * A[b * kMaxJ + k];
      }
      __syncwarp();
    }
    if (ok) {
      // L y = g
      for (int m = 0; m < n; ++m) {
        const double ym = g[m] / A[m * kMaxJ + m];
        __syncwarp();
        if (lane == m) g[m] = ym;
        if (lane > m && lane < n) g[lane] -= A[lane * kMaxJ + m] * ym;
        __syncwarp();
      }
      // L^T x = y
      for (int m = n - 1; m >= 0; --m) {
        const double xm = g[m] / A[m * kMaxJ + m];
        __syncwarp();
        if (lane == m) g[m] = xm;
        if (lane < m) g[lane] -= A[m * kMaxJ + lane] * xm;
        __syncwarp();
      }
      double dq[kMaxJ];
      double mx = 0.0;
#pragma unroll
      for (int j = 0; j < kMaxJ; ++j) {
        dq[j] = j < n ? g[j] : 0.0;
        mx = fmax(mx, fabs(dq[j]));
      }
      __syncwarp();
      if (mx < a.freeze_step) break;
      double qt[kMaxJ];
#pragma unroll
      for (int j = 0; j < kMaxJ; ++j) {
        double v = q[j] + dq[j];
        if (j < n) {
          if (v < rd.lo[j]) v = rd.lo[j];
          if (v > rd.hi[j]) v = rd.hi[j];
        }
        qt[j] = v;
      }
      F zt[3] = {z[0], z[1], z[2]}, ot[3] = {o[0], o[1], o[2]}, et[6];
      const double Ft = chain_eval<F>(rb, qt, lane, Rt, pt, zt, ot, et);
      if (Ft < Fc) {
#pragma unroll
        for (int j = 0; j < kMaxJ; ++j) q[j] = qt[j];
#pragma unroll
        for (int k = 0; k < 3; ++k) { z[k] = zt[k]; o[k] = ot[k]; }
#pragma unroll
        for (int k = 0; k < 6; ++k) e[k] = et[k];
        Fc = Ft;
        lam = fmax(lam / a.lambda_down, a.lambda_min);
      } else {
        lam = fmin(lam * a.lambda_up, a.lambda_max);
      }
    } else {
      __syncwarp();
      lam = fmin(lam * a.lambda_up, a.lambda_max);
    }
  }
  if (lane < n) rq.q_out[(size_t)i * n + lane] = (float)q[lane];
  if (a.want_err && rq.pose_err && lane == 0) {
    // FP64 pose error of the delivered (FP32-rounded) configuration
    double qq[kMaxJ], R[9], p[3], RtD[9];
    for (int j = 0; j < n; ++j) qq[j] = (double)(float)q[j];
    fk_f64(rd, qq, R, p);
    const double* t7 = rq.targets + 7 * (size_t)i;
    quat_to_rot(t7 + 3, RtD);
    const double dx = p[0] - t7[0], dy = p[1] - t7[1], dz = p[2] - t7[2];
    rq.pose_err[2 * (size_t)i] = sqrt(dx * dx + dy * dy + dz * dz);
    rq.pose_err[2 * (size_t)i + 1] = geodesic<double>(RtD, R);
  }
}

// ------------------------------------------------------------------ FP64 check
template <class Src>
__global__ void __launch_bounds__(kChkThreads) check_kernel(const __grid_constant__ Src src,
                                                             const CheckArgs a) {
  const Req& rq = src.req(blockIdx.x);
  __shared__ RobotD rd;
  __shared__ double red[5][kChkThreads / 32];
  __shared__ int redi[3][kChkThreads / 32];
  stage_robot(src.rob(rq.robot), 0.0, nullptr, &rd);
  __syncthreads();
  const int n = rd.n, T = rq.T, tid = threadIdx.x;
  double mpos = 0, mrot = 0, mjac = 0, slinf = 0, tlen = 0;
  int npose = 0, nlim = 0, njump = 0;
  for (int i = tid; i < T; i += kChkThreads) {
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
  // fixed-order block reduction
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
  if (tid == 0 && rq.report) {
    cpp_report_t r;
    r.max_pos = r.max_rot = r.mjac = r.sum_linf = r.traj_len = 0.0;
    r.n_pose_fail = r.n_limit_fail = r.n_jump_fail = 0;
    for (int w = 0; w < kChkThreads / 32; ++w) {
      r.max_pos = fmax(r.max_pos, red[0][w]);
      r.max_rot = fmax(r.max_rot, red[1][w]);
      r.mjac = fmax(r.mjac, red[2][w]);
      r.sum_linf += red[3][w];
      r.traj_len += red[4][w];
      r.n_pose_fail += redi[0][w];
      r.n_limit_fail += redi[1][w];
      r.n_jump_fail += redi[2][w];
    }
    r.valid = (r.n_pose_fail == 0 && r.n_limit_fail == 0 && r.n_jump_fail == 0) ? 1 : 0;
    *rq.report = r;
  }
}

// ------------------------------------------------------------------ launchers
static LmArgs make_lm_args(const cpp_params_t& P, bool want_err) {
  LmArgs a;
  a.want_err = want_err ? 1 : 0;
  a.lambda0 = P.lambda0; a.lambda_up = P.lambda_up; a.lambda_down = P.lambda_down;
  a.lambda_min = P.lambda_min; a.lambda_max = P.lambda_max;
  a.freeze_step = P.freeze_step; a.freeze_cost = P.freeze_cost;
  a.iters = P.lm_iters; a.free_mask = P.free_mask;
  return a;
}

template <class Src>
static cudaError_t launch_lm_t(const Src& s, int nreq, int max_T, const cpp_params_t& P,
                               bool want_err, cudaStream_t st) {
  const LmArgs a = make_lm_args(P, want_err);
  dim3 grid((unsigned)((max_T + kLmWarps - 1) / kLmWarps), (unsigned)nreq);
  if (P.lm_fp64) lm_kernel<double, Src><<<grid, kLmThreads, 0, st>>>(s, a);
  else lm_kernel<float, Src><<<grid, kLmThreads, 0, st>>>(s, a);
  return cudaGetLastError();
}

cudaError_t launch_lm(const SingleSrc& s, const cpp_params_t& P, bool want_err, cudaStream_t st) {
  return launch_lm_t(s, 1, s.r.T, P, want_err, st);
}
cudaError_t launch_lm_batch(const BatchSrc& s, int nreq, int max_T, const cpp_params_t& P,
                            cudaStream_t st) {
  return launch_lm_t(s, nreq, max_T, P, false, st);
}

template <class Src>
static cudaError_t launch_check_t(const Src& s, int nreq, const cpp_params_t& P, cudaStream_t st) {
  CheckArgs a{P.tau_pos, P.tau_rot, P.jump_max};
  check_kernel<Src><<<nreq, kChkThreads, 0, st>>>(s, a);
  return cudaGetLastError();
}
cudaError_t launch_check(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st) {
  return launch_check_t(s, 1, P, st);
}
cudaError_t launch_check_batch(const BatchSrc& s, int nreq, const cpp_params_t& P,
                               cudaStream_t st) {
  return launch_check_t(s, nreq, P, st);
}

}  // namespace cppflow
