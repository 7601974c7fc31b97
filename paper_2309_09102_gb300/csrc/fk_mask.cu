// fk_mask.cu -- batched forward kinematics, pose error, joint-limit / pose masks
// and node costs for the candidate lattice (paper §II "Pose error", "Joint
// limits"; §III-B node costs).
//
// Layout: candidates are [T][n][Kp] FP32, k fastest. A task is one waypoint and
// a block of 128 candidates; one warp runs tasks_per_warp consecutive tasks
// (default 4: the 4 blocks of one waypoint at K = 512; the batch autotuner
// picks it per batch), so the robot staging of a block and the target
// conversion of a waypoint are paid once for several tasks. Lane l
// reads joints j of candidates 4l .. 4l+3 as one float4 per joint (512
// contiguous bytes per warp per joint), runs the FP32 DH chain for its four
// candidates in registers, and writes one uchar4 mask word, one float4 of costs
// and two float4 of errors.
#include <cmath>
#include <type_traits>

#include "collide.cuh"
#include "internal.h"

namespace cppflow {

constexpr int kMaskThreads = 256;
constexpr int kMaskWarps = kMaskThreads / 32;
constexpr int kMaskBlockK = 128;
constexpr int kMaskTasksPerWarp = 4;  // default tasks per warp

struct MaskArgs {
  float tau_pos, tau_rot;
  // the pose test without a root or atan2: |dp|^2 > tau_pos^2, and (for tau_rot <
  // pi / 2) angle > tau_rot <=> c <= 0 or |v|^2 > 4 c^2 tan^2 tau_rot (geodesic_parts)
  float tau_pos2, tan2_rot;
  int rot_fast;
  float pen_table[8];  // [limit bit | pose bit << 1 | collision bit << 2]: each the FP64 sum
                       // of its costs in that order, rounded once
  double near_margin;
  int tasks_per_warp;
};

// The target of waypoint i as FP32 rotation + position. The quaternion is
// rounded to FP32 and converted in FP32 (GB300's FP64 pipe is ~64x narrower
// than FP32); this adds ~1e-7 to the pose errors, far inside their 1e-5
// tolerance. Lanes 0..6 each round one of the seven numbers, the warp shares
// them by shuffles. Called by all 32 lanes.
__device__ __forceinline__ void warp_target_f32(const double* t7, int lane, float Rt[9],
                                                float pt[3]) {
  const float v = lane < 7 ? (float)__ldg(t7 + lane) : 0.f;
  pt[0] = __shfl_sync(0xffffffffu, v, 0);
  pt[1] = __shfl_sync(0xffffffffu, v, 1);
  pt[2] = __shfl_sync(0xffffffffu, v, 2);
  const float qw = __shfl_sync(0xffffffffu, v, 3), qx = __shfl_sync(0xffffffffu, v, 4);
  const float qy = __shfl_sync(0xffffffffu, v, 5), qz = __shfl_sync(0xffffffffu, v, 6);
  const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  const float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
  Rt[0] = 1.f - 2.f * (y * y + z * z); Rt[1] = 2.f * (x * y - w * z); Rt[2] = 2.f * (x * z + w * y);
  Rt[3] = 2.f * (x * y + w * z); Rt[4] = 1.f - 2.f * (x * x + z * z); Rt[5] = 2.f * (y * z - w * x);
  Rt[6] = 2.f * (x * z - w * y); Rt[7] = 2.f * (y * z + w * x); Rt[8] = 1.f - 2.f * (x * x + y * y);
}

// FP32 FK as fk_f32 (the same operations, so the same pose), placing the world
// end points of each frame's capsules as the frame is reached.
template <int NJ>
__device__ __forceinline__ void fk_caps(const RobotF& rb, const GeoF& g, const float* q, float R[9],
                                        float p[3], float (*cA)[3], float (*cB)[3]) {
  pose_identity(R, p);
  place_caps(g, 0, R, p, cA, cB);
  const int n = NJ ? NJ : rb.n;
#pragma unroll
  for (int j = 0; j < (NJ ? NJ : kMaxJ); ++j) {
    if (!NJ && j >= n) break;
    float s, c;
    __sincosf(q[j] + rb.th0[j], &s, &c);
    dh_step(R, p, c, s, rb.ca[j], rb.sa[j], rb.a[j], rb.d[j]);
    place_caps(g, j + 1, R, p, cA, cB);
  }
}

// ERR: also the pose errors themselves (cpp_mask with an error buffer); the
// decision is the same either way, so every path masks alike.
template <int NJ, bool COLL, bool ERR>
__device__ __forceinline__ void mask_one(const RobotF& rb, const MaskArgs& a, const float* q,
                                         int n, bool pad, const float Rt[9], const float pt[3],
                                         const GeoF* g, bool want_clear, uint8_t& bits,
                                         float& cost, float& epos, float& erot, float& clr) {
  if (pad) {
    bits = CPP_MASK_PAD; cost = CUDART_INF_F; epos = erot = clr = CUDART_NAN_F;
    return;
  }
  bool finite = true;
  uint32_t b = 0;
#pragma unroll
  for (int j = 0; j < (NJ ? NJ : kMaxJ); ++j) {
    if (!NJ && j >= n) break;
    const float v = q[j];
    finite &= isfinite(v);
    if (v < rb.lo[j] || v > rb.hi[j]) b |= CPP_MASK_OUT;
    if (v < rb.nlo[j] || v > rb.nhi[j]) b |= CPP_MASK_NEAR;
  }
  if (!finite) {
    bits = CPP_MASK_NONFINITE; cost = CUDART_INF_F; epos = erot = clr = CUDART_NAN_F;
    return;
  }
  float R[9], p[3];
  clr = CUDART_INF_F;
  if (COLL && g) {
    float cA[kMaxCaps][3], cB[kMaxCaps][3];
    fk_caps<NJ>(rb, *g, q, R, p, cA, cB);
    if (want_clear) {  // the exact smallest clearance is requested
      clr = clearance(*g, cA, cB);
      if (clr < 0.f) b |= CPP_MASK_COLLIDE;
    } else if (collides(*g, cA, cB)) {
      b |= CPP_MASK_COLLIDE;
    }
  } else {
    fk_f32<NJ>(rb, q, R, p);
  }
  const float dx = p[0] - pt[0], dy = p[1] - pt[1], dz = p[2] - pt[2];
  const float d2 = dx * dx + dy * dy + dz * dz;
  float c, vv;
  geodesic_parts<float>(Rt, R, c, vv);
  const bool rot_fail = a.rot_fast ? (c <= 0.f || vv > 4.f * c * c * a.tan2_rot)
                                   : atan2f(0.5f * sqrtf(vv), c) > a.tau_rot;
  if (d2 > a.tau_pos2 || rot_fail) b |= CPP_MASK_POSE;
  if (ERR) {
    epos = sqrtf(d2);
    erot = atan2f(0.5f * sqrtf(vv), c);
  } else {
    epos = erot = 0.f;
  }
  bits = (uint8_t)b;
  const bool lim = (b & (CPP_MASK_OUT | CPP_MASK_NEAR)) != 0, pose = (b & CPP_MASK_POSE) != 0;
  const bool coll = (b & CPP_MASK_COLLIDE) != 0;
  const float c0 = lim ? (pose ? a.pen_table[3] : a.pen_table[1]) : (pose ? a.pen_table[2] : a.pen_table[0]);
  const float c1 = lim ? (pose ? a.pen_table[7] : a.pen_table[5]) : (pose ? a.pen_table[6] : a.pen_table[4]);
  cost = coll ? c1 : c0;
}

// Both variants are bound by issue and dependency latency rather than registers:
// more resident warps measured faster -- three CTAs per SM for the plain mask (80
// registers, a few spills; 0.86 -> 0.81 ms with the layer minima on the 304-request
// batch, four measured slower) and four for the collision variant (64 registers;
// two at 117 registers were 1.1 ms slower per batch).
template <int NJ, bool COLL, bool ERR, class Src>
__global__ void __launch_bounds__(kMaskThreads, COLL ? 4 : 3) mask_kernel(const __grid_constant__ Src src,
                                                             const MaskArgs a) {
  pdl_trigger();
  pdl_wait();
  const Req& rq = src.req(blockIdx.y);
  __shared__ RobotF rb;
  __shared__ GeoF gsh;
  stage_robot(src.rob(rq.robot), a.near_margin, &rb, nullptr);
  const GeoF* gsrc = COLL ? src.geom(rq) : nullptr;
  if (COLL && gsrc) {  // one request per block: stage its model
    const uint32_t* from = reinterpret_cast<const uint32_t*>(gsrc);
    uint32_t* to = reinterpret_cast<uint32_t*>(&gsh);
    for (int w = threadIdx.x; w < (int)(sizeof(GeoF) / 4); w += kMaskThreads) to[w] = from[w];
  }
  __syncthreads();
  const GeoF* g = (COLL && gsrc) ? &gsh : nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (rq.Kp + kMaskBlockK - 1) / kMaskBlockK;
  const long long ntask = (long long)rq.T * nblk;
  const int tpw = a.tasks_per_warp;
  const long long t0 = ((long long)blockIdx.x * kMaskWarps + warp) * tpw;
  const long long t1 = t0 + tpw < ntask ? t0 + tpw : ntask;
  const int n = NJ ? NJ : rq.n;

  int cur_i = -1;
  float Rt[9], pt[3];
  for (long long task = t0; task < t1; ++task) {
    const int i = (int)(task / nblk), kb = (int)(task % nblk);
    if (i != cur_i) {  // warp-uniform
      warp_target_f32(rq.targets + 7 * (size_t)i, lane, Rt, pt);
      cur_i = i;
    }
    const int k0 = kb * kMaskBlockK + 4 * lane;
    if (k0 >= rq.Kp || k0 < rq.k_begin) continue;  // k_begin is a multiple of 4
    float4 qv[NJ ? NJ : kMaxJ];
    const float* base = rq.cand + (size_t)i * n * rq.Kp + k0;
#pragma unroll
    for (int j = 0; j < (NJ ? NJ : kMaxJ); ++j) {
      if (!NJ && j >= n) break;
      qv[j] = __ldg(reinterpret_cast<const float4*>(base + (size_t)j * rq.Kp));
    }
    uint8_t bits[4];
    float cost[4], ep[4], er[4], cl[4];
    // the collision code is large: one copy of it (no unrolling) keeps it in the
    // instruction cache
    constexpr int kUnroll = COLL ? 1 : 4;
#pragma unroll kUnroll
    for (int c = 0; c < 4; ++c) {
      float q[NJ ? NJ : kMaxJ];
#pragma unroll
      for (int j = 0; j < (NJ ? NJ : kMaxJ); ++j) {
        if (!NJ && j >= n) break;
        q[j] = c == 0 ? qv[j].x : c == 1 ? qv[j].y : c == 2 ? qv[j].z : qv[j].w;
      }
      mask_one<NJ, COLL, ERR>(rb, a, q, n, k0 + c >= rq.K, Rt, pt, g, rq.clear != nullptr, bits[c],
                         cost[c], ep[c], er[c], cl[c]);
    }
    const size_t o = (size_t)i * rq.Kp + k0;
    *reinterpret_cast<uchar4*>(rq.mask + o) = make_uchar4(bits[0], bits[1], bits[2], bits[3]);
    *reinterpret_cast<float4*>(rq.pen + o) = make_float4(cost[0], cost[1], cost[2], cost[3]);
    if (ERR && rq.err) {
      float4* e = reinterpret_cast<float4*>(rq.err + 2 * o);
      e[0] = make_float4(ep[0], er[0], ep[1], er[1]);
      e[1] = make_float4(ep[2], er[2], ep[3], er[3]);
    }
    if (rq.clear)
      *reinterpret_cast<float4*>(rq.clear + o) = make_float4(cl[0], cl[1], cl[2], cl[3]);
  }
}

// ------------------------------------------------------------------ plain FK calls
__global__ void fk_batch_kernel(const cpp_robot_t robot, const float* __restrict__ q, long long N,
                                float* __restrict__ R, float* __restrict__ p) {
  __shared__ RobotF rb;
  stage_robot(robot, 0.0, &rb, nullptr);
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x) {
    float qq[kMaxJ];
    for (int j = 0; j < rb.n; ++j) qq[j] = q[j * N + t];
    float Rl[9], pl[3];
    fk_f32<0>(rb, qq, Rl, pl);
#pragma unroll
    for (int e = 0; e < 9; ++e) R[e * N + t] = Rl[e];
#pragma unroll
    for (int e = 0; e < 3; ++e) p[e * N + t] = pl[e];
  }
}

// Rotation -> unit quaternion (w >= 0), largest-pivot branch.
__device__ inline void rot_to_quat(const double R[9], double* q) {
  const double tr = R[0] + R[4] + R[8];
  double w, x, y, z;
  if (tr > 0.0) {
    const double s = 2.0 * sqrt(tr + 1.0);
    w = 0.25 * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[0] - R[4] - R[8]);
    w = (R[7] - R[5]) / s; x = 0.25 * s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const double s = 2.0 * sqrt(1.0 + R[4] - R[0] - R[8]);
    w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; y = 0.25 * s; z = (R[5] + R[7]) / s;
  } else {
    const double s = 2.0 * sqrt(1.0 + R[8] - R[0] - R[4]);
    w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; z = 0.25 * s;
  }
  const double sg = w < 0.0 ? -1.0 : 1.0;
  const double inv = sg / sqrt(w * w + x * x + y * y + z * z);
  q[0] = w * inv; q[1] = x * inv; q[2] = y * inv; q[3] = z * inv;
}

__global__ void fk_pose64_kernel(const cpp_robot_t robot, const double* __restrict__ q,
                                 long long N, double* __restrict__ pose) {
  __shared__ RobotD rb;
  stage_robot(robot, 0.0, nullptr, &rb);
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x) {
    double R[9], p[3];
    fk_f64(rb, q + t * rb.n, R, p);
    double* o = pose + 7 * t;
    o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
    rot_to_quat(R, o + 3);
  }
}

// ------------------------------------------------------------------ launchers
static MaskArgs make_mask_args(const cpp_params_t& P) {
  MaskArgs a;
  a.tau_pos = (float)P.tau_pos;
  a.tau_rot = (float)P.tau_rot;
  a.tau_pos2 = (float)(P.tau_pos * P.tau_pos);
  a.rot_fast = P.tau_rot < 1.5 ? 1 : 0;  // below pi / 2: tan is finite and increasing
  a.tan2_rot = a.rot_fast ? (float)(std::tan(P.tau_rot) * std::tan(P.tau_rot)) : 0.f;
  for (int m = 0; m < 8; ++m) {
    double c = 0.0;
    if (m & 1) c += P.pen_limit;
    if (m & 2) c += P.pen_pose;
    if (m & 4) c += P.pen_collide;
    a.pen_table[m] = (float)c;
  }
  a.near_margin = P.near_margin;
  a.tasks_per_warp = kMaskTasksPerWarp;
  return a;
}

template <bool COLL, bool ERR, class Src>
static void launch_mask_c(const Src& src, int n, dim3 grid, const MaskArgs& a, cudaStream_t st) {
  switch (n) {
    case 6: mask_kernel<6, COLL, ERR, Src><<<grid, kMaskThreads, 0, st>>>(src, a); break;
    case 7: mask_kernel<7, COLL, ERR, Src><<<grid, kMaskThreads, 0, st>>>(src, a); break;
    case 9: mask_kernel<9, COLL, ERR, Src><<<grid, kMaskThreads, 0, st>>>(src, a); break;
    default: mask_kernel<0, COLL, ERR, Src><<<grid, kMaskThreads, 0, st>>>(src, a); break;
  }
}

// err: some request has an error buffer (only cpp_mask's single request can)
template <class Src>
static cudaError_t launch_mask_t(const Src& src, int n, int nreq, long long max_tasks,
                                 const cpp_params_t& P, bool coll, bool err, int tasks_per_warp,
                                 cudaStream_t st) {
  MaskArgs a = make_mask_args(P);
  a.tasks_per_warp = tasks_per_warp > 0 ? tasks_per_warp : kMaskTasksPerWarp;
  const long long per_block = (long long)kMaskWarps * a.tasks_per_warp;
  dim3 grid((unsigned)((max_tasks + per_block - 1) / per_block), (unsigned)nreq);
  if constexpr (std::is_same<Src, SingleSrc>::value) {
    if (err) {
      if (coll) launch_mask_c<true, true>(src, n, grid, a, st);
      else launch_mask_c<false, true>(src, n, grid, a, st);
      return cudaGetLastError();
    }
  }
  if (coll) launch_mask_c<true, false>(src, n, grid, a, st);
  else launch_mask_c<false, false>(src, n, grid, a, st);
  return cudaGetLastError();
}

cudaError_t launch_mask(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st) {
  const long long tasks = (long long)s.r.T * ((s.r.Kp + kMaskBlockK - 1) / kMaskBlockK);
  return launch_mask_t(s, s.r.n, 1, tasks, P, s.has_geo != 0, s.r.err != nullptr, 0, st);
}

cudaError_t launch_mask_batch(const BatchSrc& s, int n, int nreq, long long max_tasks,
                              const cpp_params_t& P, bool any_geo, cudaStream_t st,
                              int tasks_per_warp) {
  return launch_mask_t(s, n, nreq, max_tasks, P, any_geo, false, tasks_per_warp, st);
}

long long mask_tasks(int T, int Kp) {
  return (long long)T * ((Kp + kMaskBlockK - 1) / kMaskBlockK);
}

cudaError_t launch_fk_batch(const cpp_robot_t& r, const float* q, long long N, float* R,
                            float* p, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = std::min<long long>((N + threads - 1) / threads, 152LL * 16);
  fk_batch_kernel<<<(unsigned)blocks, threads, 0, st>>>(r, q, N, R, p);
  return cudaGetLastError();
}

cudaError_t launch_fk_pose64(const cpp_robot_t& r, const double* q, long long N, double* pose,
                             cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  const int threads = 128;
  const long long blocks = std::min<long long>((N + threads - 1) / threads, 152LL * 16);
  fk_pose64_kernel<<<(unsigned)blocks, threads, 0, st>>>(r, q, N, pose);
  return cudaGetLastError();
}

}  // namespace cppflow
