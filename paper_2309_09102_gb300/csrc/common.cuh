// common.cuh -- device-side building blocks shared by the planner kernels.
//
// Forward kinematics follows the paper's FK map FK(q): R^d -> SE(3) (§II) in
// standard DH form A_j = Rz(q_j + theta0_j) Tz(d_j) Tx(a_j) Rx(alpha_j).
// The chain is kept in registers as a row-major 3x3 rotation plus origin; each
// link multiplies on the right, which only mixes columns 0 and 1 of the running
// rotation by the joint angle and columns 1 and 2 by the link twist.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cppflow.h"

namespace cppflow {

constexpr int kMaxJ = CPP_MAX_JOINTS;

// ------------------------------------------------------------------ request views
// One request as the kernels see it (device pointers; unused ones may be null).
constexpr int kMaxCaps = CPP_MAX_CAPSULES;
constexpr int kMaxPairs = CPP_MAX_PAIRS;
constexpr int kMaxBoxes = CPP_MAX_BOXES;

// Device copy of a cpp_geometry_t (collision model): FP32, capsules sorted by
// frame (those of frame f are [frame_begin[f], frame_begin[f + 1])), pairs
// renumbered to that order, box rotations transposed (world -> box).
struct GeoF {
  int n_caps, n_pairs, n_boxes, pad_;
  int frame_begin[kMaxJ + 2];
  float a[kMaxCaps][3], b[kMaxCaps][3], r[kMaxCaps];
  float bound[kMaxCaps];    // bounding-sphere radius about the segment midpoint (>= |b-a|/2 + r)
  int8_t pu[kMaxPairs], pv[kMaxPairs];
  float Rt[kMaxBoxes][9], p[kMaxBoxes][3], h[kMaxBoxes][3];
  float box_bound[kMaxBoxes];  // bounding-sphere radius of the box about its centre (>= |h|)
};

struct Req {
  int T, K, Kp, n;
  int k_begin;               // first candidate lane the mask writes (a multiple of 4)
  int robot;                 // index into the robot table
  int Kb;                    // backpointer row stride (Kp rounded up to 8)
  const float* cand;         // [T][n][Kp]
  const double* targets;     // [T][7]
  uint8_t* mask;             // [T][Kp]
  float* pen;                // [T][Kp]
  float* err;                // [T][Kp][2] or null
  float* pen_min;            // [T]      per-waypoint cheapest node cost
  uint16_t* bp;              // [T][Kb]  backpointers
  float* costT;              // [Kp]     final DP costs
  int32_t* sel;              // [T]
  float* best_cost;          // [1]
  float* search_mjac;        // [1] or null: mjac of the selected path
  float* q_seed;             // [T][n] or null
  const float* q_in;         // [T][n] LM input
  float* q_out;              // [T][n]
  double* pose_err;          // [T][2] or null
  cpp_report_t* report;      // [1] or null
  int32_t* status;           // [1] or null
  const GeoF* geo;           // collision model or null
  float* clear;              // [T][Kp] smallest clearance or null
  double* smooth_ws;         // scratch of the trajectory-length step with collision rows, or null
};

// Kernels read requests and robots through one of two sources: a single request
// carried in the kernel parameters, or device arrays for a batch.
// A single request carries its collision model by value (has_geo); a batch
// request points at its model in the workspace (Req::geo).
struct SingleSrc {
  Req r;
  cpp_robot_t robot;
  int has_geo = 0;
  GeoF geo;
  __device__ __forceinline__ const Req& req(int) const { return r; }
  __device__ __forceinline__ const cpp_robot_t& rob(int) const { return robot; }
  __device__ __forceinline__ const GeoF* geom(const Req&) const { return has_geo ? &geo : nullptr; }
};
struct RobotViews;  // FP32 and FP64 views of a robot (below)
// Work distribution of a batched LM launch: robot views of the robot table,
// prefix sums of the requests' waypoint counts (wp_begin[r], nreq + 1 entries)
// and a counter that is zero when the launch starts.
struct LmAux {
  const RobotViews* views;
  const int* wp_begin;
  int* counter;
  int total, nreq;
};
struct BatchSrc {
  const Req* r;
  const cpp_robot_t* robots;
  LmAux lm;  // set by callers that run the LM on this table
  __device__ __forceinline__ const Req& req(int i) const { return r[i]; }
  __device__ __forceinline__ const cpp_robot_t& rob(int i) const { return robots[i]; }
  __device__ __forceinline__ const GeoF* geom(const Req& q) const { return q.geo; }
};

__device__ __forceinline__ void raise_status(int32_t* st, int code) {
  if (st) atomicMax(st, code);
}

// ------------------------------------------------------------------ robot in shared memory
struct RobotF {      // FP32 view for the FP32 kernels
  int n;
  float a[kMaxJ], d[kMaxJ], ca[kMaxJ], sa[kMaxJ], th0[kMaxJ];
  float lo[kMaxJ], hi[kMaxJ], nlo[kMaxJ], nhi[kMaxJ];
};
struct RobotD {      // FP64 view for the FP64 paths
  int n;
  double a[kMaxJ], d[kMaxJ], ca[kMaxJ], sa[kMaxJ], th0[kMaxJ], lo[kMaxJ], hi[kMaxJ];
};
// Both views of one robot in device memory (formed as stage_robot forms them with
// the FP64 view wanted): a lane of the batched LM may hold a waypoint of any
// request, so it reads its robot from an array of these.
struct RobotViews {
  RobotF f;
  RobotD d;
};

// Threads 0..15 of the block fill the views; the caller synchronises afterwards.
// Near-limit thresholds lo + m, hi - m are formed in FP64 and rounded once. The
// twist's cosine and sine come from FP64 sincos when the FP64 view is wanted,
// else from FP32 sincosf: kernels with many small blocks that only need the FP32
// view then spend no FP64 issue on staging (cos(pi/2) becomes -4.4e-8 instead of
// 6.1e-17, a ~1e-8 m change in the pose).
__device__ inline void stage_robot(const cpp_robot_t& r, double near_margin, RobotF* f,
                                   RobotD* dd) {
  const int j = threadIdx.x;
  if (j < kMaxJ) {
    double s = 0.0, c = 1.0;
    float sf, cf;
    if (dd) {
      sincos(r.alpha[j], &s, &c);
      sf = (float)s; cf = (float)c;
    } else {
      sincosf((float)r.alpha[j], &sf, &cf);
    }
    if (f) {
      f->a[j] = (float)r.a[j]; f->d[j] = (float)r.d[j];
      f->ca[j] = cf;           f->sa[j] = sf;
      f->th0[j] = (float)r.theta0[j];
      f->lo[j] = (float)r.lo[j]; f->hi[j] = (float)r.hi[j];
      f->nlo[j] = (float)(r.lo[j] + near_margin);
      f->nhi[j] = (float)(r.hi[j] - near_margin);
      if (j == 0) f->n = r.n;
    }
    if (dd) {
      dd->a[j] = r.a[j]; dd->d[j] = r.d[j]; dd->ca[j] = c; dd->sa[j] = s;
      dd->th0[j] = r.theta0[j]; dd->lo[j] = r.lo[j]; dd->hi[j] = r.hi[j];
      if (j == 0) dd->n = r.n;
    }
  }
}

// ------------------------------------------------------------------ DH chain
// Right-multiply the running pose (R row-major, p) by link j with joint angle
// cos/sin (ct, st). For each row (R0 R1 R2): u = ct R0 + st R1,
// w = ct R1 - st R0, new row = (u, ca w + sa R2, ca R2 - sa w), p += a u + d R2.
template <class F>
__device__ __forceinline__ void dh_step(F R[9], F p[3], F ct, F st, F ca, F sa, F a, F d) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const F R0 = R[3 * r], R1 = R[3 * r + 1], R2 = R[3 * r + 2];
    const F u = ct * R0 + st * R1;
    const F w = ct * R1 - st * R0;
    R[3 * r] = u;
    R[3 * r + 1] = ca * w + sa * R2;
    R[3 * r + 2] = ca * R2 - sa * w;
    p[r] = p[r] + a * u + d * R2;
  }
}

template <class F>
__device__ __forceinline__ void pose_identity(F R[9], F p[3]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = F(0);
  R[0] = R[4] = R[8] = F(1);
  p[0] = p[1] = p[2] = F(0);
}

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }

// FP32 FK of one configuration (NJ joints known at compile time, or NJ = 0 for
// a runtime n <= 16). The candidate path (masks, cpp_fk_batch) uses the
// hardware sine/cosine (__sincosf: absolute error below 2^-21.4 on [-pi, pi],
// which covers every in-limit joint angle; it carries at most a few 1e-6 m /
// rad into the pose), the LM uses the correctly range-reduced sincosf.
// The first link starts from the identity, so its product is written out: the
// same roundings as dh_step from the identity (one per product), without the
// multiplications by 0 and 1.
template <int NJ>
__device__ __forceinline__ void fk_f32(const RobotF& rb, const float* q, float R[9], float p[3]) {
  const int n = NJ ? NJ : rb.n;
  {
    float s, c;
    __sincosf(q[0] + rb.th0[0], &s, &c);
    const float ca = rb.ca[0], sa = rb.sa[0];
    R[0] = c; R[1] = -(ca * s); R[2] = sa * s;
    R[3] = s; R[4] = ca * c;    R[5] = -(sa * c);
    R[6] = 0.f; R[7] = sa;      R[8] = ca;
    p[0] = rb.a[0] * c; p[1] = rb.a[0] * s; p[2] = rb.d[0];
  }
#pragma unroll
  for (int j = 1; j < (NJ ? NJ : kMaxJ); ++j) {
    if (!NJ && j >= n) break;
    float s, c;
    __sincosf(q[j] + rb.th0[j], &s, &c);
    dh_step(R, p, c, s, rb.ca[j], rb.sa[j], rb.a[j], rb.d[j]);
  }
}

__device__ inline void fk_f64(const RobotD& rb, const double* q, double R[9], double p[3]) {
  pose_identity(R, p);
  for (int j = 0; j < rb.n; ++j) {
    double s, c;
    sincos(q[j] + rb.th0[j], &s, &c);
    dh_step(R, p, c, s, rb.ca[j], rb.sa[j], rb.a[j], rb.d[j]);
  }
}

// ------------------------------------------------------------------ rotations
// Unit quaternion (w, x, y, z), normalised first, to a row-major rotation (FP64).
__device__ inline void quat_to_rot(const double* q4, double R[9]) {
  const double inv = rsqrt(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
  const double w = q4[0] * inv, x = q4[1] * inv, y = q4[2] * inv, z = q4[3] * inv;
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z); R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y); R[7] = 2.0 * (y * z + w * x); R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Geodesic angle between two rotations (§II "Pose error"): the angle of
// E = Rt^T R from its skew part and trace, atan2(|vee(E - E^T)| / 2, (tr E - 1) / 2).
// Its parts: c = (tr E - 1) / 2 (the cosine of the angle) and vv = |vee(E - E^T)|^2
// (four times the squared sine), from which threshold tests need no root or atan2.
template <class F>
__device__ __forceinline__ void geodesic_parts(const F Rt[9], const F R[9], F& c, F& vv) {
  // E_ab = sum_c Rt_ca R_cb
  F tr = F(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) tr += Rt[i] * R[i];
  F vx = F(0), vy = F(0), vz = F(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    vx += Rt[3 * k + 2] * R[3 * k + 1] - Rt[3 * k + 1] * R[3 * k + 2];  // E21 - E12
    vy += Rt[3 * k + 0] * R[3 * k + 2] - Rt[3 * k + 2] * R[3 * k + 0];  // E02 - E20
    vz += Rt[3 * k + 1] * R[3 * k + 0] - Rt[3 * k + 0] * R[3 * k + 1];  // E10 - E01
  }
  vv = vx * vx + vy * vy + vz * vz;
  c = F(0.5) * (tr - F(1));
}
template <class F>
__device__ __forceinline__ F geodesic(const F Rt[9], const F R[9]) {
  F c, vv;
  geodesic_parts(Rt, R, c, vv);
  return atan2(F(0.5) * sqrt(vv), c);
}

// Rotation vector w = log(M) of a rotation M (world-frame LM residual).
// Small angles take w = vee(M - M^T) / 2, angles near pi take the axis from the
// largest diagonal entry of (M + I) / 2 with the sign of vee(M - M^T).
template <class F>
__device__ __forceinline__ void log_rot(const F M[9], F w[3], F small, F near_pi) {
  const F vx = M[7] - M[5], vy = M[2] - M[6], vz = M[3] - M[1];
  const F s = F(0.5) * sqrt(vx * vx + vy * vy + vz * vz);
  const F c = F(0.5) * (M[0] + M[4] + M[8] - F(1));
  const F th = atan2(s, c);
  if (th < small) {
    w[0] = F(0.5) * vx; w[1] = F(0.5) * vy; w[2] = F(0.5) * vz;
  } else if (th > F(3.141592653589793) - near_pi) {
    int m = 0;
    if (M[4] > M[0]) m = 1;
    if (M[8] > M[3 * m + m]) m = 2;
    F col[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) col[r] = F(0.5) * (M[3 * r + m] + (r == m ? F(1) : F(0)));
    const F nrm = sqrt(col[0] * col[0] + col[1] * col[1] + col[2] * col[2]);
    const F sg = (col[0] * vx + col[1] * vy + col[2] * vz) < F(0) ? F(-1) : F(1);
#pragma unroll
    for (int r = 0; r < 3; ++r) w[r] = sg * th * col[r] / nrm;
  } else {
    const F f = th / (F(2) * s);
    w[0] = f * vx; w[1] = f * vy; w[2] = f * vz;
  }
}

// ------------------------------------------------------------------ clusters
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// The shared::cluster address of the same shared-memory location in CTA `rank`.
__device__ __forceinline__ uint32_t map_peer(uint32_t smem_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ double ld_peer_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int ld_peer_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// ------------------------------------------------------------------ async copies
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared through the TMA engine; completion is counted
// in bytes on the mbarrier. Both addresses 16-byte aligned, size % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The same with acquire at cluster scope: the phase's bytes were written by
// other CTAs of the cluster (st.async with complete_tx).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Programmatic dependent launch (the single-request chain of stages): a kernel
// launched with the programmatic-serialization attribute may be scheduled while
// its predecessor in the stream finishes. pdl_trigger() lets the next kernel be
// scheduled once every CTA of this one has started; pdl_wait() blocks until the
// predecessor has completed and its writes are visible. Both return at once in
// an ordinary launch.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the mbarrier phase with a time limit (default 1 s). Returns false if
// the limit ran out; the caller then records CPP_ERR_TIMEOUT and stops.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = 1000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ bool mbar_wait_bounded_cluster(uint64_t* bar, uint32_t parity,
                                                          uint64_t limit_ns = 1000000000ull) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

}  // namespace cppflow
