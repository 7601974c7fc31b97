// diag.cu -- diagnostics beside the planner (not part of the paper's method):
//  * an arithmetic throughput probe: the measured FP32 lane-operation rate the
//    search is compared with (its inner loop is FP32 adds and maxima) and the
//    measured FP64 rate the LM's normal equations are compared with;
//  * the FP64 geometric Jacobian of given configurations, for conditioning
//    reports (its smallest singular value along a path near a wrist singularity).
#include <cstdarg>
#include <cstdio>

#include "internal.h"

namespace cppflow {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;   // independent dependency chains per thread
constexpr int kUnroll = 8;   // links per chain per loop trip (keeps loop overhead off the issue slots)

// x = max(x + a, b) on kChains chains: one FP32 add and one FP32 max per link.
__global__ void __launch_bounds__(kProbeThreads) probe_fp32_kernel(long long trips, float a, float b,
                                                                   double* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
  for (long long t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        asm volatile("add.f32 %0, %0, %1;" : "+f"(x[c]) : "f"(a));
        asm volatile("max.f32 %0, %0, %1;" : "+f"(x[c]) : "f"(b));
      }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0f) *sink = s;  // never true; keeps the chains alive
}

// x = fma(x, a, b) in FP64 on kChains chains (2 flops per link).
__global__ void __launch_bounds__(kProbeThreads) probe_fp64_kernel(long long trips, double a, double b,
                                                                   double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (double)(threadIdx.x + c);
  for (long long t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c)
        asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) *sink = s;
}

// Geometric Jacobian of one FP64 configuration per thread.
__global__ void __launch_bounds__(128) jacobian_f64_kernel(const cpp_robot_t robot, const double* q,
                                                            long long N, double* J) {
  __shared__ RobotD rd;
  stage_robot(robot, 0.0, nullptr, &rd);
  __syncthreads();
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int n = rd.n;
  const double* qc = q + (size_t)c * n;
  double R[9], p[3], z[kMaxJ][3], o[kMaxJ][3];
  pose_identity(R, p);
  for (int j = 0; j < n; ++j) {
    z[j][0] = R[2]; z[j][1] = R[5]; z[j][2] = R[8];
    o[j][0] = p[0]; o[j][1] = p[1]; o[j][2] = p[2];
    double s, co;
    sincos(qc[j] + rd.th0[j], &s, &co);
    dh_step(R, p, co, s, rd.ca[j], rd.sa[j], rd.a[j], rd.d[j]);
  }
  double* Jc = J + (size_t)c * 6 * n;
  for (int j = 0; j < n; ++j) {
    const double dx = p[0] - o[j][0], dy = p[1] - o[j][1], dz = p[2] - o[j][2];
    Jc[0 * n + j] = z[j][1] * dz - z[j][2] * dy;
    Jc[1 * n + j] = z[j][2] * dx - z[j][0] * dz;
    Jc[2 * n + j] = z[j][0] * dy - z[j][1] * dx;
    Jc[3 * n + j] = z[j][0];
    Jc[4 * n + j] = z[j][1];
    Jc[5 * n + j] = z[j][2];
  }
}

cpp_status dfail(cpp_status s, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

}  // namespace
}  // namespace cppflow

using namespace cppflow;

extern "C" {

cpp_status cpp_peak_probe(int32_t kind, int32_t blocks_per_sm, int64_t iters, double* sink,
                          double* lane_ops, cpp_stream_t stream) {
  if (kind != CPP_PROBE_FP32 && kind != CPP_PROBE_FP64)
    return dfail(CPP_ERR_INVALID_ARG, "cpp_peak_probe: unknown kind %d", kind);
  if (blocks_per_sm < 1 || blocks_per_sm > 8)
    return dfail(CPP_ERR_INVALID_ARG, "cpp_peak_probe: blocks_per_sm outside [1, 8]");
  if (iters < 1 || iters > 1000000000LL)
    return dfail(CPP_ERR_INVALID_ARG, "cpp_peak_probe: iters outside [1, 1e9]");
  if (!sink) return dfail(CPP_ERR_INVALID_ARG, "cpp_peak_probe: sink is NULL");
  const long long trips = (iters + kUnroll - 1) / kUnroll;
  const long long links = trips * kUnroll;
  const int blocks = blocks_per_sm * device_sm_count();
  const double chains = (double)blocks * kProbeThreads * kChains;
  if (kind == CPP_PROBE_FP32) {
    probe_fp32_kernel<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(trips, 1e-7f, -1e30f, sink);
    if (lane_ops) *lane_ops = chains * (double)links * 2.0;
  } else {
    probe_fp64_kernel<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(trips, 0.999999, 1e-6, sink);
    if (lane_ops) *lane_ops = chains * (double)links * 2.0;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return dfail(CPP_ERR_CUDA, "cpp_peak_probe: %s", cudaGetErrorString(e));
  return CPP_OK;
}

cpp_status cpp_jacobian_f64(const cpp_robot_t* robot, const double* q, int64_t N, double* J,
                            cpp_stream_t stream) {
  if (!robot || robot->n < 1 || robot->n > CPP_MAX_JOINTS)
    return dfail(CPP_ERR_INVALID_ARG, "cpp_jacobian_f64: malformed robot");
  if (N < 0) return dfail(CPP_ERR_INVALID_ARG, "cpp_jacobian_f64: N < 0");
  if (N == 0) return CPP_OK;
  if (!q || !J) return dfail(CPP_ERR_INVALID_ARG, "cpp_jacobian_f64: NULL buffer");
  const unsigned blocks = (unsigned)((N + 127) / 128);
  jacobian_f64_kernel<<<blocks, 128, 0, (cudaStream_t)stream>>>(*robot, q, N, J);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return dfail(CPP_ERR_CUDA, "cpp_jacobian_f64: %s", cudaGetErrorString(e));
  return CPP_OK;
}

}  // extern "C"
