// batchopt.cu -- cpf-BatchOpt (paper §III, in its commented text): refine the
// smoothest of the K candidate trajectories directly, without the search. Lane k
// across the waypoints is one candidate trajectory (a generative IK model's
// motion plan); its smoothness is its mjac, max over steps and joints of
// |q_{i+1,k,j} - q_{i,k,j}| in FP32 (+inf if it holds a non-finite value). The
// `lanes` smoothest lanes (ascending mjac, lowest index first among equals) are
// gathered into trajectories, refined by the batched LM (one pseudo-request per
// lane) and checked; the first valid one in that order is reported.
#include <cstring>
#include <vector>

#include "internal.h"

namespace cppflow {

constexpr int kSelThreads = 1024;

__global__ void lane_mjac_kernel(const float* __restrict__ cand, int T, int K, int Kp, int n,
                                 float* __restrict__ mjac) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  float m = 0.f;
  bool finite = true;
  for (int i = 0; i < T; ++i)
    for (int j = 0; j < n; ++j) {
      const float v = cand[((size_t)i * n + j) * Kp + k];
      finite = finite && isfinite(v);
      if (i + 1 < T) {
        const float d = fabsf(cand[((size_t)(i + 1) * n + j) * Kp + k] - v);
        if (d > m) m = d;
      }
    }
  mjac[k] = finite ? m : CUDART_INF_F;
}

// One block: `lanes` rounds of a block-wide (value, index) minimum over the
// unused lanes (lowest index among equal values).
__global__ void __launch_bounds__(kSelThreads) select_lanes_kernel(const float* __restrict__ mjac,
                                                                   int K, int lanes,
                                                                   int32_t* __restrict__ sel,
                                                                   float* __restrict__ sel_mjac) {
  __shared__ uint32_t used[2048];  // K <= 65535 lanes
  __shared__ float wv[kSelThreads / 32];
  __shared__ int wi[kSelThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int w = tid; w < 2048; w += kSelThreads) used[w] = 0;
  __syncthreads();
  for (int l = 0; l < lanes; ++l) {
    float bv = CUDART_INF_F;
    int bi = 0x7fffffff;
    for (int k = tid; k < K; k += kSelThreads) {
      if (used[k >> 5] & (1u << (k & 31))) continue;
      const float v = mjac[k];
      if (v < bv || (v == bv && k < bi)) { bv = v; bi = k; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { wv[warp] = bv; wi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kSelThreads / 32; ++w)
        if (wv[w] < bv || (wv[w] == bv && wi[w] < bi)) { bv = wv[w]; bi = wi[w]; }
      sel[l] = bi;
      sel_mjac[l] = mjac[bi];
      used[bi >> 5] |= 1u << (bi & 31);
    }
    __syncthreads();
  }
}

__global__ void gather_lanes_kernel(const float* __restrict__ cand, int T, int Kp, int n,
                                    int lanes, const int32_t* __restrict__ sel,
                                    float* __restrict__ q) {
  const long long total = (long long)lanes * T * n;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(x / ((long long)T * n));
    const int r = (int)(x - (long long)l * T * n);
    const int i = r / n, j = r - i * n;
    q[x] = cand[((size_t)i * n + j) * Kp + sel[l]];
  }
}

__global__ void first_valid_kernel(const cpp_report_t* __restrict__ reps, int lanes,
                                   int32_t* __restrict__ best) {
  int b = -1;
  for (int l = 0; l < lanes && b < 0; ++l)
    if (reps[l].valid) b = l;
  *best = b;
}

BatchOptLayout batch_opt_layout(int T, int K, int n, int lanes) {
  BatchOptLayout L;
  size_t o = 0;
  L.mjac = o;  o += align256(sizeof(float) * (size_t)K);
  L.reqs = o;  o += align256(sizeof(Req) * (size_t)lanes);
  L.robot = o; o += align256(sizeof(cpp_robot_t));
  L.lm = o;    o += lm_aux_layout(1, lanes).total;
  L.q_in = o;  o += align256(sizeof(float) * (size_t)lanes * T * n);
  L.total = o;
  return L;
}

cudaError_t launch_batch_opt(const cpp_robot_t& robot, const cpp_params_t& P, const float* cand,
                             const double* targets, int T, int K, int Kp, int lanes, char* ws,
                             int32_t* sel, float* sel_mjac, float* q_out, double* pose_err,
                             cpp_report_t* reports, int32_t* best, int32_t* dev_status,
                             cudaStream_t st) {
  const int n = robot.n;
  const BatchOptLayout L = batch_opt_layout(T, K, n, lanes);
  float* mjac = reinterpret_cast<float*>(ws + L.mjac);
  float* q_in = reinterpret_cast<float*>(ws + L.q_in);
  std::vector<Req> reqs(lanes);
  for (int l = 0; l < lanes; ++l) {
    Req q;
    memset(&q, 0, sizeof(q));
    q.T = T; q.K = 1; q.Kp = 4; q.n = n; q.robot = 0;
    q.targets = targets;
    q.q_in = q_in + (size_t)l * T * n;
    q.q_out = q_out + (size_t)l * T * n;
    q.pose_err = pose_err ? pose_err + (size_t)l * T * 2 : nullptr;
    q.report = reports + l;
    q.status = dev_status;
    reqs[l] = q;
  }
  // pageable sources: staged before the calls return
  cudaError_t e = cudaMemcpyAsync(ws + L.reqs, reqs.data(), sizeof(Req) * lanes,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.robot, &robot, sizeof(cpp_robot_t), cudaMemcpyHostToDevice, st);
  // the LM's work distribution: waypoint prefix sums and the robot's views
  const LmAuxLayout LA = lm_aux_layout(1, lanes);
  std::vector<int> wp(lanes + 1);
  const int wp_total = lm_prefix(reqs.data(), lanes, wp.data());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.lm + LA.wp, wp.data(), sizeof(int) * (lanes + 1),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_robot_views(reinterpret_cast<const cpp_robot_t*>(ws + L.robot), 1,
                           reinterpret_cast<RobotViews*>(ws + L.lm + LA.views), st);
  if (e != cudaSuccess) return e;
  lane_mjac_kernel<<<(K + 255) / 256, 256, 0, st>>>(cand, T, K, Kp, n, mjac);
  select_lanes_kernel<<<1, kSelThreads, 0, st>>>(mjac, K, lanes, sel, sel_mjac);
  const long long total = (long long)lanes * T * n;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  gather_lanes_kernel<<<blocks, 256, 0, st>>>(cand, T, Kp, n, lanes, sel, q_in);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const BatchSrc src{reinterpret_cast<const Req*>(ws + L.reqs),
                     reinterpret_cast<const cpp_robot_t*>(ws + L.robot),
                     lm_aux_at(ws + L.lm, LA, lanes, wp_total)};
  if ((e = launch_lm_batch(src, n, lanes, T, P, st)) != cudaSuccess) return e;
  if ((e = launch_check_batch(src, lanes, P, st)) != cudaSuccess) return e;
  first_valid_kernel<<<1, 1, 0, st>>>(reports, lanes, best);
  return cudaGetLastError();
}

}  // namespace cppflow
