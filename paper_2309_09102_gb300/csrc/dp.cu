// dp.cu -- the global discrete search of paper §III-B: a dynamic programme over
// the layered graph whose nodes are the K candidates of each waypoint and whose
// edges join every node of step i to every node of step i+1, followed by
// backtracking.
//
// Recurrence (FP32, one rounding per operation, ties to the lowest k):
//   r_i[k]      = pen_i[k] - m_i,   m_i = min_{k<K} pen_i[k]  (0 if that is +inf)
//   C_0[k]      = r_0[k]
//   C_{i+1}[k'] = (min_k (C_i[k] + max_j |q_{i+1,k',j} - q_{i,k,j}|)) + r_{i+1}[k']
//   bp[i+1][k'] = lowest k attaining the min
// A per-waypoint constant in the node costs changes no path's rank; taking the
// costs relative to the cheapest node keeps the running FP32 cost small enough
// to resolve the joint jumps.
//
// Kernels
//   layer_min_kernel    m_i for every waypoint (one warp per waypoint)
//   dp3_forward_kernel  one CTA per request walks the T steps (n in {6, 7, 9},
//                       Kp <= 1024). Each layer's raw block q_i [n][Kp] and its
//                       node-cost row arrive in shared memory by 1-D bulk copies
//                       (TMA engine, mbarrier completion) a step ahead; every node
//                       of the current layer becomes a record [-q_k, C_k] in
//                       shared memory; each thread owns R successors whose joint
//                       values stay in registers, and two thread groups split
//                       the predecessors. Per edge: n subtractions, n - 1
//                       abs-max, one add, one min -- 2n + 1 FP32 lane
//                       operations, no HBM traffic except 2 bytes of backpointer
//                       per successor and step.
//   dpc_forward_kernel  the same sweep for one request spread over a cluster of CTAs
//                       (requests that one wave of clusters covers).
//   dp_forward_generic  any other n or Kp that fits shared memory (slow path).
// The forward kernels live in dp_forward.cuh, compiled once per objective
// (dp_fwd_sum.cu: summed jumps; dp_fwd_minmax.cu: the paper's min-max mjac).
//   dp_backtrack_kernel lowest argmin of C_{T-1}, then the serial walk
//                       k_i = bp[i+1][k_{i+1}] over backpointer rows staged into
//                       shared memory by 1-D bulk copies (TMA engine, mbarrier
//                       completion, double-buffered), then the seed gather.
#include "dp_forward.cuh"

namespace cppflow {

constexpr int kBtThreads = 256;
constexpr uint32_t kBtChunkBytes = 32768;

int bp_stride(int Kp) { return (Kp + 7) & ~7; }

size_t dp_smem_bytes(int n, int Kp) { return (size_t)(2 * n + 2) * Kp * sizeof(float); }

bool dp_supported(int n, int Kp) {
  if (dp_smem_bytes(n, Kp) > 227u * 1024u) return false;  // generic kernel
  const bool fast = (n == 6 || n == 7 || n == 9) && Kp <= 1024;
  return !fast || dp3_smem_bytes(n, Kp, (Kp + 127) / 128) <= 227u * 1024u;
}

// ------------------------------------------------------------------ layer minimum
template <class Src>
__global__ void __launch_bounds__(256) layer_min_kernel(const __grid_constant__ Src src) {
  pdl_trigger();
  pdl_wait();
  const Req& rq = src.req(blockIdx.y);
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= rq.T) return;
  const float* row = rq.pen + (size_t)i * rq.Kp;
  float m = CUDART_INF_F;
  for (int k = lane; k < rq.K; k += 32) m = fminf(m, row[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) rq.pen_min[i] = isinf(m) ? 0.f : m;
}

// ------------------------------------------------------------------ backtrack
template <class Src>
__global__ void __launch_bounds__(kBtThreads) dp_backtrack_kernel(const __grid_constant__ Src src) {
  pdl_trigger();
  pdl_wait();
  const Req& rq = src.req(blockIdx.x);
  const int T = rq.T, K = rq.K, Kb = rq.Kb, n = rq.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(128) uint16_t sbp[];
  __shared__ uint64_t bars[2];
  __shared__ float rv[kBtThreads / 32];
  __shared__ int rk[kBtThreads / 32];
  __shared__ int start_k;

  // lowest argmin of C_{T-1} over k < K (strict '<' scan per thread, then a
  // lexicographic (value, index) reduction)
  float bv = CUDART_INF_F;
  int bk = 0x7fffffff;
  for (int k = tid; k < K; k += kBtThreads) {
    const float v = rq.costT[k];
    if (v < bv) { bv = v; bk = k; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
    if (ov < bv || (ov == bv && ok < bk)) { bv = ov; bk = ok; }
  }
  if (lane == 0) { rv[warp] = bv; rk[warp] = bk; }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kBtThreads / 32; ++w)
      if (rv[w] < bv || (rv[w] == bv && rk[w] < bk)) { bv = rv[w]; bk = rk[w]; }
    if (bk == 0x7fffffff) bk = 0;
    start_k = bk;
    if (rq.best_cost) *rq.best_cost = bv;
    if (isinf(bv)) raise_status(rq.status, CPP_ERR_INFEASIBLE);

    // serial walk over staged backpointer rows
    const int row_bytes = Kb * (int)sizeof(uint16_t);
    const int L = max(1, min(T > 1 ? T - 1 : 1, (int)(kBtChunkBytes / row_bytes)));
    uint16_t* const buf0 = sbp;
    uint16_t* const buf1 = sbp + (size_t)L * Kb;
    int k = bk;
    rq.sel[T - 1] = k;
    // chunk c covers rows [lo_c, hi_c], hi_0 = T-1, descending to row 1
    auto chunk_hi = [&](int c) { return T - 1 - c * L; };
    auto issue = [&](int c) {
      const int hi = chunk_hi(c);
      if (hi < 1) return;
      const int lo = max(1, hi - L + 1);
      const uint32_t bytes = (uint32_t)(hi - lo + 1) * row_bytes;
      mbar_expect_tx(&bars[c & 1], bytes);
      bulk_g2s((c & 1) ? buf1 : buf0, rq.bp + (size_t)lo * Kb, bytes, &bars[c & 1]);
    };
    issue(0);
    issue(1);
    bool ok = true;
    for (int c = 0; chunk_hi(c) >= 1; ++c) {
      if (!mbar_wait_bounded(&bars[c & 1], (uint32_t)((c >> 1) & 1))) {
        raise_status(rq.status, CPP_ERR_TIMEOUT);
        ok = false;
        // both copies in flight (chunks c and c + 1) must land before the CTA
        // leaves: wait for each once more, again with a limit
        mbar_wait_bounded(&bars[c & 1], (uint32_t)((c >> 1) & 1));
        if (chunk_hi(c + 1) >= 1) mbar_wait_bounded(&bars[(c + 1) & 1], (uint32_t)(((c + 1) >> 1) & 1));
        break;
      }
      const int hi = chunk_hi(c), lo = max(1, hi - L + 1);
      const uint16_t* b = (c & 1) ? buf1 : buf0;
      // Every stored backpointer is below K. Rows a timed-out forward sweep never
      // wrote hold stale values, so the walk clamps each step to [0, K) and can
      // never leave the staged rows or the candidate lanes.
      for (int row = hi; row >= lo; --row) {
        k = min((int)b[(size_t)(row - lo) * Kb + k], K - 1);
        rq.sel[row - 1] = k;
      }
      // the buffer was read through the generic proxy; order those reads before
      // the next asynchronous write into it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(c + 2);
    }
    (void)ok;
  }
  __syncthreads();
  if (rq.search_mjac) {  // mjac of the selected path: max over steps and joints of |dq|
    float m = 0.f;
    for (int i = tid; i + 1 < T; i += kBtThreads) {
      const int a = rq.sel[i], b = rq.sel[i + 1];
      for (int j = 0; j < n; ++j)
        m = fmaxf(m, fabsf(rq.cand[((size_t)(i + 1) * n + j) * rq.Kp + b] -
                           rq.cand[((size_t)i * n + j) * rq.Kp + a]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) rv[warp] = m;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kBtThreads / 32; ++w) m = fmaxf(m, rv[w]);
      *rq.search_mjac = m;
    }
  }
  if (rq.q_seed) {
    for (int x = tid; x < T * n; x += kBtThreads) {
      const int i = x / n, j = x - i * n;
      const int k = rq.sel[i];
      rq.q_seed[x] = rq.cand[((size_t)i * n + j) * rq.Kp + k];
    }
  }
}

// ------------------------------------------------------------------ launchers
template <class Src>
static cudaError_t launch_dp_t(const Src& s, unsigned stages, int objective, int n, int nreq,
                               int max_T, int max_Kp, cudaStream_t st, int form = kFormAuto,
                               int cpc = 0) {
  cudaError_t e = cudaSuccess;
  if (stages & CPP_STAGE_LAYER_MIN) {
    dim3 grid((unsigned)((max_T + 7) / 8), (unsigned)nreq);
    if ((e = launch_k(layer_min_kernel<Src>, grid, dim3(256), 0, st, 1, kPdl<Src>, s)) != cudaSuccess)
      return e;
  }
  if (stages & CPP_STAGE_DP_FORWARD) {
    e = objective == CPP_DP_MINMAX ? launch_forward_minmax(s, n, nreq, max_Kp, form, cpc, st)
                                   : launch_forward_sum(s, n, nreq, max_Kp, form, cpc, st);
    if (e != cudaSuccess) return e;
  }
  if (stages & CPP_STAGE_BACKTRACK) {
    if ((e = allow_smem(dp_backtrack_kernel<Src>, 2 * kBtChunkBytes)) != cudaSuccess) return e;
    e = launch_k(dp_backtrack_kernel<Src>, dim3((unsigned)nreq), dim3(kBtThreads),
                 2 * kBtChunkBytes, st, 1, kPdl<Src>, s);
  }
  return e;
}

cudaError_t launch_dp(const SingleSrc& s, unsigned stages, int objective, cudaStream_t st) {
  return launch_dp_t(s, stages, objective, s.r.n, 1, s.r.T, s.r.Kp, st);
}

cudaError_t launch_dp_batch(const BatchSrc& s, unsigned stages, int objective, int n, int nreq,
                            int max_T, int max_Kp, cudaStream_t st) {
  return launch_dp_t(s, stages, objective, n, nreq, max_T, max_Kp, st);
}

cudaError_t launch_dp_batch_form(const BatchSrc& s, unsigned stages, int objective, int n, int nreq,
                                 int max_T, int max_Kp, int form, int cpc, cudaStream_t st) {
  return launch_dp_t(s, stages, objective, n, nreq, max_T, max_Kp, st, form, cpc);
}

cudaError_t launch_forward(const BatchSrc& s, int objective, int n, int nreq, int max_Kp, int form,
                           int cpc, cudaStream_t st) {
  return objective == CPP_DP_MINMAX ? launch_forward_minmax(s, n, nreq, max_Kp, form, cpc, st)
                                    : launch_forward_sum(s, n, nreq, max_Kp, form, cpc, st);
}

int device_sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

// Successor candidates per CTA of the cluster form: cpc (32, 64, 128: the record
// exchange form; 256, 512: the wide form, which exchanges node costs only) or the
// default (64 up to Kp = 512, 128 above), as long as the cluster has 2..8 CTAs,
// or up to 16 (a non-portable cluster size, opted into at launch) when 32 or 64
// per CTA is asked for explicitly.
// Per CTA at two CTAs per SM a one-CTA search sweeps about 7.7e9 edges/s on GB300
// (measured: 2.35e12 edges/s over 304 CTAs); relative to it, measured at full
// occupancy with T = 300: the wide cluster form at 512 successors per CTA 1.0 (K =
// 1024), at 256 per CTA 0.79 (K = 1024) and 0.98 (K = 512), the record-exchange
// form at 128 per CTA 0.66, and at 64 per CTA (bulk record copies) about the same
// per SM at twice the width (T = 300, K = 1024 alone: 1.88 ms on 16 CTAs), the
// fallback for the longest requests. A cluster of CS CTAs owning S successors
// each takes (T - 1) S Kp / (7.7e9 x efficiency) seconds.
SearchForm pick_search_form(int T, int Kp_, double budget_ms) {
  constexpr double kCtaEdgesPerS = 7.7e9;
  const double steps = T > 1 ? T - 1 : 1, Kp = Kp_;
  const SearchForm cand[5] = {
      {kFormCta, 0, steps * Kp * Kp / kCtaEdgesPerS * 1e3, 0},
      {kFormCluster, 512, steps * 512.0 * Kp / (kCtaEdgesPerS * 1.0) * 1e3, 1},
      {kFormCluster, 256, steps * 256.0 * Kp / (kCtaEdgesPerS * (Kp_ > 512 ? 0.79 : 0.98)) * 1e3, 2},
      {kFormCluster, 128, steps * 128.0 * Kp / (kCtaEdgesPerS * 0.66) * 1e3, 3},
      {kFormCluster, 64, steps * 64.0 * Kp / (kCtaEdgesPerS * 0.66) * 1e3, 4}};
  const SearchForm* last = &cand[0];
  for (const SearchForm& f : cand) {
    if (f.form == kFormCluster && cluster_size(Kp_, f.cpc) < 2) continue;  // no such cluster
    last = &f;
    if (f.est_ms <= budget_ms) return f;
  }
  return *last;
}

int cluster_succ(int Kp, int cpc) {
  if (Kp <= 64 || Kp > 1024) return 0;
  const int S = cpc ? cpc : (Kp <= 512 ? 64 : 128);
  if (S != 32 && S != 64 && S != 128 && S != 256 && S != 512) return 0;
  const int CS = (Kp + S - 1) / S;
  const int max_cs = (cpc == 64 || cpc == 32) ? 16 : 8;
  return CS >= 2 && CS <= max_cs ? S : 0;
}

int cluster_size(int Kp, int cpc) {
  const int S = cluster_succ(Kp, cpc);
  return S ? (Kp + S - 1) / S : 0;
}

}  // namespace cppflow
