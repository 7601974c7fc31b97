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
//   dp_forward_kernel   one CTA per request walks the T steps. The whole layer
//                       q_i ([n][Kp]) and C_i sit in shared memory; each thread
//                       owns R successor nodes k' whose joint values stay in
//                       registers, and streams every predecessor k through a
//                       float4 broadcast read (4 k per load). Per edge: n FADD,
//                       n-1 abs-max, one FADD, one compare/select -- pure ALU
//                       work, no HBM traffic except 2 bytes of backpointer.
//   dp_backtrack_kernel lowest argmin of C_{T-1}, then the serial walk
//                       k_i = bp[i+1][k_{i+1}] over backpointer rows staged into
//                       shared memory by 1-D bulk copies (TMA engine, mbarrier
//                       completion, double-buffered), then the seed gather.
#include "internal.h"

namespace cppflow {

constexpr int kDpThreads = 256;
constexpr int kBtThreads = 256;
constexpr uint32_t kBtChunkBytes = 32768;

int bp_stride(int Kp) { return (Kp + 7) & ~7; }

size_t dp_smem_bytes(int n, int Kp) { return (size_t)(2 * n + 2) * Kp * sizeof(float); }

size_t dp2_smem_bytes(int nj, int Kp);

bool dp_supported(int n, int Kp) {
  if (dp_smem_bytes(n, Kp) > 227u * 1024u) return false;
  const bool fast = (n == 6 || n == 7 || n == 9) && Kp <= 1024;
  return !fast || dp2_smem_bytes(n, Kp) <= 227u * 1024u;
}

// ------------------------------------------------------------------ layer minimum
template <class Src>
__global__ void __launch_bounds__(256) layer_min_kernel(const __grid_constant__ Src src) {
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

// ------------------------------------------------------------------ forward sweep
template <int NJ, int R>
__device__ __forceinline__ void load_own(const float* __restrict__ cand, int i, int Kp,
                                         const int (&kp)[R], float (&dst)[R][NJ]) {
  const float* layer = cand + (size_t)i * NJ * Kp;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < NJ; ++j) dst[r][j] = kp[r] < Kp ? __ldg(layer + (size_t)j * Kp + kp[r]) : 0.f;
}

#define CPP_DP_EDGE(CMP, OFF)                                              \
  {                                                                        \
    const float cv = c.CMP;                                                \
    _Pragma("unroll") for (int r = 0; r < R; ++r) {                        \
      float d = fabsf(qn[r][0] - qa[0].CMP);                               \
      _Pragma("unroll") for (int j = 1; j < NJ; ++j)                       \
          d = fmaxf(d, fabsf(qn[r][j] - qa[j].CMP));                       \
      const float v = cv + d;                                              \
      if (v < best[r]) {                                                   \
        best[r] = v;                                                       \
        arg[r] = 4 * k4 + (OFF);                                           \
      }                                                                    \
    }                                                                      \
  }

template <int NJ, int R, class Src>
__global__ void __launch_bounds__(kDpThreads) dp_forward_kernel(const __grid_constant__ Src src) {
  const Req& rq = src.req(blockIdx.x);
  const int T = rq.T, K = rq.K, Kp = rq.Kp, Kb = rq.Kb;
  extern __shared__ __align__(16) float sm[];
  // q layers at sm + b * NJ * Kp, cost vectors at sm + 2 * NJ * Kp + b * Kp (b = step parity)
  float* const qbase = sm;
  float* const cbase = sm + 2 * NJ * Kp;
  const int tid = threadIdx.x;
  const float* __restrict__ cand = rq.cand;

  // layer 0 and C_0
  {
    const float m0 = rq.pen_min[0];
    const float4* src4 = reinterpret_cast<const float4*>(cand);
    float4* dst4 = reinterpret_cast<float4*>(qbase);
    for (int x = tid; x < NJ * Kp / 4; x += kDpThreads) dst4[x] = __ldg(src4 + x);
    for (int k = tid; k < Kp; k += kDpThreads) cbase[k] = k < K ? rq.pen[k] - m0 : CUDART_INF_F;
  }
  int kp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) kp[r] = tid + r * kDpThreads;
  float qn[R][NJ];
  if (T > 1) load_own<NJ, R>(cand, 1, Kp, kp, qn);
  __syncthreads();

  const int K4 = (K + 3) >> 2, Kp4 = Kp >> 2;
  for (int i = 0; i + 1 < T; ++i) {
    const int cur = i & 1, nxt = cur ^ 1;
    const float4* __restrict__ q4 = reinterpret_cast<const float4*>(qbase + cur * NJ * Kp);
    const float4* __restrict__ c4 = reinterpret_cast<const float4*>(cbase + cur * Kp);
    float* qnxt = qbase + nxt * NJ * Kp;
    float* cnxt = cbase + nxt * Kp;

    float qnn[R][NJ];
    if (i + 2 < T) load_own<NJ, R>(cand, i + 2, Kp, kp, qnn);
    const float m1 = rq.pen_min[i + 1];
    float rpen[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
      rpen[r] = kp[r] < K ? __ldg(rq.pen + (size_t)(i + 1) * Kp + kp[r]) - m1 : CUDART_INF_F;

    float best[R];
    int arg[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { best[r] = CUDART_INF_F; arg[r] = 0; }

#pragma unroll 1
    for (int k4 = 0; k4 < K4; ++k4) {
      const float4 c = c4[k4];
      float4 qa[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) qa[j] = q4[j * Kp4 + k4];
      CPP_DP_EDGE(x, 0)
      CPP_DP_EDGE(y, 1)
      CPP_DP_EDGE(z, 2)
      CPP_DP_EDGE(w, 3)
    }

    uint16_t* bprow = rq.bp + (size_t)(i + 1) * Kb;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (kp[r] < Kp) {
        cnxt[kp[r]] = kp[r] < K ? best[r] + rpen[r] : CUDART_INF_F;
        bprow[kp[r]] = (uint16_t)arg[r];
#pragma unroll
        for (int j = 0; j < NJ; ++j) qnxt[j * Kp + kp[r]] = qn[r][j];
      }
    }
    __syncthreads();
    if (i + 2 < T) {
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < NJ; ++j) qn[r][j] = qnn[r][j];
    }
  }
  const float* cfin = cbase + ((T - 1) & 1) * Kp;
  for (int k = tid; k < Kp; k += kDpThreads) rq.costT[k] = cfin[k];
}

// ------------------------------------------------------------------ forward sweep, staged
// Second form of the sweep (used for n in {6, 7, 9}, Kp <= 1024):
//  * each layer's raw block q_i [n][Kp] and node-cost row pen_i arrive in shared
//    memory by 1-D bulk copies (TMA engine, mbarrier completion) issued two
//    steps ahead, so no thread waits on HBM inside the sweep;
//  * every node k of the current layer is a record [-q_{k,0} .. -q_{k,n-1}, C_k]
//    (NW floats, 16-byte multiple): one predecessor costs NW/4 broadcast float4
//    loads, and the joint differences are packed FP32 pair additions
//    q' + (-q) (bit-identical to q' - q, round-to-nearest);
//  * the sweep keeps only the running minimum per 32-node tile and the first
//    tile that lowered it; the lowest index attaining the minimum is then
//    recovered by re-evaluating that one tile. Same values, same ties.
template <int NJ>
struct Rec {
  static constexpr int NW = ((NJ + 1 + 3) / 4) * 4;  // floats per record
  static constexpr int NP = (NJ + 1) / 2;             // packed pairs of own joints
};

__device__ __forceinline__ uint64_t pack2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t addx2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// max_j |own_j - q_j| for one predecessor record (negated joints in rec[0..NJ-1]).
// The differences are packed pair additions own + (-q); the absolute values are
// folded into three-input max operations (max is exact, so any grouping gives the
// same value, and NaN terms are ignored as with fmaxf).
template <int NJ>
__device__ __forceinline__ float linf_rec(const uint64_t (&own)[Rec<NJ>::NP], const float* rec) {
  float a[2 * Rec<NJ>::NP];
#pragma unroll
  for (int p = 0; p < Rec<NJ>::NP; ++p) {
    if (2 * p + 1 < NJ) {
      unpack2(addx2(own[p], pack2(rec[2 * p], rec[2 * p + 1])), a[2 * p], a[2 * p + 1]);
    } else {
      float ol, oh;
      unpack2(own[p], ol, oh);
      a[2 * p] = ol + rec[2 * p];
    }
  }
  if (NJ == 1) return fabsf(a[0]);
  if (NJ == 2) return fmaxf(fabsf(a[0]), fabsf(a[1]));
  float d = max3f(fabsf(a[0]), fabsf(a[1]), fabsf(a[2]));
  int j = 3;
#pragma unroll
  for (; j + 1 < NJ; j += 2) d = max3f(d, fabsf(a[j]), fabsf(a[j + 1]));
  if (j < NJ) d = fmaxf(d, fabsf(a[j]));
  return d;
}

constexpr int kDp2Threads = 256;
constexpr int kDp2Tile = 32;

// Records of one layer: node k at float offset k * NW + (k / 32) * 4. The
// 16-byte skew per 32-node tile puts the same slot of different tiles on
// different shared-memory banks (the tile rescan reads one tile per thread).
__host__ __device__ __forceinline__ int rec_layer_floats(int NW, int Kp) {
  return Kp * NW + ((Kp + 31) / 32) * 4;
}
__device__ __forceinline__ int rec_off(int NW, int k) { return k * NW + (k >> 5) * 4; }

size_t dp2_smem_bytes(int nj, int Kp) {
  const int NW = ((nj + 1 + 3) / 4) * 4;
  return (size_t)2 * rec_layer_floats(NW, Kp) * 4  // records, two layers
         + (size_t)2 * nj * Kp * 4    // raw layer staging, two slots
         + (size_t)2 * Kp * 4         // node-cost staging, two slots
         + 64;                        // barriers
}

template <int NJ, int R, class Src>
__global__ void __launch_bounds__(kDp2Threads) dp2_forward_kernel(const __grid_constant__ Src src) {
  constexpr int NW = Rec<NJ>::NW, NP = Rec<NJ>::NP;
  const Req& rq = src.req(blockIdx.x);
  const int T = rq.T, K = rq.K, Kp = rq.Kp, Kb = rq.Kb;
  const int tid = threadIdx.x;
  extern __shared__ __align__(128) float sm2[];
  const int RL = rec_layer_floats(NW, Kp);
  float* const rec = sm2;                                 // [2][RL] (records, skewed)
  float* const stg = rec + 2 * (size_t)RL;                // [2][NJ][Kp]
  float* const pst = stg + 2 * (size_t)NJ * Kp;           // [2][Kp]
  uint64_t* const bars = reinterpret_cast<uint64_t*>(pst + 2 * (size_t)Kp);
  __shared__ int timeout_flag;

  const uint32_t layer_bytes = (uint32_t)(NJ * Kp * 4), pen_bytes = (uint32_t)(Kp * 4);
  auto issue = [&](int L) {  // one thread: stage layer L into slot L & 1
    const int sl = L & 1;
    mbar_expect_tx(&bars[sl], layer_bytes + pen_bytes);
    bulk_g2s(stg + (size_t)sl * NJ * Kp, rq.cand + (size_t)L * NJ * Kp, layer_bytes, &bars[sl]);
    bulk_g2s(pst + (size_t)sl * Kp, rq.pen + (size_t)L * Kp, pen_bytes, &bars[sl]);
  };
  auto wait_layer = [&](int L) -> bool {
    return mbar_wait_bounded(&bars[L & 1], (uint32_t)((L >> 1) & 1));
  };

  if (tid == 0) {
    timeout_flag = 0;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    issue(0);
    if (T > 1) issue(1);
  }
  if (!wait_layer(0)) atomicExch(&timeout_flag, 1);
  {
    const float m0 = rq.pen_min[0];
    for (int k = tid; k < Kp; k += kDp2Threads) {
      float* rk = rec + rec_off(NW, k);
#pragma unroll
      for (int j = 0; j < NJ; ++j) rk[j] = -stg[(size_t)j * Kp + k];
      rk[NJ] = k < K ? pst[k] - m0 : CUDART_INF_F;
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) rk[j] = 0.f;
    }
  }
  __syncthreads();
  if (timeout_flag) {
    raise_status(rq.status, CPP_ERR_TIMEOUT);
    if (tid == 0 && T > 1) wait_layer(1);
    return;
  }
  if (tid == 0 && T > 2) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(2);
  }

  int kp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) kp[r] = tid + r * kDp2Threads;
  const int K4 = (K + 3) & ~3;
  const int ntiles = (K4 + kDp2Tile - 1) / kDp2Tile;

  for (int i = 0; i + 1 < T; ++i) {
    const int L = i + 1;
    if (!wait_layer(L)) atomicExch(&timeout_flag, 1);
    const float* sq = stg + (size_t)(L & 1) * NJ * Kp;
    const float* sp = pst + (size_t)(L & 1) * Kp;
    const float* rc = rec + (size_t)(i & 1) * RL;
    float* rn = rec + (size_t)(L & 1) * RL;
    const float m1 = rq.pen_min[L];

    uint64_t own[R][NP];
    float rpen[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = kp[r] < Kp ? kp[r] : Kp - 1;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float a = sq[(size_t)(2 * p) * Kp + k];
        const float b = (2 * p + 1 < NJ) ? sq[(size_t)(2 * p + 1) * Kp + k] : 0.f;
        own[r][p] = pack2(a, b);
      }
      rpen[r] = kp[r] < K ? sp[kp[r]] - m1 : CUDART_INF_F;
    }

    float best[R];
    int btile[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { best[r] = CUDART_INF_F; btile[r] = -1; }

#pragma unroll 1
    for (int t = 0; t < ntiles; ++t) {
      const int kb = t * kDp2Tile, ke = min(kb + kDp2Tile, K4);
      float tb[R];
#pragma unroll
      for (int r = 0; r < R; ++r) tb[r] = CUDART_INF_F;
#pragma unroll 2
      for (int k = kb; k < ke; k += 2) {  // ke - kb is a multiple of 4
        float r0[NW], r1[NW];
#pragma unroll
        for (int w = 0; w < NW; w += 4) {
          const float4 v = *reinterpret_cast<const float4*>(rc + rec_off(NW, k) + w);
          const float4 u = *reinterpret_cast<const float4*>(rc + rec_off(NW, k + 1) + w);
          r0[w] = v.x; r0[w + 1] = v.y; r0[w + 2] = v.z; r0[w + 3] = v.w;
          r1[w] = u.x; r1[w + 1] = u.y; r1[w + 2] = u.z; r1[w + 3] = u.w;
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
          tb[r] = min3f(tb[r], r0[NJ] + linf_rec<NJ>(own[r], r0), r1[NJ] + linf_rec<NJ>(own[r], r1));
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (tb[r] < best[r]) { best[r] = tb[r]; btile[r] = t; }
    }

    // lowest index attaining the minimum, inside the first tile that reached it
    uint16_t* bprow = rq.bp + (size_t)L * Kb;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int arg = 0;
      if (btile[r] >= 0) {
        const int kb = btile[r] * kDp2Tile, ke = min(kb + kDp2Tile, K4);
        for (int k = kb; k < ke; ++k) {
          const float* rk = rc + rec_off(NW, k);
          if (rk[NJ] + linf_rec<NJ>(own[r], rk) == best[r]) { arg = k; break; }
        }
      }
      if (kp[r] < Kp) {
        float v[NW];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          float a, b;
          unpack2(own[r][p], a, b);
          v[2 * p] = -a;
          if (2 * p + 1 < NJ) v[2 * p + 1] = -b;
        }
        v[NJ] = kp[r] < K ? best[r] + rpen[r] : CUDART_INF_F;
#pragma unroll
        for (int j = NJ + 1; j < NW; ++j) v[j] = 0.f;
        float4* dst = reinterpret_cast<float4*>(rn + rec_off(NW, kp[r]));
#pragma unroll
        for (int w = 0; w < NW / 4; ++w)
          dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
        bprow[kp[r]] = (uint16_t)arg;
      }
    }
    __syncthreads();
    if (timeout_flag) {
      raise_status(rq.status, CPP_ERR_TIMEOUT);
      if (tid == 0 && L + 1 < T) wait_layer(L + 1);
      return;
    }
    if (tid == 0 && L + 2 < T) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(L + 2);
    }
  }
  const float* rf = rec + (size_t)((T - 1) & 1) * RL;
  for (int k = tid; k < Kp; k += kDp2Threads) rq.costT[k] = rf[rec_off(NW, k) + NJ];
}

// ------------------------------------------------------------------ forward sweep, split
// Third form (the one used for n in {6, 7, 9}, Kp <= 1024). As the staged form,
// plus:
//  * the 256 threads form two groups of 128 that own the same R successors per
//    thread (Kp <= 128 R) and split the predecessor tiles in two contiguous
//    halves, so each broadcast record feeds R edges; the halves' (minimum,
//    tile) pairs merge through shared memory, the lower half winning ties, so
//    the lowest index still wins;
//  * one staging buffer and one record buffer: the bulk copy of layer i+2 is
//    issued as soon as every thread has taken its own layer-(i+1) values, and
//    the new records overwrite the old ones after the rescans;
//  * full 32-record tiles are unrolled from a tile base pointer.
constexpr int kDp3Threads = 256;
constexpr int kDp3Group = 128;

size_t dp3_smem_bytes(int nj, int Kp, int R) {
  const int NW = ((nj + 1 + 3) / 4) * 4;
  return (size_t)rec_layer_floats(NW, Kp) * 4  // records
         + (size_t)nj * Kp * 4                  // raw layer staging
         + (size_t)Kp * 4                       // node-cost staging
         + (size_t)3 * R * kDp3Group * 4        // group exchange: min, tile, index
         + 64;                                  // barrier
}

template <int NJ, int R>
__device__ __forceinline__ void sweep_pair(const uint64_t (&own)[R][Rec<NJ>::NP], const float* r0,
                                           const float* r1, float (&tb)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r)
    tb[r] = min3f(tb[r], r0[NJ] + linf_rec<NJ>(own[r], r0), r1[NJ] + linf_rec<NJ>(own[r], r1));
}

template <int NW>
__device__ __forceinline__ void load_rec(const float* p, float (&v)[NW]) {
#pragma unroll
  for (int w = 0; w < NW; w += 4) {
    const float4 x = *reinterpret_cast<const float4*>(p + w);
    v[w] = x.x; v[w + 1] = x.y; v[w + 2] = x.z; v[w + 3] = x.w;
  }
}

template <int NJ, int R, class Src>
__global__ void __launch_bounds__(kDp3Threads, 2) dp3_forward_kernel(const __grid_constant__ Src src) {
  constexpr int NW = Rec<NJ>::NW, NP = Rec<NJ>::NP;
  const Req& rq = src.req(blockIdx.x);
  const int T = rq.T, K = rq.K, Kp = rq.Kp, Kb = rq.Kb;
  const int tid = threadIdx.x, g = tid / kDp3Group, lt = tid % kDp3Group;
  extern __shared__ __align__(128) float sm3[];
  const int RL = rec_layer_floats(NW, Kp);
  float* const rec = sm3;                                   // [RL] records (skewed)
  float* const stg = rec + RL;                              // [NJ][Kp] staged layer
  float* const pst = stg + (size_t)NJ * Kp;                 // [Kp] staged node costs
  float* const xmin = pst + Kp;                             // [R][128]
  int* const xtile = reinterpret_cast<int*>(xmin + R * kDp3Group);  // [R][128]
  int* const xarg = xtile + R * kDp3Group;                  // [R][128]
  uint64_t* const bar = reinterpret_cast<uint64_t*>(xarg + R * kDp3Group);
  __shared__ int timeout_flag;

  const uint32_t layer_bytes = (uint32_t)(NJ * Kp * 4), pen_bytes = (uint32_t)(Kp * 4);
  auto issue = [&](int L) {  // one thread; layer L completes phase L of the barrier
    mbar_expect_tx(bar, layer_bytes + pen_bytes);
    bulk_g2s(stg, rq.cand + (size_t)L * NJ * Kp, layer_bytes, bar);
    bulk_g2s(pst, rq.pen + (size_t)L * Kp, pen_bytes, bar);
  };
  auto wait_layer = [&](int L) -> bool { return mbar_wait_bounded(bar, (uint32_t)(L & 1)); };

  if (tid == 0) {
    timeout_flag = 0;
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) issue(0);
  if (!wait_layer(0)) atomicExch(&timeout_flag, 1);
  {
    const float m0 = rq.pen_min[0];
    for (int k = tid; k < Kp; k += kDp3Threads) {
      float v[NW];
#pragma unroll
      for (int j = 0; j < NJ; ++j) v[j] = -stg[(size_t)j * Kp + k];
      v[NJ] = k < K ? pst[k] - m0 : CUDART_INF_F;
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) v[j] = 0.f;
      float4* dst = reinterpret_cast<float4*>(rec + rec_off(NW, k));
#pragma unroll
      for (int w = 0; w < NW / 4; ++w) dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
    }
  }
  __syncthreads();
  if (timeout_flag) {  // a copy that never completed: wait once more (bounded), then stop
    raise_status(rq.status, CPP_ERR_TIMEOUT);
    if (tid == 0) wait_layer(0);
    return;
  }
  if (tid == 0 && T > 1) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(1);
  }

  int kp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) kp[r] = lt + r * kDp3Group;
  const int K4 = (K + 3) & ~3;
  const int ntiles = (K4 + kDp2Tile - 1) / kDp2Tile;
  const int half = (ntiles + 1) / 2;
  const int t_lo = g == 0 ? 0 : half, t_hi = g == 0 ? half : ntiles;

  for (int i = 0; i + 1 < T; ++i) {
    const int L = i + 1;
    if (!wait_layer(L)) atomicExch(&timeout_flag, 1);
    uint64_t own[R][NP];
    float rpen[R];
    const float m1 = rq.pen_min[L];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = kp[r] < Kp ? kp[r] : Kp - 1;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float a = stg[(size_t)(2 * p) * Kp + k];
        const float b = (2 * p + 1 < NJ) ? stg[(size_t)(2 * p + 1) * Kp + k] : 0.f;
        own[r][p] = pack2(a, b);
      }
      rpen[r] = kp[r] < K ? pst[kp[r]] - m1 : CUDART_INF_F;
    }
    __syncthreads();  // everyone holds its layer-L values: the staging buffer is free
    if (timeout_flag) {
      raise_status(rq.status, CPP_ERR_TIMEOUT);
      if (tid == 0) wait_layer(L);
      return;
    }
    if (tid == 0 && L + 1 < T) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(L + 1);
    }

    float best[R];
    int btile[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { best[r] = CUDART_INF_F; btile[r] = -1; }
#pragma unroll 1
    for (int t = t_lo; t < t_hi; ++t) {
      const int kb = t * kDp2Tile;
      const float* base = rec + rec_off(NW, kb);
      float tb[R];
#pragma unroll
      for (int r = 0; r < R; ++r) tb[r] = CUDART_INF_F;
      if (kb + kDp2Tile <= K4) {
#pragma unroll
        for (int k = 0; k < kDp2Tile; k += 2) {
          float r0[NW], r1[NW];
          load_rec<NW>(base + k * NW, r0);
          load_rec<NW>(base + (k + 1) * NW, r1);
          sweep_pair<NJ, R>(own, r0, r1, tb);
        }
      } else {
        for (int k = 0; kb + k < K4; k += 2) {
          float r0[NW], r1[NW];
          load_rec<NW>(base + k * NW, r0);
          load_rec<NW>(base + (k + 1) * NW, r1);
          sweep_pair<NJ, R>(own, r0, r1, tb);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (tb[r] < best[r]) { best[r] = tb[r]; btile[r] = t; }
    }
    // merge the halves: the upper half (larger k) replaces only a strictly smaller minimum
    if (g == 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) { xmin[r * kDp3Group + lt] = best[r]; xtile[r * kDp3Group + lt] = btile[r]; }
    }
    __syncthreads();
    if (g == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float b1 = xmin[r * kDp3Group + lt];
        const int t1 = xtile[r * kDp3Group + lt];
        if (b1 < best[r]) { best[r] = b1; btile[r] = t1; }
        xmin[r * kDp3Group + lt] = best[r];
        xtile[r * kDp3Group + lt] = btile[r];
      }
    }
    __syncthreads();
    // rescans: successor r is handled by group r % 2 (group 0 when R == 1)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if ((R == 1 ? 0 : (r & 1)) != g) continue;
      const float bv = xmin[r * kDp3Group + lt];
      const int bt = xtile[r * kDp3Group + lt];
      int arg = 0;
      if (bt >= 0) {
        const int kb = bt * kDp2Tile, ke = min(kb + kDp2Tile, K4);
        const float* base = rec + rec_off(NW, kb);
        for (int k = kb; k < ke; ++k) {
          const float* rk = base + (k - kb) * NW;
          if (rk[NJ] + linf_rec<NJ>(own[r], rk) == bv) { arg = k; break; }
        }
      }
      xarg[r * kDp3Group + lt] = arg;
    }
    __syncthreads();  // rescans done: the records may be replaced
    uint16_t* bprow = rq.bp + (size_t)L * Kb;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if ((R == 1 ? 0 : (r & 1)) != g || kp[r] >= Kp) continue;
      float v[NW];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float a, b;
        unpack2(own[r][p], a, b);
        v[2 * p] = -a;
        if (2 * p + 1 < NJ) v[2 * p + 1] = -b;
      }
      v[NJ] = kp[r] < K ? xmin[r * kDp3Group + lt] + rpen[r] : CUDART_INF_F;
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) v[j] = 0.f;
      float4* dst = reinterpret_cast<float4*>(rec + rec_off(NW, kp[r]));
#pragma unroll
      for (int w = 0; w < NW / 4; ++w) dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
      bprow[kp[r]] = (uint16_t)xarg[r * kDp3Group + lt];
    }
    __syncthreads();
  }
  for (int k = tid; k < Kp; k += kDp3Threads) rq.costT[k] = rec[rec_off(NW, k) + NJ];
}

// Any n and Kp that fit in shared memory: successor values are read back from
// shared memory instead of registers.
template <class Src>
__global__ void __launch_bounds__(kDpThreads) dp_forward_generic(const __grid_constant__ Src src) {
  const Req& rq = src.req(blockIdx.x);
  const int T = rq.T, K = rq.K, Kp = rq.Kp, Kb = rq.Kb, n = rq.n;
  extern __shared__ __align__(16) float sm[];
  float* const qbase = sm;
  float* const cbase = sm + 2 * n * Kp;
  const int tid = threadIdx.x;
  const float* __restrict__ cand = rq.cand;
  const float m0 = rq.pen_min[0];
  for (int x = tid; x < n * Kp; x += kDpThreads) qbase[x] = cand[x];
  for (int k = tid; k < Kp; k += kDpThreads) cbase[k] = k < K ? rq.pen[k] - m0 : CUDART_INF_F;
  __syncthreads();
  for (int i = 0; i + 1 < T; ++i) {
    const int cur = i & 1, nxt = cur ^ 1;
    const float* qc = qbase + cur * n * Kp;
    const float* cc = cbase + cur * Kp;
    float* qx = qbase + nxt * n * Kp;
    float* cx = cbase + nxt * Kp;
    const float* layer = cand + (size_t)(i + 1) * n * Kp;
    for (int x = tid; x < Kp; x += kDpThreads)
      for (int j = 0; j < n; ++j) qx[j * Kp + x] = layer[(size_t)j * Kp + x];
    const float m1 = rq.pen_min[i + 1];
    for (int x = tid; x < Kp; x += kDpThreads) {
      float best = CUDART_INF_F;
      int arg = 0;
      for (int k = 0; k < K; ++k) {
        float d = fabsf(qx[x] - qc[k]);
        for (int j = 1; j < n; ++j) d = fmaxf(d, fabsf(qx[j * Kp + x] - qc[j * Kp + k]));
        const float v = cc[k] + d;
        if (v < best) { best = v; arg = k; }
      }
      cx[x] = x < K ? best + (rq.pen[(size_t)(i + 1) * Kp + x] - m1) : CUDART_INF_F;
      rq.bp[(size_t)(i + 1) * Kb + x] = (uint16_t)arg;
    }
    __syncthreads();
  }
  const float* cfin = cbase + ((T - 1) & 1) * Kp;
  for (int k = tid; k < Kp; k += kDpThreads) rq.costT[k] = cfin[k];
}

// ------------------------------------------------------------------ backtrack
template <class Src>
__global__ void __launch_bounds__(kBtThreads) dp_backtrack_kernel(const __grid_constant__ Src src) {
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
        if (chunk_hi(c + 1) >= 1) mbar_wait_bounded(&bars[(c + 1) & 1], (uint32_t)(((c + 1) >> 1) & 1));
        break;
      }
      const int hi = chunk_hi(c), lo = max(1, hi - L + 1);
      const uint16_t* b = (c & 1) ? buf1 : buf0;
      for (int row = hi; row >= lo; --row) {
        k = b[(size_t)(row - lo) * Kb + k];
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
  if (rq.q_seed) {
    for (int x = tid; x < T * n; x += kBtThreads) {
      const int i = x / n, j = x - i * n;
      const int k = rq.sel[i];
      rq.q_seed[x] = rq.cand[((size_t)i * n + j) * rq.Kp + k];
    }
  }
}

// ------------------------------------------------------------------ launchers
template <class KernelT>
static cudaError_t allow_smem(KernelT kernel, size_t bytes) {
  if (bytes <= 48u * 1024u) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int NJ, int R, class Src>
static cudaError_t launch_fwd_r(const Src& s, int nreq, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_smem(dp_forward_kernel<NJ, R, Src>, smem);
  if (e != cudaSuccess) return e;
  dp_forward_kernel<NJ, R, Src><<<nreq, kDpThreads, smem, st>>>(s);
  return cudaGetLastError();
}

template <int NJ, int R, class Src>
static cudaError_t launch_fwd2_r(const Src& s, int nreq, size_t smem, cudaStream_t st) {
  cudaError_t e = allow_smem(dp2_forward_kernel<NJ, R, Src>, smem);
  if (e != cudaSuccess) return e;
  dp2_forward_kernel<NJ, R, Src><<<nreq, kDp2Threads, smem, st>>>(s);
  return cudaGetLastError();
}

template <int NJ, int R, class Src>
static cudaError_t launch_fwd3_r(const Src& s, int nreq, int max_Kp, cudaStream_t st) {
  const size_t smem = dp3_smem_bytes(NJ, max_Kp, R);
  cudaError_t e = allow_smem(dp3_forward_kernel<NJ, R, Src>, smem);
  if (e != cudaSuccess) return e;
  dp3_forward_kernel<NJ, R, Src><<<nreq, kDp3Threads, smem, st>>>(s);
  return cudaGetLastError();
}

template <int NJ, class Src>
static cudaError_t launch_fwd_nj(const Src& s, int nreq, int max_Kp, cudaStream_t st) {
  const int R = (max_Kp + kDp3Group - 1) / kDp3Group;
  if (R <= 1) return launch_fwd3_r<NJ, 1>(s, nreq, max_Kp, st);
  if (R <= 2) return launch_fwd3_r<NJ, 2>(s, nreq, max_Kp, st);
  if (R <= 4) return launch_fwd3_r<NJ, 4>(s, nreq, max_Kp, st);
  return launch_fwd3_r<NJ, 8>(s, nreq, max_Kp, st);
}

template <class Src>
static cudaError_t launch_dp_t(const Src& s, unsigned stages, int n, int nreq, int max_T,
                               int max_Kp, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (stages & CPP_STAGE_LAYER_MIN) {
    dim3 grid((unsigned)((max_T + 7) / 8), (unsigned)nreq);
    layer_min_kernel<Src><<<grid, 256, 0, st>>>(s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (stages & CPP_STAGE_DP_FORWARD) {
    const bool fast = max_Kp <= 4 * kDpThreads;
    if (fast && n == 7) e = launch_fwd_nj<7>(s, nreq, max_Kp, st);
    else if (fast && n == 9) e = launch_fwd_nj<9>(s, nreq, max_Kp, st);
    else if (fast && n == 6) e = launch_fwd_nj<6>(s, nreq, max_Kp, st);
    else {
      const size_t smem = dp_smem_bytes(n, max_Kp);
      if ((e = allow_smem(dp_forward_generic<Src>, smem)) != cudaSuccess) return e;
      dp_forward_generic<Src><<<nreq, kDpThreads, smem, st>>>(s);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
  }
  if (stages & CPP_STAGE_BACKTRACK) {
    if ((e = allow_smem(dp_backtrack_kernel<Src>, 2 * kBtChunkBytes)) != cudaSuccess) return e;
    dp_backtrack_kernel<Src><<<nreq, kBtThreads, 2 * kBtChunkBytes, st>>>(s);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_dp(const SingleSrc& s, unsigned stages, cudaStream_t st) {
  return launch_dp_t(s, stages, s.r.n, 1, s.r.T, s.r.Kp, st);
}

cudaError_t launch_dp_batch(const BatchSrc& s, unsigned stages, int n, int nreq, int max_T,
                            int max_Kp, cudaStream_t st) {
  return launch_dp_t(s, stages, n, nreq, max_T, max_Kp, st);
}

}  // namespace cppflow
