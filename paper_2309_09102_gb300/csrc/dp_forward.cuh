// dp_forward.cuh -- the forward sweep of the global discrete search (paper
// §III-B), shared by dp_fwd_sum.cu (summed per-step L-inf jumps) and
// dp_fwd_minmax.cu (the paper's min-max mjac objective), which instantiate it
// for one objective each.
#pragma once

#include <atomic>

#include "internal.h"

namespace cppflow {

constexpr int kDpThreads = 256;

// ------------------------------------------------------------------ predecessor records
// Every node k of the current layer is a record [-q_{k,0} .. -q_{k,n-1}, C_k]
// (NW floats, a 16-byte multiple): one predecessor costs NW/4 broadcast float4
// loads, and the joint differences are additions q' + (-q) (bit-identical to
// q' - q, round-to-nearest). The sweep keeps only the running
// minimum per 16-node tile and the first tile that lowered it; the lowest index
// attaining the minimum is then recovered by re-evaluating that one tile. Same
// values, same ties.
template <int NJ>
struct Rec {
  static constexpr int NW = ((NJ + 1 + 3) / 4) * 4;  // floats per record
  static constexpr int NP = (NJ + 1) / 2;             // register pairs of own joints
};

__device__ __forceinline__ uint64_t pack2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}


// max_j |own_j - q_j| for one predecessor record (negated joints in rec[0..NJ-1]).
// IEEE subtraction a - b is a + (-b); max is exact, so the grouping does not
// matter, and NaN terms are ignored as with fmaxf. (Packed pair additions and
// three-input max/min give the same values but measured no faster on GB300:
// every one of the 2n + 1 operations per edge still occupies an FP32 lane.)
template <int NJ>
__device__ __forceinline__ float linf_rec(const uint64_t (&own)[Rec<NJ>::NP], const float* rec) {
  float d = 0.f;
#pragma unroll
  for (int p = 0; p < Rec<NJ>::NP; ++p) {
    float ol, oh;
    unpack2(own[p], ol, oh);
    const float a0 = fabsf(ol + rec[2 * p]);
    d = p == 0 ? a0 : fmaxf(d, a0);
    if (2 * p + 1 < NJ) d = fmaxf(d, fabsf(oh + rec[2 * p + 1]));
  }
  return d;
}

constexpr int kDp2Tile = 16;  // predecessor nodes per tile of the deferred argmin

// The search objective (§III-B): OBJ 0 sums the per-step L-inf jumps (C + d);
// OBJ 1 is the paper's own, the smallest mjac a path through the node can
// reach: a bottleneck path (max(C, d)). Node costs combine the same way. Both are exact IEEE operations.
template <int OBJ>
__device__ __forceinline__ float comb(float c, float d) {
  return OBJ ? fmaxf(c, d) : c + d;
}

// Records of one layer: node k at float offset k * NW + (k / 16) * 4. The
// 16-byte skew per 16-node tile puts the same slot of different tiles on
// different shared-memory banks (the tile rescan reads one tile per thread).
__host__ __device__ __forceinline__ int rec_layer_floats(int NW, int Kp) {
  return Kp * NW + ((Kp + kDp2Tile - 1) / kDp2Tile) * 4;
}
__device__ __forceinline__ int rec_off(int NW, int k) { return k * NW + (k / kDp2Tile) * 4; }

// ------------------------------------------------------------------ forward sweep
//  * the 256 threads form two groups of 128 that own the same R successors per
//    thread (Kp <= 128 R) and split the predecessor tiles in two contiguous
//    halves, so each broadcast record feeds R edges; the halves' (minimum,
//    tile) pairs merge through shared memory, the lower half winning ties, so
//    the lowest index still wins;
//  * one staging buffer and one record buffer: the bulk copy of layer i+2 is
//    issued as soon as every thread has taken its own layer-(i+1) values, and
//    the new records overwrite the old ones after the rescans;
//  * full 16-record tiles are unrolled from a tile base pointer.
constexpr int kDp3Threads = 256;
constexpr int kDp3Group = 128;

inline size_t dp3_smem_bytes(int nj, int Kp, int R) {
  const int NW = ((nj + 1 + 3) / 4) * 4;
  return (size_t)rec_layer_floats(NW, Kp) * 4  // records
         + (size_t)nj * Kp * 4                  // raw layer staging
         + (size_t)Kp * 4                       // node-cost staging
         + (size_t)4 * R * kDp3Group * 4        // group exchange: min, tile per group
         + 64;                                  // barrier
}

template <int NJ, int R, int OBJ>
__device__ __forceinline__ void sweep_pair(const uint64_t (&own)[R][Rec<NJ>::NP], const float* r0,
                                           const float* r1, float (&tb)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float v0 = comb<OBJ>(r0[NJ], linf_rec<NJ>(own[r], r0));
    const float v1 = comb<OBJ>(r1[NJ], linf_rec<NJ>(own[r], r1));
    tb[r] = fminf(fminf(tb[r], v0), v1);
  }
}

template <int NW>
__device__ __forceinline__ void load_rec(const float* p, float (&v)[NW]) {
#pragma unroll
  for (int w = 0; w < NW; w += 4) {
    const float4 x = *reinterpret_cast<const float4*>(p + w);
    v[w] = x.x; v[w + 1] = x.y; v[w + 2] = x.z; v[w + 3] = x.w;
  }
}

template <int NJ, int R, int OBJ, class Src>
__global__ void __launch_bounds__(kDp3Threads, 2) dp3_forward_kernel(const __grid_constant__ Src src) {
  pdl_trigger();
  pdl_wait();
  constexpr int NW = Rec<NJ>::NW, NP = Rec<NJ>::NP;
  const Req& rq = src.req(blockIdx.x);
  const int T = rq.T, K = rq.K, Kp = rq.Kp, Kb = rq.Kb;
  const int tid = threadIdx.x, g = tid / kDp3Group, lt = tid % kDp3Group;
  extern __shared__ __align__(128) float sm3[];
  const int RL = rec_layer_floats(NW, Kp);
  float* const rec = sm3;                                   // [RL] records (skewed)
  float* const stg = rec + RL;                              // [NJ][Kp] staged layer
  float* const pst = stg + (size_t)NJ * Kp;                 // [Kp] staged node costs
  float* const xmin = pst + Kp;                             // [2][R][128]
  int* const xtile = reinterpret_cast<int*>(xmin + 2 * R * kDp3Group);  // [2][R][128]
  uint64_t* const bar = reinterpret_cast<uint64_t*>(xtile + 2 * R * kDp3Group);
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
    // everyone holds its layer-L values (the staging buffer is free) and the
    // previous step's records are complete
    __syncthreads();
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
          sweep_pair<NJ, R, OBJ>(own, r0, r1, tb);
        }
      } else {
        for (int k = 0; kb + k < K4; k += 2) {
          float r0[NW], r1[NW];
          load_rec<NW>(base + k * NW, r0);
          load_rec<NW>(base + (k + 1) * NW, r1);
          sweep_pair<NJ, R, OBJ>(own, r0, r1, tb);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (tb[r] < best[r]) { best[r] = tb[r]; btile[r] = t; }
    }
    // both halves publish their (minimum, tile); successor r is finished by group r % 2
    // (group 0 when R == 1), which merges the halves -- the upper half (larger k)
    // replaces only a strictly smaller minimum, so the lowest index still wins --
    // and rescans the winning tile
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xmin[(g * R + r) * kDp3Group + lt] = best[r];
      xtile[(g * R + r) * kDp3Group + lt] = btile[r];
    }
    __syncthreads();
    float mv[R];
    int ma[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      mv[r] = 0.f;
      ma[r] = 0;
      if ((R == 1 ? 0 : (r & 1)) != g) continue;
      float bv = xmin[r * kDp3Group + lt];
      int bt = xtile[r * kDp3Group + lt];
      const float b1 = xmin[(R + r) * kDp3Group + lt];
      if (b1 < bv) { bv = b1; bt = xtile[(R + r) * kDp3Group + lt]; }
      int arg = 0;
      if (bt >= 0) {
        const int kb = bt * kDp2Tile, ke = min(kb + kDp2Tile, K4);
        const float* base = rec + rec_off(NW, kb);
        for (int k = kb; k < ke; ++k) {
          const float* rk = base + (k - kb) * NW;
          if (comb<OBJ>(rk[NJ], linf_rec<NJ>(own[r], rk)) == bv) { arg = k; break; }
        }
      }
      mv[r] = bv;
      ma[r] = arg;
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
      v[NJ] = kp[r] < K ? comb<OBJ>(mv[r], rpen[r]) : CUDART_INF_F;
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) v[j] = 0.f;
      float4* dst = reinterpret_cast<float4*>(rec + rec_off(NW, kp[r]));
#pragma unroll
      for (int w = 0; w < NW / 4; ++w) dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
      bprow[kp[r]] = (uint16_t)ma[r];
    }
    // the next step's first barrier orders these records before its sweep
  }
  __syncthreads();
  for (int k = tid; k < Kp; k += kDp3Threads) rq.costT[k] = rec[rec_off(NW, k) + NJ];
}

// ------------------------------------------------------------------ forward sweep, cluster
// One request alone (the plain per-request path, or a batch too small to fill
// the GPU) would leave most SMs idle with one CTA per request, and its T
// dependent steps would each run on a single SM. This form spreads one request
// over a thread-block cluster of CS CTAs (CS = ceil(Kp / 32R) <= 16):
//  * CTA c owns successors [32 R c, 32 R (c + 1)); its 8 warps split the
//    predecessor tiles into 8 contiguous ranges and keep the running minimum
//    per 16-node tile and the first tile that lowered it, as the one-CTA form;
//  * the 8 partial (minimum, tile) pairs merge in warp order, the lower range
//    winning ties, and the 8 warps re-evaluate 2 nodes each of the winning
//    tile for the lowest index attaining the minimum;
//  * each new record [-q', C'] goes into the record buffer of every CTA that
//    owns successors of the request by asynchronous distributed-shared-memory
//    stores that count their bytes on the receiving CTA's mbarrier for that
//    buffer; a CTA starts step i+1 once its barrier has seen all Kp records of
//    layer i+1 (a bounded wait). Records are double-buffered. A CTA writes
//    layer i+2 into a peer only after it has received the peer's layer-i+1
//    records, which the peer sends after its last read of the buffer that
//    layer i+2 overwrites, so no step needs a cluster-wide barrier. That
//    argument needs every receiver to be a sender too: CTAs of the cluster
//    beyond the request's own Kp (a launch's cluster fits its largest Kp) own
//    nothing, so they receive nothing either.
constexpr int kDpcThreads = 256;
constexpr int kDpcWarps = kDpcThreads / 32;
static_assert(kDp2Tile == 2 * kDpcWarps, "the rescan gives each warp 2 nodes of a tile");

// Floats from node lo's record to the end of node lo + n - 1's (the skew gaps
// between tiles included): one contiguous span of the record layout.
__host__ __device__ __forceinline__ int rec_span_floats(int NW, int lo, int n) {
  return (lo + n - 1) * NW + ((lo + n - 1) / kDp2Tile) * 4 + NW - (lo * NW + (lo / kDp2Tile) * 4);
}

inline size_t dpc_smem_bytes(int nj, int Kp, int R) {
  const int NW = ((nj + 1 + 3) / 4) * 4;
  return (size_t)2 * rec_layer_floats(NW, Kp) * 4 + (size_t)3 * kDpcWarps * 32 * R * 4 +
         (R <= 2 ? (size_t)2 * rec_span_floats(NW, 0, 32 * R) * 4 : 0);  // bulk send staging
}

// 16 bytes into a peer's shared memory; completion counts 16 bytes on the
// peer's mbarrier (both addresses from mapa).
__device__ __forceinline__ void st_async_v4(uint32_t addr, float4 v, uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::
          "r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
      : "memory");
}

// A bulk copy (TMA engine) from this CTA's shared memory into a CTA of the
// cluster; completion counts its bytes on that CTA's mbarrier (dst and bar from
// mapa). Both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_s2cluster(uint32_t dst, uint32_t src, uint32_t bytes,
                                               uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst), "r"(src), "r"(bytes), "r"(bar)
      : "memory");
}

template <int NJ, int R, int OBJ, class Src>
__global__ void __launch_bounds__(kDpcThreads) dpc_forward_kernel(const __grid_constant__ Src src,
                                                                   const int CS) {
  pdl_trigger();
  pdl_wait();
  constexpr int NW = Rec<NJ>::NW, NP = Rec<NJ>::NP, S = 32 * R;
  // how records travel: 32 and 64 successors per CTA (the latency forms) as one
  // bulk copy per owner CTA from a staging span written by warp 0; 128 per CTA
  // (a throughput form, 4 records per lane) by asynchronous stores from every
  // warp (measured: the single writing warp slowed that form in full batches)
  constexpr bool kBulk = R <= 2;
  const uint32_t crank = cluster_rank();
  const Req& rq = src.req(blockIdx.x / CS);
  const int T = rq.T, K = rq.K, Kp = rq.Kp, Kb = rq.Kb;
  // The cluster is sized for the launch's largest Kp. A CTA past this request's
  // own extent owns no successor: it sends nothing, so the owners never wait for
  // it and could run layers ahead of it, into buffers and barrier phases it has
  // not finished with. It takes no part in the exchange and only keeps the
  // cluster's two barriers.
  if ((int)crank * S >= Kp) {
    cluster_barrier();
    cluster_barrier();
    return;
  }
  const int CSr = (Kp + S - 1) / S;  // CTAs that own successors of this request
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(16) float smc[];
  const int RL = rec_layer_floats(NW, Kp);
  float* const recb = smc;                               // [2][RL] records (skewed)
  float* const xmin = recb + 2 * (size_t)RL;             // [warps][S]
  int* const xtile = reinterpret_cast<int*>(xmin + kDpcWarps * S);
  int* const xarg = xtile + kDpcWarps * S;
  const int SPAN = rec_span_floats(NW, 0, S);
  float* const sendb = reinterpret_cast<float*>(xarg + kDpcWarps * S);  // [2][SPAN] staging
  __shared__ uint64_t rbar[2];  // layer L's records arrive on rbar[L & 1]
  __shared__ int timeout_flag;
  const float* __restrict__ cand = rq.cand;
  // this CTA's records as one span of the layout, and the bytes a layer brings
  // (every owner's span, this CTA's own included)
  const int own_lo = (int)crank * S, own_n = min(S, Kp - own_lo);
  const int own_base = rec_off(NW, own_lo);
  const uint32_t own_bytes = (uint32_t)rec_span_floats(NW, own_lo, own_n) * 4u;
  uint32_t layer_bytes = kBulk ? 0u : (uint32_t)Kp * NW * 4u;
  for (int c = 0; kBulk && c < CSr; ++c)
    layer_bytes += (uint32_t)rec_span_floats(NW, c * S, min(S, Kp - c * S)) * 4u;
  if (tid == 0) {
    timeout_flag = 0;
    mbar_init(&rbar[0], 1);
    mbar_init(&rbar[1], 1);
    fence_mbar_init();
  }

  // layer 0: every CTA builds all records locally
  {
    const float m0 = rq.pen_min[0];
    for (int k = tid; k < Kp; k += kDpcThreads) {
      float v[NW];
#pragma unroll
      for (int j = 0; j < NJ; ++j) v[j] = -cand[(size_t)j * Kp + k];
      v[NJ] = k < K ? rq.pen[k] - m0 : CUDART_INF_F;
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) v[j] = 0.f;
      float4* dst = reinterpret_cast<float4*>(recb + rec_off(NW, k));
#pragma unroll
      for (int w = 0; w < NW / 4; ++w) dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
    }
  }
  int kp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) kp[r] = (int)crank * S + lane + 32 * r;
  float qn[R][NJ];  // own successor values and node costs of the next layer
  float pn[R], mn = 0.f;
  auto load_own = [&](int L) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = kp[r] < Kp ? kp[r] : Kp - 1;
#pragma unroll
      for (int j = 0; j < NJ; ++j) qn[r][j] = __ldg(cand + ((size_t)L * NJ + j) * Kp + k);
      pn[r] = __ldg(rq.pen + (size_t)L * Kp + k);
    }
    mn = __ldg(rq.pen_min + L);
  };
  if (T > 1) load_own(1);
  const int K4 = (K + 3) & ~3;
  const int ntiles = (K4 + kDp2Tile - 1) / kDp2Tile;
  const int t_lo = warp * ntiles / kDpcWarps, t_hi = (warp + 1) * ntiles / kDpcWarps;
  __syncthreads();
  cluster_barrier();

  // layer L >= 1 completes phase (L - 1) / 2 of rbar[L & 1]
  auto wait_layer = [&](int L) {
    if (!mbar_wait_bounded_cluster(&rbar[L & 1], (uint32_t)(((L - 1) >> 1) & 1))) {
      timeout_flag = 1;
      raise_status(rq.status, CPP_ERR_TIMEOUT);
    }
  };
  for (int i = 0; i + 1 < T; ++i) {
    const int L = i + 1;
    const float* cur = recb + (size_t)(i & 1) * RL;
    float* nxt = recb + (size_t)(L & 1) * RL;
    if (tid == 0) mbar_expect_tx(&rbar[L & 1], layer_bytes);
    if (i > 0) wait_layer(i);
    uint64_t own[R][NP];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int p = 0; p < NP; ++p)
        own[r][p] = pack2(qn[r][2 * p], (2 * p + 1 < NJ) ? qn[r][2 * p + 1] : 0.f);
    float rpen[R];
#pragma unroll
    for (int r = 0; r < R; ++r) rpen[r] = kp[r] < K ? pn[r] - mn : CUDART_INF_F;
    if (L + 1 < T) load_own(L + 1);  // prefetch, consumed next step

    float best[R];
    int btile[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { best[r] = CUDART_INF_F; btile[r] = -1; }
    // The records are swept a pair at a time (two pairs into two running minima for
    // one successor per lane), with the next pair already loaded (the first pair of
    // the next tile included), so the shared-memory load latency overlaps the
    // arithmetic before it: with 8 warps per SM it is not hidden otherwise. (min is
    // exact: the split changes no value.)
    float p0[NW], p1[NW];  // the pair swept next
    if (t_lo < t_hi) {
      const float* b0 = cur + rec_off(NW, t_lo * kDp2Tile);
      load_rec<NW>(b0, p0);
      load_rec<NW>(b0 + NW, p1);
    }
#pragma unroll 1
    for (int t = t_lo; t < t_hi; ++t) {
      const int kb = t * kDp2Tile;
      const float* base = cur + rec_off(NW, kb);
      // the next tile's first record (this tile's own first one for the last tile)
      const float* nbase = t + 1 < t_hi ? base + kDp2Tile * NW + 4 : base;
      float tb[R], tb2[R];  // two running minima (two pairs in flight), merged per tile
#pragma unroll
      for (int r = 0; r < R; ++r) tb[r] = tb2[r] = CUDART_INF_F;
      if (kb + kDp2Tile <= K4 && R == 1) {  // measured: two pairs in flight help only R = 1
#pragma unroll
        for (int k = 0; k < kDp2Tile; k += 4) {
          float q0[NW], q1[NW], n0[NW], n1[NW];
          load_rec<NW>(base + (k + 2) * NW, q0);
          load_rec<NW>(base + (k + 3) * NW, q1);
          const float* np = k + 4 < kDp2Tile ? base + (k + 4) * NW : nbase;
          load_rec<NW>(np, n0);
          load_rec<NW>(np + NW, n1);
          sweep_pair<NJ, R, OBJ>(own, p0, p1, tb);
          sweep_pair<NJ, R, OBJ>(own, q0, q1, tb2);
#pragma unroll
          for (int w = 0; w < NW; ++w) { p0[w] = n0[w]; p1[w] = n1[w]; }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) tb[r] = fminf(tb[r], tb2[r]);
      } else if (kb + kDp2Tile <= K4) {
#pragma unroll
        for (int k = 0; k < kDp2Tile; k += 2) {
          float q0[NW], q1[NW];
          const float* np = k + 2 < kDp2Tile ? base + (k + 2) * NW : nbase;
          load_rec<NW>(np, q0);
          load_rec<NW>(np + NW, q1);
          sweep_pair<NJ, R, OBJ>(own, p0, p1, tb);
#pragma unroll
          for (int w = 0; w < NW; ++w) { p0[w] = q0[w]; p1[w] = q1[w]; }
        }
      } else {  // the ragged last tile: its first pair is in p0, p1
        sweep_pair<NJ, R, OBJ>(own, p0, p1, tb);
        for (int k = 2; kb + k < K4; k += 2) {
          float r0[NW], r1[NW];
          load_rec<NW>(base + k * NW, r0);
          load_rec<NW>(base + (k + 1) * NW, r1);
          sweep_pair<NJ, R, OBJ>(own, r0, r1, tb);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (tb[r] < best[r]) { best[r] = tb[r]; btile[r] = t; }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xmin[warp * S + lane + 32 * r] = best[r];
      xtile[warp * S + lane + 32 * r] = btile[r];
    }
    __syncthreads();
    if (timeout_flag) break;  // CTA-uniform after the barrier
    // every warp merges the 8 ranges of its lane's slots in order (the same
    // result in all warps) and re-evaluates 2 records of the winning tile:
    // warp w takes nodes 2w, 2w + 1 of it, so the lowest match is the first
    // one in warp order
    float bvr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int slot = lane + 32 * r;
      float bv = xmin[slot];
      int bt = xtile[slot];
      for (int w = 1; w < kDpcWarps; ++w)
        if (xmin[w * S + slot] < bv) { bv = xmin[w * S + slot]; bt = xtile[w * S + slot]; }
      bvr[r] = bv;
      int found = 0x7fffffff;
      const int k0 = bt * kDp2Tile + 2 * warp;
      if (bt >= 0 && k0 < K4) {
        const float* r0 = cur + rec_off(NW, k0);
        if (comb<OBJ>(r0[NJ], linf_rec<NJ>(own[r], r0)) == bv) {
          found = k0;
        } else {
          const float* r1 = r0 + NW;  // k0 + 1 is in the same tile
          if (comb<OBJ>(r1[NJ], linf_rec<NJ>(own[r], r1)) == bv) found = k0 + 1;
        }
      }
      xarg[warp * S + slot] = found;
    }
    __syncthreads();
    // every warp takes the lowest match of its lane's slots. Bulk form: warp 0
    // writes the new records into the send staging (laid out as the span they
    // fill), which one bulk copy per owner CTA (this one included) carries into
    // its record buffer; the staging of layer L is rewritten for layer L + 2,
    // after every owner has sent layer L + 1, which each did only after receiving
    // layer L. Store form: warp w sends its lanes' records to CTAs w, w + 8.
    float* const sb = sendb + (size_t)(L & 1) * SPAN;
    int bsel[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int slot = lane + 32 * r;
      int ba = xarg[slot];
      for (int w = 1; w < kDpcWarps; ++w) ba = min(ba, xarg[w * S + slot]);
      bsel[r] = ba == 0x7fffffff ? 0 : ba;
      if ((kBulk && warp != 0) || kp[r] >= Kp) continue;
      float v[NW];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float a, b;
        unpack2(own[r][p], a, b);
        v[2 * p] = -a;
        if (2 * p + 1 < NJ) v[2 * p + 1] = -b;
      }
      v[NJ] = kp[r] < K ? comb<OBJ>(bvr[r], rpen[r]) : CUDART_INF_F;
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) v[j] = 0.f;
      if (kBulk) {
        float4* dst = reinterpret_cast<float4*>(sb + (rec_off(NW, kp[r]) - own_base));
#pragma unroll
        for (int w = 0; w < NW / 4; ++w) dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
      } else {
        const uint32_t base = smem_u32(nxt + rec_off(NW, kp[r])), bar = smem_u32(&rbar[L & 1]);
        for (int c = warp; c < CSr; c += kDpcWarps) {
          const uint32_t peer = map_peer(base, (uint32_t)c), pbar = map_peer(bar, (uint32_t)c);
#pragma unroll
          for (int w = 0; w < NW / 4; ++w)
            st_async_v4(peer + 16 * w, make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]),
                        pbar);
        }
      }
    }
    if (kBulk && warp == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the staging, to the copy engine
      __syncwarp();
      if (lane < CSr)
        bulk_s2cluster(map_peer(smem_u32(nxt + own_base), (uint32_t)lane), smem_u32(sb), own_bytes,
                       map_peer(smem_u32(&rbar[L & 1]), (uint32_t)lane));
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (warp == (r & (kDpcWarps - 1)) && kp[r] < Kp) rq.bp[(size_t)L * Kb + kp[r]] = (uint16_t)bsel[r];
  }
  if (T > 1 && !timeout_flag) wait_layer(T - 1);
  __syncthreads();
  if (!timeout_flag) {
    const float* fin = recb + (size_t)((T - 1) & 1) * RL;
    for (int k = (int)crank * S + tid; k < min(Kp, ((int)crank + 1) * S); k += kDpcThreads)
      rq.costT[k] = fin[rec_off(NW, k) + NJ];
  }
  cluster_barrier();  // no CTA leaves while a peer may still store into it
}

// ------------------------------------------------------------------ forward sweep, wide cluster
// The throughput form for long requests: the one-CTA sweep above spread over a
// cluster of CS CTAs (2..8), each owning S = 128 R successors (256 or 512), with
// only the node costs crossing the cluster:
//  * every CTA stages the whole next layer [n][Kp] and its node-cost row by 1-D
//    bulk copies (TMA engine) a step ahead, takes its own successors' values from
//    it, and writes the joint part [-q] of every node's record into the next
//    record buffer itself;
//  * the two thread groups split the predecessor tiles and merge as in the
//    one-CTA form, so the lowest index wins ties;
//  * the owner of successor k' sends C_{i+1}[k'] (4 bytes) into the record's cost
//    slot of every other CTA by an asynchronous distributed-shared-memory store
//    that counts its bytes on the receiver's mbarrier for that buffer; a CTA
//    starts step i+1 once its barrier has seen every peer's costs of layer i+1
//    (a bounded wait). Record buffers are double-buffered; a CTA writes layer
//    i+2's costs into a peer only after it has received the peer's layer i+1
//    costs, which the peer sends after its last read of the buffer that layer
//    i+2 overwrites, so no step needs a cluster-wide barrier (CTAs beyond the
//    request's own Kp send and receive nothing).
// Per step a CTA exchanges S * (CS - 1) * 4 bytes instead of S * (CS - 1) * 32,
// and sweeps S * Kp edges between three CTA barriers.
inline size_t dpx_smem_bytes(int nj, int Kp, int R) {
  const int NW = ((nj + 1 + 3) / 4) * 4;
  return (size_t)2 * rec_layer_floats(NW, Kp) * 4  // records, double-buffered
         + (size_t)nj * Kp * 4                      // raw layer staging
         + (size_t)Kp * 4                           // node-cost staging
         + (size_t)4 * R * kDp3Group * 4;           // group exchange
}

// 4 bytes into a peer's shared memory; completion counts 4 bytes on the peer's
// mbarrier (both addresses from mapa).
__device__ __forceinline__ void st_async_f32(uint32_t addr, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
               "r"(__float_as_uint(v)), "r"(bar)
               : "memory");
}

template <int NJ, int R, int OBJ, class Src>
__global__ void __launch_bounds__(kDp3Threads, 2) dpx_forward_kernel(const __grid_constant__ Src src,
                                                                      const int CS) {
  pdl_trigger();
  pdl_wait();
  constexpr int NW = Rec<NJ>::NW, NP = Rec<NJ>::NP, S = R * kDp3Group;
  const uint32_t crank = cluster_rank();
  const Req& rq = src.req(blockIdx.x / CS);
  const int T = rq.T, K = rq.K, Kp = rq.Kp, Kb = rq.Kb;
  // a CTA past this request's own extent owns no successor and stays out of the
  // exchange, as in the record-exchange form above
  if ((int)crank * S >= Kp) {
    cluster_barrier();
    cluster_barrier();
    return;
  }
  const int CSr = (Kp + S - 1) / S;  // CTAs that own successors of this request
  const int tid = threadIdx.x, g = tid / kDp3Group, lt = tid % kDp3Group;
  extern __shared__ __align__(128) float smx[];
  const int RL = rec_layer_floats(NW, Kp);
  float* const recb = smx;                                  // [2][RL] records (skewed)
  float* const stg = recb + 2 * (size_t)RL;                 // [NJ][Kp] staged layer
  float* const pst = stg + (size_t)NJ * Kp;                 // [Kp] staged node costs
  float* const xmin = pst + Kp;                             // [2][R][128]
  int* const xtile = reinterpret_cast<int*>(xmin + 2 * R * kDp3Group);  // [2][R][128]
  __shared__ uint64_t tbar;     // layer L's staging completes phase L
  __shared__ uint64_t cbar[2];  // peers' costs of layer L arrive on cbar[L & 1]
  __shared__ int timeout_flag;

  const int own_lo = (int)crank * S, own_n = min(S, Kp - own_lo);
  const uint32_t recv_bytes = (uint32_t)(Kp - own_n) * 4u;
  const uint32_t layer_bytes = (uint32_t)(NJ * Kp * 4), pen_bytes = (uint32_t)(Kp * 4);
  auto issue = [&](int L) {  // one thread
    mbar_expect_tx(&tbar, layer_bytes + pen_bytes);
    bulk_g2s(stg, rq.cand + (size_t)L * NJ * Kp, layer_bytes, &tbar);
    bulk_g2s(pst, rq.pen + (size_t)L * Kp, pen_bytes, &tbar);
  };
  if (tid == 0) {
    timeout_flag = 0;
    mbar_init(&tbar, 1);
    mbar_init(&cbar[0], 1);
    mbar_init(&cbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  cluster_barrier();  // every CTA's barriers exist before any peer stores into it
  int pending = -1;  // thread 0: the layer whose bulk copy is issued and not yet seen complete
  if (tid == 0) { issue(0); pending = 0; }
  if (!mbar_wait_bounded(&tbar, 0)) atomicExch(&timeout_flag, 1);
  else if (tid == 0) pending = -1;
  {  // layer 0: every CTA builds all records locally
    const float m0 = rq.pen_min[0];
    for (int k = tid; k < Kp; k += kDp3Threads) {
      float v[NW];
#pragma unroll
      for (int j = 0; j < NJ; ++j) v[j] = -stg[(size_t)j * Kp + k];
      v[NJ] = k < K ? pst[k] - m0 : CUDART_INF_F;
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) v[j] = 0.f;
      float4* dst = reinterpret_cast<float4*>(recb + rec_off(NW, k));
#pragma unroll
      for (int w = 0; w < NW / 4; ++w) dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
    }
  }
  __syncthreads();
  const bool ok0 = !timeout_flag;  // read right after a barrier: the same in every thread
  if (ok0 && tid == 0 && T > 1) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(1);
    pending = 1;
  }

  int kp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) kp[r] = own_lo + lt + r * kDp3Group;
  const int K4 = (K + 3) & ~3;
  const int ntiles = (K4 + kDp2Tile - 1) / kDp2Tile;
  const int half = (ntiles + 1) / 2;
  const int t_lo = g == 0 ? 0 : half, t_hi = g == 0 ? half : ntiles;
  for (int i = 0; ok0 && i + 1 < T; ++i) {
    const int L = i + 1;
    const float* cur = recb + (size_t)(i & 1) * RL;
    float* nxt = recb + (size_t)(L & 1) * RL;
    if (tid == 0) mbar_expect_tx(&cbar[L & 1], recv_bytes);
    // layer i's costs from the peers (layer 0 is local)
    if (i > 0 && !mbar_wait_bounded_cluster(&cbar[i & 1], (uint32_t)(((i - 1) >> 1) & 1)))
      atomicExch(&timeout_flag, 1);
    if (!mbar_wait_bounded(&tbar, (uint32_t)(L & 1))) atomicExch(&timeout_flag, 1);
    else if (tid == 0) pending = -1;
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
    // the joint part of every node's record of layer L (cost slots are filled by
    // the owners: this CTA below, the peers through the cluster)
    for (int k = tid; k < Kp; k += kDp3Threads) {
      float v[NW];
#pragma unroll
      for (int j = 0; j < NJ; ++j) v[j] = -stg[(size_t)j * Kp + k];
      float* dst = nxt + rec_off(NW, k);
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
#pragma unroll
      for (int j = 4; j < NJ; ++j) dst[j] = v[j];
#pragma unroll
      for (int j = NJ + 1; j < NW; ++j) dst[j] = 0.f;
    }
    // everyone holds its layer-L values (the staging buffer is free), layer i's
    // records are complete
    __syncthreads();
    if (timeout_flag) break;  // read right after a barrier: the same in every thread
    if (tid == 0 && L + 1 < T) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(L + 1);
      pending = L + 1;
    }

    float best[R];
    int btile[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { best[r] = CUDART_INF_F; btile[r] = -1; }
#pragma unroll 1
    for (int t = t_lo; t < t_hi; ++t) {
      const int kb = t * kDp2Tile;
      const float* base = cur + rec_off(NW, kb);
      float tb[R];
#pragma unroll
      for (int r = 0; r < R; ++r) tb[r] = CUDART_INF_F;
      if (kb + kDp2Tile <= K4) {
#pragma unroll
        for (int k = 0; k < kDp2Tile; k += 2) {
          float r0[NW], r1[NW];
          load_rec<NW>(base + k * NW, r0);
          load_rec<NW>(base + (k + 1) * NW, r1);
          sweep_pair<NJ, R, OBJ>(own, r0, r1, tb);
        }
      } else {
        for (int k = 0; kb + k < K4; k += 2) {
          float r0[NW], r1[NW];
          load_rec<NW>(base + k * NW, r0);
          load_rec<NW>(base + (k + 1) * NW, r1);
          sweep_pair<NJ, R, OBJ>(own, r0, r1, tb);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (tb[r] < best[r]) { best[r] = tb[r]; btile[r] = t; }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xmin[(g * R + r) * kDp3Group + lt] = best[r];
      xtile[(g * R + r) * kDp3Group + lt] = btile[r];
    }
    __syncthreads();
    // successor slot r is finished by group r % 2 (group 0 when R == 1): merge of the
    // halves (the upper half replaces only a strictly smaller minimum), rescan of the
    // winning tile, the cost sent to every CTA of the cluster
    uint16_t* bprow = rq.bp + (size_t)L * Kb;
    const uint32_t nbar = smem_u32(&cbar[L & 1]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if ((R == 1 ? 0 : (r & 1)) != g || kp[r] >= Kp) continue;
      float bv = xmin[r * kDp3Group + lt];
      int bt = xtile[r * kDp3Group + lt];
      const float b1 = xmin[(R + r) * kDp3Group + lt];
      if (b1 < bv) { bv = b1; bt = xtile[(R + r) * kDp3Group + lt]; }
      int arg = 0;
      if (bt >= 0) {
        const int kb = bt * kDp2Tile, ke = min(kb + kDp2Tile, K4);
        const float* base = cur + rec_off(NW, kb);
        for (int k = kb; k < ke; ++k) {
          const float* rk = base + (k - kb) * NW;
          if (comb<OBJ>(rk[NJ], linf_rec<NJ>(own[r], rk)) == bv) { arg = k; break; }
        }
      }
      const float c = kp[r] < K ? comb<OBJ>(bv, rpen[r]) : CUDART_INF_F;
      float* slot = nxt + rec_off(NW, kp[r]) + NJ;
      *slot = c;
      const uint32_t a = smem_u32(slot);
      for (int p = 1; p < CSr; ++p) {
        const uint32_t peer = (crank + (uint32_t)p) % (uint32_t)CSr;
        st_async_f32(map_peer(a, peer), c, map_peer(nbar, peer));
      }
      bprow[kp[r]] = (uint16_t)arg;
    }
    __syncthreads();  // rescans of `cur` done: the next step writes its joint part
  }
  __syncthreads();
  if (timeout_flag) {
    // a copy that never completed: wait for it once more (bounded) before leaving
    raise_status(rq.status, CPP_ERR_TIMEOUT);
    if (tid == 0 && pending >= 0) mbar_wait_bounded(&tbar, (uint32_t)(pending & 1));
  } else if (T > 1) {
    if (!mbar_wait_bounded_cluster(&cbar[(T - 1) & 1], (uint32_t)(((T - 2) >> 1) & 1)))
      raise_status(rq.status, CPP_ERR_TIMEOUT);
  }
  __syncthreads();
  if (!timeout_flag) {
    const float* fin = recb + (size_t)((T - 1) & 1) * RL;
    for (int k = own_lo + tid; k < own_lo + own_n; k += kDp3Threads) rq.costT[k] = fin[rec_off(NW, k) + NJ];
  }
  cluster_barrier();  // no CTA leaves while a peer may still store into it
}

// Any n and Kp that fit in shared memory: successor values are read back from
// shared memory instead of registers.
template <int OBJ, class Src>
__global__ void __launch_bounds__(kDpThreads) dp_forward_generic(const __grid_constant__ Src src) {
  pdl_trigger();
  pdl_wait();
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
        const float v = comb<OBJ>(cc[k], d);
        if (v < best) { best = v; arg = k; }
      }
      cx[x] = x < K ? comb<OBJ>(best, rq.pen[(size_t)(i + 1) * Kp + x] - m1) : CUDART_INF_F;
      rq.bp[(size_t)(i + 1) * Kb + x] = (uint16_t)arg;
    }
    __syncthreads();
  }
  const float* cfin = cbase + ((T - 1) & 1) * Kp;
  for (int k = tid; k < Kp; k += kDpThreads) rq.costT[k] = cfin[k];
}

// ------------------------------------------------------------------ launchers
template <class KernelT>
static cudaError_t allow_smem(KernelT kernel, size_t bytes) {
  if (bytes <= 48u * 1024u) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int NJ, int R, int OBJ, class Src>
static cudaError_t launch_fwd3_r(const Src& s, int nreq, int max_Kp, cudaStream_t st) {
  const size_t smem = dp3_smem_bytes(NJ, max_Kp, R);
  cudaError_t e = allow_smem(dp3_forward_kernel<NJ, R, OBJ, Src>, smem);
  if (e != cudaSuccess) return e;
  return launch_k(dp3_forward_kernel<NJ, R, OBJ, Src>, dim3((unsigned)nreq), dim3(kDp3Threads), smem,
                  st, 1, kPdl<Src>, s);
}

template <int NJ, int R, int OBJ, class Src>
static cudaError_t launch_fwdx_r(const Src& s, int nreq, int max_Kp, cudaStream_t st) {
  const int CS = (max_Kp + R * kDp3Group - 1) / (R * kDp3Group);
  const size_t smem = dpx_smem_bytes(NJ, max_Kp, R);
  cudaError_t e = allow_smem(dpx_forward_kernel<NJ, R, OBJ, Src>, smem);
  if (e != cudaSuccess) return e;
  return launch_k(dpx_forward_kernel<NJ, R, OBJ, Src>, dim3((unsigned)(nreq * CS)), dim3(kDp3Threads),
                  smem, st, (unsigned)CS, kPdl<Src>, s, CS);
}

template <int NJ, int R, int OBJ, class Src>
static cudaError_t launch_fwdc_r(const Src& s, int nreq, int max_Kp, cudaStream_t st) {
  const int CS = (max_Kp + 32 * R - 1) / (32 * R);
  const size_t smem = dpc_smem_bytes(NJ, max_Kp, R);
  cudaError_t e = allow_smem(dpc_forward_kernel<NJ, R, OBJ, Src>, smem);
  if (e != cudaSuccess) return e;
  if (CS > 8) {  // 9..16 CTAs: a non-portable cluster size
    e = cudaFuncSetAttribute(dpc_forward_kernel<NJ, R, OBJ, Src>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return launch_k(dpc_forward_kernel<NJ, R, OBJ, Src>, dim3((unsigned)(nreq * CS)), dim3(kDpcThreads),
                  smem, st, (unsigned)CS, kPdl<Src>, s, CS);
}

// Requests that one wave of clusters covers use the cluster form (lower latency);
// larger batches use one CTA per request (higher throughput).
static int sm_count() {
  static int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

// Whether 16-CTA clusters of this kernel (64 successors per CTA at Kp = 1024) can
// be resident on this device (asked once).
template <int NJ, int OBJ, class Src>
static bool cluster16_ok() {
  static const bool ok = [] {
    auto kernel = dpc_forward_kernel<NJ, 2, OBJ, Src>;
    const size_t smem = dpc_smem_bytes(NJ, 1024, 2);
    if (allow_smem(kernel, smem) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kDpcThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return clusters > 0;
  }();
  return ok;
}

// How many clusters of cs CTAs (32 R successors each) the device holds at once
// with one CTA per SM: a cluster lives inside one GPC, so past that count
// clusters share SMs and a step of the latency form slows down (asked once per
// size; 0 if none).
template <int NJ, int R, int OBJ, class Src>
static int spread_clusters(int cs) {
  static std::atomic<int> cache[17];  // value + 1; 0 = not asked yet
  if (cs < 2 || cs > 16) return 0;
  if (const int v = cache[cs].load(std::memory_order_relaxed)) return v - 1;
  auto kernel = dpc_forward_kernel<NJ, R, OBJ, Src>;
  constexpr size_t kOnePerSm = 120u * 1024u;  // more than half an SM's shared memory
  int clusters = 0;
  if (allow_smem(kernel, kOnePerSm) == cudaSuccess &&
      (cs <= 8 ||
       cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
           cudaSuccess)) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(kDpcThreads);
    cfg.dynamicSmemBytes = kOnePerSm;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess) clusters = 0;
  }
  cudaGetLastError();
  cache[cs].store(clusters + 1, std::memory_order_relaxed);
  return clusters;
}

template <int NJ, int OBJ, class Src>
static cudaError_t launch_fwd_nj(const Src& s, int nreq, int max_Kp, int form, int cpc,
                                 cudaStream_t st) {
  // the latency form takes the smallest tile (32 successors per CTA up to Kp =
  // 512, 64 above; clusters of up to 16 CTAs) when the device holds all the
  // requests' clusters at once with one CTA per SM
  if (cpc == 0 && form == kFormAuto && cluster16_ok<NJ, OBJ, Src>()) {
    if (max_Kp <= 512 && cluster_size(max_Kp, 32) > 0 &&
        nreq <= spread_clusters<NJ, 1, OBJ, Src>(cluster_size(max_Kp, 32)))
      cpc = 32;
    else if (max_Kp > 512 && nreq <= spread_clusters<NJ, 2, OBJ, Src>(cluster_size(max_Kp, 64)))
      cpc = 64;
  }
  const int S = cluster_succ(max_Kp, cpc), CS = cluster_size(max_Kp, cpc);
  if (S >= 256 && form != kFormCta && (form == kFormCluster || nreq * CS <= sm_count()))
    return S == 256 ? launch_fwdx_r<NJ, 2, OBJ>(s, nreq, max_Kp, st)
                    : launch_fwdx_r<NJ, 4, OBJ>(s, nreq, max_Kp, st);
  if (S > 0 && form != kFormCta && (form == kFormCluster || nreq * CS <= sm_count()))
    return S == 32 ? launch_fwdc_r<NJ, 1, OBJ>(s, nreq, max_Kp, st)
         : S == 64 ? launch_fwdc_r<NJ, 2, OBJ>(s, nreq, max_Kp, st)
                   : launch_fwdc_r<NJ, 4, OBJ>(s, nreq, max_Kp, st);
  const int R = (max_Kp + kDp3Group - 1) / kDp3Group;
  if (R <= 1) return launch_fwd3_r<NJ, 1, OBJ>(s, nreq, max_Kp, st);
  if (R <= 2) return launch_fwd3_r<NJ, 2, OBJ>(s, nreq, max_Kp, st);
  if (R <= 4) return launch_fwd3_r<NJ, 4, OBJ>(s, nreq, max_Kp, st);
  return launch_fwd3_r<NJ, 8, OBJ>(s, nreq, max_Kp, st);
}

// Forward sweep for n joints: the fast forms for n in {6, 7, 9} and Kp <= 1024
// (form: kFormAuto picks clusters when one wave of them covers the requests,
// kFormCta / kFormCluster force one; cpc: successor candidates per CTA of the
// cluster form, 64 or 128, 0 for the default), the generic kernel otherwise.
template <int OBJ, class Src>
static cudaError_t launch_forward_t(const Src& s, int n, int nreq, int max_Kp, int form, int cpc,
                                    cudaStream_t st) {
  const bool fast = max_Kp <= 1024;
  if (fast && n == 7) return launch_fwd_nj<7, OBJ>(s, nreq, max_Kp, form, cpc, st);
  if (fast && n == 9) return launch_fwd_nj<9, OBJ>(s, nreq, max_Kp, form, cpc, st);
  if (fast && n == 6) return launch_fwd_nj<6, OBJ>(s, nreq, max_Kp, form, cpc, st);
  const size_t smem = dp_smem_bytes(n, max_Kp);
  cudaError_t e = allow_smem(dp_forward_generic<OBJ, Src>, smem);
  if (e != cudaSuccess) return e;
  return launch_k(dp_forward_generic<OBJ, Src>, dim3((unsigned)nreq), dim3(kDpThreads), smem, st, 1,
                  kPdl<Src>, s);
}

}  // namespace cppflow
