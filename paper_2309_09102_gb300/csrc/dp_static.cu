// dp_static.cu -- the search entry point for callers that cannot allocate.
//
// cpp_dp_search needs device scratch (per-waypoint cost minima, the T x Kb
// backpointer table and the final cost row) that its caller allocates and
// passes in. Some callers cannot call cudaMalloc, or any allocating routine,
// at the point where they plan: hard real-time control loops that forbid
// allocation after start-up (an allocation can block for an unbounded time),
// and plug-ins whose host application owns every device allocation and gives
// them none of their own. cpp_dp_search_static serves them from one
// fixed-size scratch array that lives in this library's device image: it is
// reserved when the library is loaded on a device and held until the process
// exits, and the call itself allocates nothing.
//
// In host code the name of a __device__ array is only a host-side stand-in,
// not a device address; passing it to a kernel would fault (or, where the GPU
// can reach host memory, silently touch the wrong memory). The device address
// is therefore looked up once per device, with that device current, through
// cudaGetSymbolAddress, and cached. The cache does not survive a reset of the
// device (cudaDeviceReset, or a reset of its primary context): the cached
// address then points into a context that no longer exists, so a process that
// resets a device must not call this entry point on it afterwards.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace cppflow {
namespace {

static __device__ __align__(256) unsigned char g_dp_scratch[CPP_DP_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_dp_scratch on the current device (looked up on first use).
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dp_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

cpp_status reject(cpp_status s, const char* fmt, ...) {
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

extern "C" {

cpp_status cpp_dp_search_static(const float* cand, const float* pen, int32_t T, int32_t K,
                                int32_t Kp, int32_t n, int32_t* sel, float* best_cost,
                                float* q_seed, int32_t* dev_status, cpp_stream_t stream) {
  using namespace cppflow;
  if (T < 1 || K < 1 || K > 65535 || Kp < K || Kp % 4 != 0 || n < 1 || n > CPP_MAX_JOINTS)
    return reject(CPP_ERR_INVALID_ARG, "cpp_dp_search_static: invalid lattice T=%d K=%d Kp=%d n=%d",
                  T, K, Kp, n);
  if (!cand || !pen || !sel || !best_cost)
    return reject(CPP_ERR_INVALID_ARG, "cpp_dp_search_static: NULL buffer");
  if ((reinterpret_cast<uintptr_t>(cand) | reinterpret_cast<uintptr_t>(pen)) % 16 != 0)
    return reject(CPP_ERR_INVALID_ARG, "cpp_dp_search_static: cand and pen must be 16-byte aligned");
  if (!dp_supported(n, Kp))
    return reject(CPP_ERR_INVALID_ARG, "cpp_dp_search_static: Kp * (n + 1) too large for shared memory");
  const DpLayout L = dp_layout(T, Kp);
  const size_t need = L.total;
  if (need > (size_t)CPP_DP_STATIC_SCRATCH_BYTES)
    return reject(CPP_ERR_INVALID_ARG,
                  "cpp_dp_search_static: T=%d, Kp=%d needs %zu bytes of scratch but the static "
                  "scratch holds %zu; use cpp_dp_search with a caller workspace",
                  T, Kp, need, (size_t)CPP_DP_STATIC_SCRATCH_BYTES);
  void* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess)
    return reject(CPP_ERR_CUDA, "cpp_dp_search_static: cudaGetSymbolAddress: %s",
                  cudaGetErrorString(e));
  // Every scratch word the kernels read is written earlier in the same call
  // (layer minima, all Kp backpointers of rows 1..T-1, the final cost row), so
  // nothing left over from a previous call is used and nothing is cleared. The
  // one exception is a forward sweep that gives up on a bounded wait (status
  // CPP_ERR_TIMEOUT): the rows after that step keep an earlier call's values,
  // and the backtracking clamps every index it reads from them to [0, K).
  char* ws = static_cast<char*>(base);
  SingleSrc s{};  // value-initialised: every field not set below is zero
  s.r.T = T; s.r.K = K; s.r.Kp = Kp; s.r.n = n; s.r.Kb = bp_stride(Kp);
  s.r.cand = cand; s.r.pen = const_cast<float*>(pen);
  s.r.pen_min = reinterpret_cast<float*>(ws + L.pen_min);
  s.r.bp = reinterpret_cast<uint16_t*>(ws + L.bp);
  s.r.costT = reinterpret_cast<float*>(ws + L.costT);
  s.r.sel = sel; s.r.best_cost = best_cost; s.r.q_seed = q_seed; s.r.status = dev_status;
  e = launch_dp(s, CPP_STAGE_LAYER_MIN | CPP_STAGE_DP_FORWARD | CPP_STAGE_BACKTRACK, CPP_DP_SUM,
                (cudaStream_t)stream);
  if (e != cudaSuccess)
    return reject(CPP_ERR_CUDA, "cpp_dp_search_static: launch: %s", cudaGetErrorString(e));
  return CPP_OK;
}

}  // extern "C"
