// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <math_constants.h>
#include <type_traits>

#include "common.cuh"

namespace cppflow {

// fk_mask.cu
cudaError_t launch_mask(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st);
// tasks_per_warp: 128-candidate tasks per warp (0: the default, 4)
cudaError_t launch_mask_batch(const BatchSrc& s, int n, int nreq, long long max_tasks,
                              const cpp_params_t& P, bool any_geo, cudaStream_t st,
                              int tasks_per_warp = 0);
long long mask_tasks(int T, int Kp);
cudaError_t launch_fk_batch(const cpp_robot_t& r, const float* q, long long N, float* R,
                            float* p, cudaStream_t st);
cudaError_t launch_fk_pose64(const cpp_robot_t& r, const double* q, long long N, double* pose,
                             cudaStream_t st);

// dp.cu
int bp_stride(int Kp);
size_t dp_smem_bytes(int n, int Kp);
bool dp_supported(int n, int Kp);
cudaError_t launch_dp(const SingleSrc& s, unsigned stages, int objective, cudaStream_t st);
cudaError_t launch_dp_batch(const BatchSrc& s, unsigned stages, int objective, int n, int nreq,
                            int max_T, int max_Kp, cudaStream_t st);
// the same with the forward sweep's form and successors per CTA (see launch_forward)
cudaError_t launch_dp_batch_form(const BatchSrc& s, unsigned stages, int objective, int n, int nreq,
                                 int max_T, int max_Kp, int form, int cpc, cudaStream_t st);

// dp_fwd_sum.cu, dp_fwd_minmax.cu
constexpr int kFormAuto = 0;     // clusters when one wave of them covers the requests
constexpr int kFormCta = 1;      // one CTA per request (throughput form)
constexpr int kFormCluster = 2;  // one thread-block cluster per request (latency form)
cudaError_t launch_forward_sum(const SingleSrc& s, int n, int nreq, int max_Kp, int form, int cpc,
                               cudaStream_t st);
cudaError_t launch_forward_sum(const BatchSrc& s, int n, int nreq, int max_Kp, int form, int cpc,
                               cudaStream_t st);
cudaError_t launch_forward_minmax(const SingleSrc& s, int n, int nreq, int max_Kp, int form,
                                  int cpc, cudaStream_t st);
cudaError_t launch_forward_minmax(const BatchSrc& s, int n, int nreq, int max_Kp, int form,
                                  int cpc, cudaStream_t st);
// the forward sweep of one objective over nreq requests of a table (cpc: successor
// candidates per CTA of the cluster form, 0 for the default)
cudaError_t launch_forward(const BatchSrc& s, int objective, int n, int nreq, int max_Kp, int form,
                           int cpc, cudaStream_t st);
// The search form with the highest edge rate per SM whose estimated time is at
// most budget_ms, else the fastest of them (see pick_search_form in dp.cu).
struct SearchForm {
  int form, cpc;   // forward sweep form and successors per CTA
  double est_ms;   // estimated search time
  int rank;        // index of the form (one CTA, wide 512, wide 256, 128, 64 per CTA)
};
SearchForm pick_search_form(int T, int Kp, double budget_ms);
int cluster_succ(int Kp, int cpc);  // successors per CTA of the cluster form (0: no cluster form)
int cluster_size(int Kp, int cpc);  // CTAs per cluster (0: no cluster form)
int device_sm_count();     // SMs of the current device

// lm.cu
// Robot views (RobotViews) of n robots, for the batched LM (one block per robot).
cudaError_t launch_robot_views(const cpp_robot_t* robots, int n, RobotViews* views,
                               cudaStream_t st);
cudaError_t launch_lm(const SingleSrc& s, const cpp_params_t& P, bool want_err, cudaStream_t st);
cudaError_t launch_lm_batch(const BatchSrc& s, int n, int nreq, int max_T, const cpp_params_t& P,
                            cudaStream_t st);
cudaError_t launch_smooth(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st);
// the refinement (pose phases and trajectory-length steps) of a batch; any_geo:
// some request has a collision model (its steps then carry the collision rows)
cudaError_t launch_lm_batch_geo(const BatchSrc& s, int n, int nreq, int max_T,
                                const cpp_params_t& P, bool any_geo, cudaStream_t st);
// one anytime improvement round of a batch: a trajectory-length step, a pose
// phase from the current trajectory, the check
cudaError_t launch_improve_batch(const BatchSrc& s, int n, int nreq, int max_T,
                                 const cpp_params_t& P, bool any_geo, cudaStream_t st);
size_t smooth_smem_bytes(int T, int n);  // shared memory of the trajectory-length step
int lm_launches(const cpp_params_t& P, bool any_geo);  // kernel launches of one refinement
cudaError_t launch_check(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st);
cudaError_t launch_check_batch(const BatchSrc& s, int nreq, const cpp_params_t& P,
                               cudaStream_t st);

// batchopt.cu
struct BatchOptLayout {  // workspace of cpf-BatchOpt: lane mjac, pseudo-request table, robot,
                         // gathered trajectories
  size_t mjac, reqs, robot, lm, q_in, total;
};
BatchOptLayout batch_opt_layout(int T, int K, int n, int lanes);
cudaError_t launch_batch_opt(const cpp_robot_t& robot, const cpp_params_t& P, const float* cand,
                             const double* targets, int T, int K, int Kp, int lanes, char* ws,
                             int32_t* sel, float* sel_mjac, float* q_out, double* pose_err,
                             cpp_report_t* reports, int32_t* best, int32_t* dev_status,
                             cudaStream_t st);

// capi.cu
void set_last_error(const char* msg);  // message returned by cpp_last_error()
size_t geo_bytes();                    // sizeof(GeoF)
// Validate a host collision model for an n-joint robot and convert it to the
// device form (FP32, capsules sorted by frame) in `out` (geo_bytes() bytes).
// Returns false with a message in err (>= 160 bytes) when the model is invalid.
bool make_geo(const cpp_geometry_t& g, int n, void* out, char* err);

// Launch of `kernel` with an optional thread-block cluster (cluster > 1) and, for
// the single-request chain (pdl), programmatic serialization after the previous
// kernel in the stream (the kernels call pdl_trigger / pdl_wait first).
template <class Src>
constexpr bool kPdl = std::is_same<Src, SingleSrc>::value;

template <class... KArgs, class... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, unsigned cluster, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  unsigned na = 0;
  if (cluster > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------------ workspace layouts
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct DpLayout {  // scratch of the search: layer minima, backpointers, final costs
  size_t pen_min, bp, costT, total;
};
inline DpLayout dp_layout(int T, int Kp) {
  DpLayout L;
  size_t o = 0;
  L.pen_min = o; o += align256((size_t)T * sizeof(float));
  L.bp = o;      o += align256((size_t)T * bp_stride(Kp) * sizeof(uint16_t));
  L.costT = o;   o += align256((size_t)Kp * sizeof(float));
  L.total = o;
  return L;
}

// Scratch of the trajectory-length step with collision rows: per waypoint the
// packed J^T J block and J^T r of its rows, the inverse Schur complement and the
// eliminated right-hand side (FP64).
inline size_t smooth_ws_bytes(int T, int n) {
  return (size_t)T * (n * (n + 1) / 2 + n + n * n + n) * sizeof(double);
}

struct PlanLayout {  // scratch of one whole plan: the search's, masks, node costs, seed,
                    // collision model, trajectory-length step
  DpLayout dp;
  size_t dp_base, mask, pen, q_seed, geo, smooth, total;
};
inline PlanLayout plan_layout(int T, int Kp, int n) {
  PlanLayout L;
  L.dp = dp_layout(T, Kp);
  size_t o = 0;
  L.dp_base = o; o += L.dp.total;
  L.mask = o;    o += align256((size_t)T * Kp);
  L.pen = o;     o += align256((size_t)T * Kp * sizeof(float));
  L.q_seed = o;  o += align256((size_t)T * n * sizeof(float));
  L.geo = o;     o += align256(geo_bytes());
  L.smooth = o;  o += align256(smooth_ws_bytes(T, n));
  L.total = o;
  return L;
}

// Device region of a batched LM's work distribution (LmAux): robot views of the
// robot table, waypoint prefix sums, the counter.
struct LmAuxLayout {
  size_t views, wp, counter, total;
};
inline LmAuxLayout lm_aux_layout(int n_views, int nreq) {
  LmAuxLayout L;
  size_t o = 0;
  L.views = o;   o += align256(sizeof(RobotViews) * (size_t)n_views);
  L.wp = o;      o += align256(sizeof(int) * (size_t)(nreq + 1));
  L.counter = o; o += 256;
  L.total = o;
  return L;
}
// Prefix sums of the waypoint counts of `reqs` (nreq + 1 entries); returns the total.
inline int lm_prefix(const Req* reqs, int nreq, int* wp) {
  int t = 0;
  for (int r = 0; r < nreq; ++r) { wp[r] = t; t += reqs[r].T; }
  wp[nreq] = t;
  return t;
}
inline LmAux lm_aux_at(char* base, const LmAuxLayout& L, int nreq, int total) {
  LmAux a;
  a.views = reinterpret_cast<const RobotViews*>(base + L.views);
  a.wp_begin = reinterpret_cast<const int*>(base + L.wp);
  a.counter = reinterpret_cast<int*>(base + L.counter);
  a.total = total;
  a.nreq = nreq;
  return a;
}

// Fill the scratch pointers of a request from a plan workspace at `base`.
inline void carve_plan(Req& q, char* base, const PlanLayout& L) {
  q.mask = reinterpret_cast<uint8_t*>(base + L.mask);
  q.pen = reinterpret_cast<float*>(base + L.pen);
  q.pen_min = reinterpret_cast<float*>(base + L.dp_base + L.dp.pen_min);
  q.bp = reinterpret_cast<uint16_t*>(base + L.dp_base + L.dp.bp);
  q.costT = reinterpret_cast<float*>(base + L.dp_base + L.dp.costT);
  q.q_seed = reinterpret_cast<float*>(base + L.q_seed);
  q.q_in = q.q_seed;
  q.smooth_ws = reinterpret_cast<double*>(base + L.smooth);
}

}  // namespace cppflow
