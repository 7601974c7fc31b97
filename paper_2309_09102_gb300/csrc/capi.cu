// capi.cu -- host side of the C ABI in include/cppflow.h: argument checks,
// workspace carving and the kernel launch sequence of each call. Every call
// validates on the host before it enqueues anything, and reports failures as a
// cpp_status plus a thread-local message.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace cppflow;

namespace {

thread_local std::string g_err;

cpp_status fail(cpp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

cpp_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return CPP_OK;
  return fail(CPP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool finite_d(double v) { return std::isfinite(v); }

cpp_status check_robot(const cpp_robot_t* r) {
  if (!r) return fail(CPP_ERR_INVALID_ARG, "robot is NULL");
  if (r->n < 1 || r->n > CPP_MAX_JOINTS)
    return fail(CPP_ERR_INVALID_ARG, "robot.n = %d outside [1, %d]", r->n, CPP_MAX_JOINTS);
  for (int j = 0; j < r->n; ++j) {
    if (!finite_d(r->a[j]) || !finite_d(r->d[j]) || !finite_d(r->alpha[j]) ||
        !finite_d(r->theta0[j]) || !finite_d(r->lo[j]) || !finite_d(r->hi[j]))
      return fail(CPP_ERR_INVALID_ARG, "robot parameter of joint %d is not finite", j);
    if (!(r->lo[j] <= r->hi[j]))
      return fail(CPP_ERR_INVALID_ARG, "robot joint %d has lo > hi", j);
  }
  return CPP_OK;
}

cpp_status check_params(const cpp_params_t* p) {
  if (!p) return fail(CPP_ERR_INVALID_ARG, "params is NULL");
  const double v[] = {p->tau_pos, p->tau_rot, p->near_margin, p->pen_limit, p->pen_pose,
                      p->jump_max, p->lambda0, p->lambda_up, p->lambda_down, p->lambda_min,
                      p->lambda_max, p->freeze_step, p->freeze_cost};
  for (double x : v)
    if (!finite_d(x)) return fail(CPP_ERR_INVALID_ARG, "a params field is not finite");
  if (p->pen_limit < 0 || p->pen_pose < 0) return fail(CPP_ERR_INVALID_ARG, "negative node cost");
  if (p->lambda0 <= 0 || p->lambda_min <= 0 || p->lambda_max < p->lambda_min ||
      p->lambda_up < 1 || p->lambda_down < 1)
    return fail(CPP_ERR_INVALID_ARG, "invalid damping schedule");
  if (p->lm_iters < 0 || p->lm_iters > 100000) return fail(CPP_ERR_INVALID_ARG, "lm_iters out of range");
  if (p->dp_objective != CPP_DP_SUM && p->dp_objective != CPP_DP_MINMAX)
    return fail(CPP_ERR_INVALID_ARG, "dp_objective %d is neither CPP_DP_SUM nor CPP_DP_MINMAX",
                p->dp_objective);
  if (p->smooth_rounds < 0 || p->smooth_rounds > 1000)
    return fail(CPP_ERR_INVALID_ARG, "smooth_rounds outside [0, 1000]");
  if (!(finite_d(p->smooth_lambda) && p->smooth_lambda > 0))
    return fail(CPP_ERR_INVALID_ARG, "smooth_lambda must be finite and > 0");
  if (!(finite_d(p->pen_collide) && p->pen_collide >= 0))
    return fail(CPP_ERR_INVALID_ARG, "pen_collide must be finite and >= 0");
  if (!(finite_d(p->coll_margin) && p->coll_margin >= 0 && finite_d(p->coll_weight) &&
        p->coll_weight >= 0))
    return fail(CPP_ERR_INVALID_ARG, "coll_margin and coll_weight must be finite and >= 0");
  return CPP_OK;
}

constexpr size_t kMaxSmemBytes = 227u * 1024u;

// The trajectory-length step keeps (n + 1) T doubles in shared memory.
cpp_status check_smooth(const cpp_params_t* p, int T, int n) {
  if (p->smooth_rounds > 0 && smooth_smem_bytes(T, n) > kMaxSmemBytes)
    return fail(CPP_ERR_INVALID_ARG, "smooth_rounds > 0 needs (n + 1) * T * 8 <= 227 KB (T = %d)", T);
  return CPP_OK;
}

cpp_status check_lattice(int T, int K, int Kp, int n) {
  if (T < 1) return fail(CPP_ERR_INVALID_ARG, "T = %d < 1", T);
  if (K < 1 || K > 65535) return fail(CPP_ERR_INVALID_ARG, "K = %d outside [1, 65535]", K);
  if (Kp < K || Kp % 4 != 0)
    return fail(CPP_ERR_INVALID_ARG, "Kp = %d must be >= K = %d and a multiple of 4", Kp, K);
  if (n < 1 || n > CPP_MAX_JOINTS) return fail(CPP_ERR_INVALID_ARG, "n = %d outside [1, 16]", n);
  return CPP_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

Req empty_req() {
  Req r;
  memset(&r, 0, sizeof(r));
  return r;
}

}  // namespace

namespace cppflow {
void set_last_error(const char* msg) { g_err = msg; }

size_t geo_bytes() { return sizeof(GeoF); }

bool make_geo(const cpp_geometry_t& g, int n, void* out, char* err) {
  auto bad = [&](const char* m) {
    snprintf(err, 160, "collision model: %s", m);
    return false;
  };
  if (g.n_caps < 0 || g.n_caps > kMaxCaps || g.n_pairs < 0 || g.n_pairs > kMaxPairs ||
      g.n_boxes < 0 || g.n_boxes > kMaxBoxes)
    return bad("counts outside [0, CPP_MAX_CAPSULES / PAIRS / BOXES]");
  GeoF f;
  memset(&f, 0, sizeof(f));
  f.n_caps = g.n_caps; f.n_pairs = g.n_pairs; f.n_boxes = g.n_boxes;
  int order[kMaxCaps], pos[kMaxCaps], m = 0;
  for (int fr = 0; fr <= n; ++fr) {  // sort capsules by frame, stable
    f.frame_begin[fr] = m;
    for (int c = 0; c < g.n_caps; ++c)
      if (g.caps[c].frame == fr) { pos[c] = m; order[m++] = c; }
  }
  for (int fr = n + 1; fr < kMaxJ + 2; ++fr) f.frame_begin[fr] = m;
  if (m != g.n_caps) return bad("a capsule frame is outside [0, n]");
  for (int k = 0; k < m; ++k) {
    const cpp_capsule_t& c = g.caps[order[k]];
    for (int q = 0; q < 3; ++q) {
      if (!finite_d(c.a[q]) || !finite_d(c.b[q])) return bad("non-finite capsule end point");
      f.a[k][q] = (float)c.a[q];
      f.b[k][q] = (float)c.b[q];
    }
    if (!(finite_d(c.radius) && c.radius >= 0)) return bad("capsule radius must be finite and >= 0");
    f.r[k] = (float)c.radius;
    // bounding sphere about the midpoint, widened by 1e-5 m so FP32 rounding of the
    // separation test can only keep extra pairs, never drop a touching one
    const double dx = c.b[0] - c.a[0], dy = c.b[1] - c.a[1], dz = c.b[2] - c.a[2];
    f.bound[k] = (float)(0.5 * std::sqrt(dx * dx + dy * dy + dz * dz) + c.radius + 1e-5);
  }
  for (int k = 0; k < g.n_pairs; ++k) {
    const int u = g.pairs[k][0], v = g.pairs[k][1];
    if (u < 0 || u >= g.n_caps || v < 0 || v >= g.n_caps || u == v)
      return bad("pair index out of range or a capsule paired with itself");
    f.pu[k] = (int8_t)pos[u];
    f.pv[k] = (int8_t)pos[v];
  }
  for (int o = 0; o < g.n_boxes; ++o) {
    const cpp_cuboid_t& b = g.boxes[o];
    for (int q = 0; q < 9; ++q)
      if (!finite_d(b.R[q])) return bad("non-finite box rotation");
    for (int q = 0; q < 3; ++q) {
      if (!finite_d(b.p[q])) return bad("non-finite box centre");
      if (!(finite_d(b.half[q]) && b.half[q] >= 0)) return bad("box half extents must be >= 0");
      f.p[o][q] = (float)b.p[q];
      f.h[o][q] = (float)b.half[q];
    }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) f.Rt[o][3 * r + c] = (float)b.R[3 * c + r];  // transpose
    f.box_bound[o] = (float)(std::sqrt(b.half[0] * b.half[0] + b.half[1] * b.half[1] +
                                       b.half[2] * b.half[2]) + 1e-5);
  }
  memcpy(out, &f, sizeof(f));
  return true;
}
}  // namespace cppflow

namespace cppflow {
// One thread initialises an mbarrier that expects one arrival, never arrives,
// and waits for its first phase with the library's bounded wait; when the limit
// runs out it records CPP_ERR_TIMEOUT.
__global__ void wait_selftest_kernel(uint64_t limit_ns, bool cluster_scope, int32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const bool done = cluster_scope ? mbar_wait_bounded_cluster(&bar, 0, limit_ns)
                                  : mbar_wait_bounded(&bar, 0, limit_ns);
  if (!done) raise_status(status, CPP_ERR_TIMEOUT);
}
}  // namespace cppflow

extern "C" {

const char* cpp_last_error(void) { return g_err.c_str(); }

const char* cpp_status_string(int s) {
  switch (s) {
    case CPP_OK: return "ok";
    case CPP_PENDING: return "pending";
    case CPP_ERR_INVALID_ARG: return "invalid argument";
    case CPP_ERR_INFEASIBLE: return "infeasible";
    case CPP_ERR_OOM: return "out of memory";
    case CPP_ERR_BUDGET: return "over HBM budget";
    case CPP_ERR_TIMEOUT: return "timeout";
    case CPP_ERR_CUDA: return "CUDA error";
    case CPP_ERR_NOT_FOUND: return "not found";
    case CPP_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

int32_t cpp_version(void) { return 100; }

void cpp_params_default(cpp_params_t* p) {
  if (!p) return;
  const double deg = 3.14159265358979323846 / 180.0;
  p->tau_pos = 1e-3;
  p->tau_rot = 0.1 * deg;
  p->near_margin = 1.5 * deg;
  p->pen_limit = 10.0;
  p->pen_pose = 100.0;
  p->jump_max = 7.0 * deg;
  p->lambda0 = 1e-3;
  p->lambda_up = 10.0;
  p->lambda_down = 10.0;
  p->lambda_min = 1e-12;
  p->lambda_max = 1e12;
  p->freeze_step = 1e-10;
  p->freeze_cost = 1e-13;
  p->lm_iters = 20;
  p->free_mask = 0xFFFFFFFFu;
  p->lm_fp64 = 0;
  p->dp_objective = CPP_DP_SUM;
  p->smooth_rounds = 0;
  p->reserved_ = 0;
  p->smooth_lambda = 1.0;
  p->pen_collide = 100.0;
  p->coll_margin = 0.02;
  p->coll_weight = 1.0;
}

cpp_status cpp_fk_batch(const cpp_robot_t* robot, const float* q, int64_t N, float* R, float* p,
                        cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (N < 0) return fail(CPP_ERR_INVALID_ARG, "N < 0");
  if (N > 0 && (!q || !R || !p)) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  return cuda_status(launch_fk_batch(*robot, q, N, R, p, (cudaStream_t)stream), "cpp_fk_batch");
}

cpp_status cpp_fk_pose_f64(const cpp_robot_t* robot, const double* q, int64_t N, double* pose,
                           cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (N < 0) return fail(CPP_ERR_INVALID_ARG, "N < 0");
  if (N > 0 && (!q || !pose)) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  return cuda_status(launch_fk_pose64(*robot, q, N, pose, (cudaStream_t)stream), "cpp_fk_pose_f64");
}

// A collision model into a single request's source (by value), validated.
static cpp_status set_geo(SingleSrc& s, const cpp_geometry_t* geometry, int n) {
  s.has_geo = 0;
  if (!geometry) return CPP_OK;
  char msg[160];
  if (!make_geo(*geometry, n, &s.geo, msg)) return fail(CPP_ERR_INVALID_ARG, "%s", msg);
  s.has_geo = 1;
  return CPP_OK;
}

static cpp_status mask_impl(const cpp_robot_t* robot, const cpp_params_t* params,
                            const cpp_geometry_t* geometry, const float* cand,
                            const double* targets, int32_t T, int32_t K, int32_t Kp,
                            int32_t k_begin, uint8_t* mask, float* pen, float* err, float* clear,
                            int32_t* dev_status, cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  if (cpp_status s = check_lattice(T, K, Kp, robot->n)) return s;
  if (k_begin < 0 || k_begin > K || k_begin % 4 != 0)
    return fail(CPP_ERR_INVALID_ARG, "k_begin = %d must be a multiple of 4 in [0, K]", k_begin);
  if (!cand || !targets || !mask || !pen) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(cand, 16) || !aligned(pen, 16) || !aligned(mask, 4) || (err && !aligned(err, 16)) ||
      (clear && !aligned(clear, 16)))
    return fail(CPP_ERR_INVALID_ARG, "cand/pen/err/clearance must be 16-byte and mask 4-byte aligned");
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.K = K; s.r.Kp = Kp; s.r.n = robot->n; s.r.k_begin = k_begin;
  s.r.cand = cand; s.r.targets = targets; s.r.mask = mask; s.r.pen = pen; s.r.err = err;
  s.r.clear = clear;
  s.r.status = dev_status;
  s.robot = *robot;
  if (cpp_status e = set_geo(s, geometry, robot->n)) return e;
  return cuda_status(launch_mask(s, *params, (cudaStream_t)stream), "cpp_mask");
}

cpp_status cpp_mask(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                    const double* targets, int32_t T, int32_t K, int32_t Kp, uint8_t* mask,
                    float* pen, float* err, int32_t* dev_status, cpp_stream_t stream) {
  return mask_impl(robot, params, nullptr, cand, targets, T, K, Kp, 0, mask, pen, err, nullptr,
                   dev_status, stream);
}

cpp_status cpp_mask_geo(const cpp_robot_t* robot, const cpp_params_t* params,
                        const cpp_geometry_t* geometry, const float* cand,
                        const double* targets, int32_t T, int32_t K, int32_t Kp, uint8_t* mask,
                        float* pen, float* err, float* clearance, int32_t* dev_status,
                        cpp_stream_t stream) {
  return mask_impl(robot, params, geometry, cand, targets, T, K, Kp, 0, mask, pen, err, clearance,
                   dev_status, stream);
}

cpp_status cpp_mask_range(const cpp_robot_t* robot, const cpp_params_t* params,
                          const float* cand, const double* targets, int32_t T, int32_t K,
                          int32_t Kp, int32_t k_begin, uint8_t* mask, float* pen, float* err,
                          int32_t* dev_status, cpp_stream_t stream) {
  return mask_impl(robot, params, nullptr, cand, targets, T, K, Kp, k_begin, mask, pen, err,
                   nullptr, dev_status, stream);
}

size_t cpp_dp_workspace_size(int32_t T, int32_t Kp) {
  if (T < 1 || Kp < 1) return 0;
  return dp_layout(T, Kp).total;
}

cpp_status cpp_dp_search_ex(const float* cand, const float* pen, int32_t T, int32_t K, int32_t Kp,
                            int32_t n, int32_t objective, void* workspace, size_t ws_bytes,
                            int32_t* sel, float* best_cost, float* q_seed, float* search_mjac,
                            int32_t* dev_status, cpp_stream_t stream) {
  if (cpp_status s = check_lattice(T, K, Kp, n)) return s;
  if (objective != CPP_DP_SUM && objective != CPP_DP_MINMAX)
    return fail(CPP_ERR_INVALID_ARG, "objective %d is neither CPP_DP_SUM nor CPP_DP_MINMAX",
                objective);
  if (!dp_supported(n, Kp))
    return fail(CPP_ERR_INVALID_ARG, "Kp * (n + 1) = %d exceeds the shared-memory limit (29056)",
                Kp * (n + 1));
  if (!cand || !pen || !sel || !best_cost || !workspace)
    return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(cand, 16) || !aligned(pen, 16))
    return fail(CPP_ERR_INVALID_ARG, "cand and pen must be 16-byte aligned");
  const DpLayout L = dp_layout(T, Kp);
  if (ws_bytes < L.total || !aligned(workspace, 256))
    return fail(CPP_ERR_INVALID_ARG, "workspace needs %zu bytes, 256-byte aligned", L.total);
  char* ws = static_cast<char*>(workspace);
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.K = K; s.r.Kp = Kp; s.r.n = n; s.r.Kb = bp_stride(Kp);
  s.r.cand = cand; s.r.pen = const_cast<float*>(pen);
  s.r.pen_min = reinterpret_cast<float*>(ws + L.pen_min);
  s.r.bp = reinterpret_cast<uint16_t*>(ws + L.bp);
  s.r.costT = reinterpret_cast<float*>(ws + L.costT);
  s.r.sel = sel; s.r.best_cost = best_cost; s.r.q_seed = q_seed; s.r.search_mjac = search_mjac;
  s.r.status = dev_status;
  memset(&s.robot, 0, sizeof(s.robot));
  return cuda_status(launch_dp(s, CPP_STAGE_LAYER_MIN | CPP_STAGE_DP_FORWARD | CPP_STAGE_BACKTRACK,
                               objective, (cudaStream_t)stream), "cpp_dp_search");
}

cpp_status cpp_dp_search(const float* cand, const float* pen, int32_t T, int32_t K, int32_t Kp,
                         int32_t n, void* workspace, size_t ws_bytes, int32_t* sel,
                         float* best_cost, float* q_seed, int32_t* dev_status,
                         cpp_stream_t stream) {
  return cpp_dp_search_ex(cand, pen, T, K, Kp, n, CPP_DP_SUM, workspace, ws_bytes, sel,
                          best_cost, q_seed, nullptr, dev_status, stream);
}

cpp_status cpp_lm_refine(const cpp_robot_t* robot, const cpp_params_t* params, const float* q_in,
                         const double* targets, int32_t T, float* q_out, double* pose_err,
                         int32_t* dev_status, cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  if (T < 1) return fail(CPP_ERR_INVALID_ARG, "T < 1");
  if (!q_in || !targets || !q_out) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  if (cpp_status e = check_smooth(params, T, robot->n)) return e;
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.n = robot->n;
  s.r.q_in = q_in; s.r.q_out = q_out; s.r.targets = targets; s.r.pose_err = pose_err;
  s.r.status = dev_status;
  s.robot = *robot;
  return cuda_status(launch_lm(s, *params, true, (cudaStream_t)stream), "cpp_lm_refine");
}

cpp_status cpp_smooth_step(const cpp_robot_t* robot, const cpp_params_t* params, float* q,
                           const double* targets, int32_t T, int32_t* dev_status,
                           cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  if (T < 1) return fail(CPP_ERR_INVALID_ARG, "T < 1");
  if (!q || !targets) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  if (smooth_smem_bytes(T, robot->n) > kMaxSmemBytes)
    return fail(CPP_ERR_INVALID_ARG, "(n + 1) * T * 8 exceeds 227 KB (T = %d)", T);
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.n = robot->n;
  s.r.q_out = q; s.r.targets = targets;
  s.r.status = dev_status;
  s.robot = *robot;
  return cuda_status(launch_smooth(s, *params, (cudaStream_t)stream), "cpp_smooth_step");
}

size_t cpp_smooth_workspace_size(int32_t T, int32_t n) {
  if (T < 1 || n < 1 || n > CPP_MAX_JOINTS) return 0;
  return smooth_ws_bytes(T, n);
}

cpp_status cpp_smooth_step_geo(const cpp_robot_t* robot, const cpp_params_t* params,
                               const cpp_geometry_t* geometry, float* q, const double* targets,
                               int32_t T, void* workspace, size_t ws_bytes, int32_t* dev_status,
                               cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  if (T < 1) return fail(CPP_ERR_INVALID_ARG, "T < 1");
  if (!q || !targets) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  if (smooth_smem_bytes(T, robot->n) > kMaxSmemBytes)
    return fail(CPP_ERR_INVALID_ARG, "(n + 1) * T * 8 exceeds 227 KB (T = %d)", T);
  if (geometry && (!workspace || ws_bytes < smooth_ws_bytes(T, robot->n) || !aligned(workspace, 256)))
    return fail(CPP_ERR_INVALID_ARG, "workspace needs %zu bytes, 256-byte aligned",
                smooth_ws_bytes(T, robot->n));
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.n = robot->n;
  s.r.q_out = q; s.r.targets = targets;
  s.r.smooth_ws = static_cast<double*>(workspace);
  s.r.status = dev_status;
  s.robot = *robot;
  if (cpp_status e = set_geo(s, geometry, robot->n)) return e;
  return cuda_status(launch_smooth(s, *params, (cudaStream_t)stream), "cpp_smooth_step_geo");
}

cpp_status cpp_wait_selftest(int64_t limit_ns, int32_t cluster_scope, int32_t* dev_status,
                             cpp_stream_t stream) {
  if (limit_ns < 1000 || limit_ns > 10000000000LL)
    return fail(CPP_ERR_INVALID_ARG, "limit_ns must be in [1e3, 1e10]");
  if (!dev_status) return fail(CPP_ERR_INVALID_ARG, "dev_status is NULL");
  wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)limit_ns, cluster_scope != 0,
                                                           dev_status);
  return cuda_status(cudaGetLastError(), "cpp_wait_selftest");
}

cpp_status cpp_check(const cpp_robot_t* robot, const cpp_params_t* params, const float* q,
                     const double* targets, int32_t T, double* pose_err, cpp_report_t* report,
                     cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  if (T < 1) return fail(CPP_ERR_INVALID_ARG, "T < 1");
  if (!q || !targets) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.n = robot->n;
  s.r.q_out = const_cast<float*>(q); s.r.targets = targets; s.r.pose_err = pose_err;
  s.r.report = report;
  s.robot = *robot;
  return cuda_status(launch_check(s, *params, (cudaStream_t)stream), "cpp_check");
}

size_t cpp_plan_workspace_size(int32_t T, int32_t K, int32_t Kp, int32_t n) {
  if (T < 1 || K < 1 || Kp < K || n < 1) return 0;
  return plan_layout(T, Kp, n).total;
}

cpp_status cpp_plan(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                    const double* targets, int32_t T, int32_t K, int32_t Kp, void* workspace,
                    size_t ws_bytes, int32_t* sel, float* best_cost, float* q_out,
                    double* pose_err, cpp_report_t* report, int32_t* dev_status,
                    cpp_stream_t stream) {
  return cpp_plan_geo(robot, params, nullptr, cand, targets, T, K, Kp, workspace, ws_bytes, sel,
                      best_cost, q_out, pose_err, report, dev_status, stream);
}

cpp_status cpp_plan_geo(const cpp_robot_t* robot, const cpp_params_t* params,
                        const cpp_geometry_t* geometry, const float* cand,
                        const double* targets, int32_t T, int32_t K, int32_t Kp, void* workspace,
                        size_t ws_bytes, int32_t* sel, float* best_cost, float* q_out,
                        double* pose_err, cpp_report_t* report, int32_t* dev_status,
                        cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  const int n = robot->n;
  if (cpp_status s = check_lattice(T, K, Kp, n)) return s;
  if (cpp_status s = check_smooth(params, T, n)) return s;
  if (!dp_supported(n, Kp))
    return fail(CPP_ERR_INVALID_ARG, "Kp * (n + 1) exceeds the shared-memory limit");
  if (!cand || !targets || !sel || !best_cost || !q_out || !workspace)
    return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(cand, 16)) return fail(CPP_ERR_INVALID_ARG, "cand must be 16-byte aligned");
  const PlanLayout L = plan_layout(T, Kp, n);
  if (ws_bytes < L.total || !aligned(workspace, 256))
    return fail(CPP_ERR_INVALID_ARG, "workspace needs %zu bytes, 256-byte aligned", L.total);
  char* ws = static_cast<char*>(workspace);
  cudaStream_t st = (cudaStream_t)stream;
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.K = K; s.r.Kp = Kp; s.r.n = n; s.r.Kb = bp_stride(Kp);
  s.r.cand = cand; s.r.targets = targets;
  s.r.mask = reinterpret_cast<uint8_t*>(ws + L.mask);
  s.r.pen = reinterpret_cast<float*>(ws + L.pen);
  s.r.pen_min = reinterpret_cast<float*>(ws + L.dp_base + L.dp.pen_min);
  s.r.bp = reinterpret_cast<uint16_t*>(ws + L.dp_base + L.dp.bp);
  s.r.costT = reinterpret_cast<float*>(ws + L.dp_base + L.dp.costT);
  s.r.sel = sel; s.r.best_cost = best_cost;
  s.r.q_seed = reinterpret_cast<float*>(ws + L.q_seed);
  s.r.q_in = s.r.q_seed; s.r.q_out = q_out; s.r.pose_err = pose_err; s.r.report = report;
  s.r.smooth_ws = reinterpret_cast<double*>(ws + L.smooth);
  s.r.status = dev_status;
  s.robot = *robot;
  if (cpp_status e = set_geo(s, geometry, n)) return e;
  if (cpp_status e = cuda_status(launch_mask(s, *params, st), "cpp_plan/mask")) return e;
  if (cpp_status e = cuda_status(launch_dp(s, CPP_STAGE_LAYER_MIN | CPP_STAGE_DP_FORWARD |
                                                   CPP_STAGE_BACKTRACK, params->dp_objective, st),
                                 "cpp_plan/dp"))
    return e;
  // the check below writes the FP64 pose errors
  if (cpp_status e = cuda_status(launch_lm(s, *params, false, st), "cpp_plan/lm")) return e;
  return cuda_status(launch_check(s, *params, st), "cpp_plan/check");
}

// ------------------------------------------------------------------ plain path from host memory
namespace {
struct HostPlanLayout {  // device copies of inputs and outputs, status word, plan scratch
  size_t cand, tgt, sel, q, err, rep, best, status, plan, total;
};
HostPlanLayout host_plan_layout(int T, int Kp, int n) {
  HostPlanLayout L;
  size_t o = 0;
  L.cand = o;   o += align256((size_t)T * n * Kp * sizeof(float));
  L.tgt = o;    o += align256((size_t)T * 7 * sizeof(double));
  L.sel = o;    o += align256((size_t)T * sizeof(int32_t));
  L.q = o;      o += align256((size_t)T * n * sizeof(float));
  L.err = o;    o += align256((size_t)T * 2 * sizeof(double));
  L.rep = o;    o += align256(sizeof(cpp_report_t));
  L.best = o;   o += align256(sizeof(float));
  L.status = o; o += align256(sizeof(int32_t));
  L.plan = o;   o += plan_layout(T, Kp, n).total;
  L.total = o;
  return L;
}
}  // namespace

size_t cpp_plan_host_workspace_size(int32_t T, int32_t K, int32_t Kp, int32_t n) {
  if (T < 1 || K < 1 || Kp < K || n < 1) return 0;
  return host_plan_layout(T, Kp, n).total;
}

cpp_status cpp_plan_host(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                         const double* targets, int32_t T, int32_t K, int32_t Kp,
                         void* workspace, size_t ws_bytes, int32_t* sel, float* best_cost,
                         float* q_out, double* pose_err, cpp_report_t* report,
                         cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  const int n = robot->n;
  if (cpp_status s = check_lattice(T, K, Kp, n)) return s;
  if (cpp_status s = check_smooth(params, T, n)) return s;
  if (!dp_supported(n, Kp))
    return fail(CPP_ERR_INVALID_ARG, "Kp * (n + 1) exceeds the shared-memory limit");
  if (!cand || !targets || !workspace) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  const HostPlanLayout L = host_plan_layout(T, Kp, n);
  if (ws_bytes < L.total || !aligned(workspace, 256))
    return fail(CPP_ERR_INVALID_ARG, "workspace needs %zu bytes, 256-byte aligned", L.total);
  char* ws = static_cast<char*>(workspace);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cand_b = (size_t)T * n * Kp * sizeof(float), tgt_b = (size_t)T * 7 * sizeof(double);
  int32_t* d_status = reinterpret_cast<int32_t*>(ws + L.status);
  if (cpp_status e = cuda_status(cudaMemcpyAsync(ws + L.cand, cand, cand_b, cudaMemcpyHostToDevice, st),
                                 "cpp_plan_host/H2D"))
    return e;
  if (cpp_status e = cuda_status(cudaMemcpyAsync(ws + L.tgt, targets, tgt_b, cudaMemcpyHostToDevice, st),
                                 "cpp_plan_host/H2D"))
    return e;
  if (cpp_status e = cuda_status(cudaMemsetAsync(d_status, 0, sizeof(int32_t), st), "cpp_plan_host"))
    return e;
  const cpp_status ps = cpp_plan(robot, params, reinterpret_cast<const float*>(ws + L.cand),
                                 reinterpret_cast<const double*>(ws + L.tgt), T, K, Kp, ws + L.plan,
                                 ws_bytes - L.plan, reinterpret_cast<int32_t*>(ws + L.sel),
                                 reinterpret_cast<float*>(ws + L.best),
                                 reinterpret_cast<float*>(ws + L.q),
                                 reinterpret_cast<double*>(ws + L.err),
                                 reinterpret_cast<cpp_report_t*>(ws + L.rep), d_status, stream);
  if (ps != CPP_OK) {
    cudaStreamSynchronize(st);  // the input copies read host memory the caller may free
    return ps;
  }
  struct Back { void* dst; size_t off, bytes; } back[] = {
      {sel, L.sel, (size_t)T * sizeof(int32_t)},
      {best_cost, L.best, sizeof(float)},
      {q_out, L.q, (size_t)T * n * sizeof(float)},
      {pose_err, L.err, (size_t)T * 2 * sizeof(double)},
      {report, L.rep, sizeof(cpp_report_t)}};
  for (const Back& b : back) {
    if (!b.dst) continue;
    if (cpp_status e = cuda_status(cudaMemcpyAsync(b.dst, ws + b.off, b.bytes, cudaMemcpyDeviceToHost, st),
                                   "cpp_plan_host/D2H"))
      return e;
  }
  int32_t h_status = 0;
  if (cpp_status e = cuda_status(cudaMemcpyAsync(&h_status, d_status, sizeof(int32_t),
                                                 cudaMemcpyDeviceToHost, st),
                                 "cpp_plan_host/D2H"))
    return e;
  if (cpp_status e = cuda_status(cudaStreamSynchronize(st), "cpp_plan_host/wait")) return e;
  if (h_status != 0)
    return fail((cpp_status)h_status, "cpp_plan_host: device status %d", h_status);
  return CPP_OK;
}

// ------------------------------------------------------------------ cpf-BatchOpt
size_t cpp_batch_opt_workspace_size(int32_t T, int32_t K, int32_t n, int32_t lanes) {
  if (T < 1 || K < 1 || n < 1 || lanes < 1) return 0;
  return batch_opt_layout(T, K, n, lanes).total;
}

cpp_status cpp_batch_opt(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                         const double* targets, int32_t T, int32_t K, int32_t Kp, int32_t lanes,
                         void* workspace, size_t ws_bytes, int32_t* lane_sel, float* lane_mjac,
                         float* q_out, double* pose_err, cpp_report_t* reports, int32_t* best,
                         int32_t* dev_status, cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  const int n = robot->n;
  if (cpp_status s = check_lattice(T, K, Kp, n)) return s;
  if (cpp_status s = check_smooth(params, T, n)) return s;
  if (lanes < 1 || lanes > K) return fail(CPP_ERR_INVALID_ARG, "lanes = %d outside [1, K]", lanes);
  if (!cand || !targets || !lane_sel || !lane_mjac || !q_out || !reports || !best || !workspace)
    return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  const BatchOptLayout L = batch_opt_layout(T, K, n, lanes);
  if (ws_bytes < L.total || !aligned(workspace, 256))
    return fail(CPP_ERR_INVALID_ARG, "workspace needs %zu bytes, 256-byte aligned", L.total);
  return cuda_status(launch_batch_opt(*robot, *params, cand, targets, T, K, Kp, lanes,
                                      static_cast<char*>(workspace), lane_sel, lane_mjac, q_out,
                                      pose_err, reports, best, dev_status, (cudaStream_t)stream),
                     "cpp_batch_opt");
}

// ------------------------------------------------------------------ many requests
namespace {
struct BatchLayout {
  size_t reqs, sched, robots, lm, per_req_base, total;
  LmAuxLayout lm_layout;
  std::vector<PlanLayout> L;
  std::vector<size_t> off;
};
BatchLayout batch_layout(const cpp_plan_desc_t* d, int count, int n_robots, const cpp_robot_t* robots) {
  BatchLayout B;
  size_t o = 0;
  B.reqs = o;   o += align256(sizeof(Req) * (size_t)count);
  B.sched = o;  o += align256(sizeof(Req) * (size_t)count);
  B.robots = o; o += align256(sizeof(cpp_robot_t) * (size_t)n_robots);
  B.lm_layout = lm_aux_layout(n_robots, count);
  B.lm = o;     o += B.lm_layout.total;
  B.per_req_base = o;
  for (int r = 0; r < count; ++r) {
    const int n = robots[d[r].robot].n;
    B.L.push_back(plan_layout(d[r].T, d[r].Kp, n));
    B.off.push_back(o);
    o += B.L.back().total;
  }
  B.total = o;
  return B;
}
}  // namespace

size_t cpp_plan_batch_workspace_size(const cpp_plan_desc_t* descs, int32_t count,
                                     const cpp_robot_t* robots, int32_t n_robots) {
  if (!descs || count < 1 || !robots || n_robots < 1) return 0;
  for (int r = 0; r < count; ++r)
    if (descs[r].robot < 0 || descs[r].robot >= n_robots) return 0;
  return batch_layout(descs, count, n_robots, robots).total;
}

}  // extern "C"

// ------------------------------------------------------------------ batch schedule
// The search stage of an uneven batch is scheduled, not launched over the whole
// table at once: a request is serial in T, so one long request on one CTA sets
// the batch's time however many SMs sit idle. Requests whose lattice (edges
// (T - 1) Kp^2) exceeds alpha times the mean load of a CTA slot (total edges /
// 2 SMs) are "heavy" and run as thread-block clusters (grouped by cluster size,
// one launch per group, each on its own stream); the rest run one CTA per
// request in a second table sorted longest first, so the hardware block
// scheduler hands out the longest requests first. The launches fork from and
// join back into the caller's stream through events, so a capture of the stream
// records the whole fork/join. alpha comes from cpp_batch_tune (timed on the
// batch itself, or read from a persisted table); the default is kDefaultAlpha.
namespace {
constexpr int kMaxGroups = 8;
constexpr double kDefaultAlpha = 2.0;

struct SchedGroup {
  int begin, count, max_Kp, form, cpc;
};

bool fast_n(int n) { return n == 6 || n == 7 || n == 9; }
}  // namespace

struct cpp_batch {
  BatchSrc src;  // request table in descriptor order
  cpp_params_t params;
  int n, count, max_T, max_Kp;
  long long max_tasks;
  // schedule of the search stage
  Req* d_sched;
  const cpp_robot_t* d_robots;
  std::vector<Req> reqs;            // descriptor order (host copy)
  std::vector<long long> edges;     // (T - 1) Kp^2 per request
  std::vector<SchedGroup> groups;   // cluster groups, then the one-CTA group (last)
  bool any_geo;  // some request has a collision model
  double alpha;
  int cpc;  // successor candidates per CTA of the cluster form (0: default)
  double budget_ms;  // > 0: per-request forms within this search time (alpha, cpc unused)
  int mask_tpw;  // 128-candidate tasks per warp of the mask stage (0: default)
  int min_kp;    // smallest Kp that may run as a cluster (0: any)
  int heavy;
  cudaStream_t aux[kMaxGroups];
  cudaEvent_t fork, join[kMaxGroups];
  cudaGraphExec_t graph;
  uint32_t graph_stages;
};

namespace {

void drop_graph(cpp_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_stages = 0;
}

// The schedule from a per-request choice: cpc_of[r] < 0 runs request r on one
// CTA, 0 as a cluster of the default tile, > 0 as a cluster of that many
// successors per CTA. Cluster requests are grouped by that choice and cluster
// size (one launch per group, each on its own stream), the rest form the
// one-CTA group in a table sorted longest first. Uploads the schedule table.
cpp_status build_schedule(cpp_batch* b, const std::vector<int>& cpc_of, cudaStream_t st) {
  const int count = b->count;
  std::vector<int> heavy, light;
  for (int r = 0; r < count; ++r) (cpc_of[r] >= 0 ? heavy : light).push_back(r);
  auto longer = [&](int x, int y) {
    return b->edges[x] != b->edges[y] ? b->edges[x] > b->edges[y] : x < y;
  };
  auto cs_of = [&](int r) { return cluster_size(b->reqs[r].Kp, cpc_of[r]); };
  std::sort(heavy.begin(), heavy.end(), [&](int x, int y) {
    if (cpc_of[x] != cpc_of[y]) return cpc_of[x] > cpc_of[y];
    const int cx = cs_of(x), cy = cs_of(y);
    return cx != cy ? cx > cy : longer(x, y);
  });
  std::sort(light.begin(), light.end(), longer);
  std::vector<SchedGroup> groups;
  std::vector<Req> table;
  table.reserve(count);
  for (size_t i = 0; i < heavy.size();) {
    const int cpc = cpc_of[heavy[i]], cs = cs_of(heavy[i]);
    SchedGroup g{(int)table.size(), 0, 0, kFormCluster, cpc};
    for (; i < heavy.size() && cpc_of[heavy[i]] == cpc && cs_of(heavy[i]) == cs; ++i) {
      table.push_back(b->reqs[heavy[i]]);
      g.max_Kp = std::max(g.max_Kp, b->reqs[heavy[i]].Kp);
      ++g.count;
    }
    groups.push_back(g);
  }
  if ((int)groups.size() > kMaxGroups) return fail(CPP_ERR_INVALID_ARG, "too many cluster groups");
  SchedGroup lg{(int)table.size(), (int)light.size(), 0, groups.empty() ? kFormAuto : kFormCta, 0};
  for (int r : light) {
    table.push_back(b->reqs[r]);
    lg.max_Kp = std::max(lg.max_Kp, b->reqs[r].Kp);
  }
  groups.push_back(lg);
  for (size_t g = 0; g + 1 < groups.size(); ++g) {
    if (!b->aux[g])
      if (cpp_status e = cuda_status(cudaStreamCreateWithFlags(&b->aux[g], cudaStreamNonBlocking),
                                     "batch schedule"))
        return e;
    if (!b->join[g])
      if (cpp_status e = cuda_status(cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming),
                                     "batch schedule"))
        return e;
  }
  if (!b->fork)
    if (cpp_status e = cuda_status(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming),
                                   "batch schedule"))
      return e;
  // pageable source: staged before cudaMemcpyAsync returns
  if (cpp_status e = cuda_status(cudaMemcpyAsync(b->d_sched, table.data(), sizeof(Req) * count,
                                                 cudaMemcpyHostToDevice, st), "batch schedule"))
    return e;
  b->groups = groups;
  b->heavy = (int)heavy.size();
  drop_graph(b);
  return CPP_OK;
}

// Split the requests for alpha (<= 0: none heavy) and cluster tiles of cpc
// successors per CTA: requests whose lattice (edges (T - 1) Kp^2) is at least
// alpha times the mean load of a CTA slot run as clusters.
cpp_status set_schedule(cpp_batch* b, double alpha, int cpc, cudaStream_t st) {
  long long total = 0;
  for (long long e : b->edges) total += e;
  const double slots = 2.0 * device_sm_count();
  const double thr = alpha > 0 ? alpha * (double)total / slots : HUGE_VAL;
  std::vector<int> cpc_of(b->count, -1);
  for (int r = 0; r < b->count; ++r) {
    const bool h =
        fast_n(b->n) && cluster_size(b->reqs[r].Kp, cpc) > 0 && (double)b->edges[r] >= thr &&
        b->reqs[r].Kp >= b->min_kp;
    if (h) cpc_of[r] = cpc;
  }
  if (cpp_status e = build_schedule(b, cpc_of, st)) return e;
  b->alpha = alpha;
  b->cpc = cpc;
  b->budget_ms = 0.0;
  return CPP_OK;
}

// Each request in the search form with the highest edge rate per SM whose
// estimated time is within budget_ms (the server's policy, pick_search_form).
std::vector<int> budget_forms(const cpp_batch* b, double budget_ms) {
  std::vector<int> cpc_of(b->count, -1);
  if (!fast_n(b->n)) return cpc_of;
  for (int r = 0; r < b->count; ++r) {
    const SearchForm f = pick_search_form(b->reqs[r].T, b->reqs[r].Kp, budget_ms);
    if (f.form == kFormCluster) cpc_of[r] = f.cpc;
  }
  return cpc_of;
}
int schedule_groups(const cpp_batch* b, const std::vector<int>& cpc_of) {
  std::vector<std::pair<int, int>> keys;
  for (int r = 0; r < b->count; ++r)
    if (cpc_of[r] >= 0) keys.emplace_back(cpc_of[r], cluster_size(b->reqs[r].Kp, cpc_of[r]));
  std::sort(keys.begin(), keys.end());
  return (int)(std::unique(keys.begin(), keys.end()) - keys.begin());
}
cpp_status set_budget(cpp_batch* b, double budget_ms, cudaStream_t st) {
  if (cpp_status e = build_schedule(b, budget_forms(b, budget_ms), st)) return e;
  b->budget_ms = budget_ms;
  return CPP_OK;
}

// The search's forward sweep under the current schedule.
cudaError_t run_forward(cpp_batch* b, cudaStream_t st) {
  const int objective = b->params.dp_objective;
  const int ng = (int)b->groups.size();
  auto launch = [&](const SchedGroup& g, cudaStream_t s) {
    const BatchSrc src{b->d_sched + g.begin, b->d_robots};
    return launch_forward(src, objective, b->n, g.count, g.max_Kp, g.form, g.cpc, s);
  };
  if (ng == 1) return launch(b->groups[0], st);
  cudaError_t e = cudaEventRecord(b->fork, st);
  for (int g = 0; g + 1 < ng && e == cudaSuccess; ++g) {
    if ((e = cudaStreamWaitEvent(b->aux[g], b->fork, 0)) != cudaSuccess) break;
    if ((e = launch(b->groups[g], b->aux[g])) != cudaSuccess) break;
    e = cudaEventRecord(b->join[g], b->aux[g]);
  }
  if (e == cudaSuccess && b->groups[ng - 1].count > 0) e = launch(b->groups[ng - 1], st);
  for (int g = 0; g + 1 < ng && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(st, b->join[g], 0);
  return e;
}

cpp_status run_stages(cpp_batch* b, uint32_t stages, cudaStream_t st) {
  if (stages & CPP_STAGE_MASK)
    if (cpp_status e = cuda_status(launch_mask_batch(b->src, b->n, b->count, b->max_tasks,
                                                     b->params, b->any_geo, st, b->mask_tpw),
                                   "batch/mask"))
      return e;
  if (stages & CPP_STAGE_LAYER_MIN)
    if (cpp_status e = cuda_status(launch_dp_batch(b->src, CPP_STAGE_LAYER_MIN, b->params.dp_objective,
                                                   b->n, b->count, b->max_T, b->max_Kp, st),
                                   "batch/layer_min"))
      return e;
  if (stages & CPP_STAGE_DP_FORWARD)
    if (cpp_status e = cuda_status(run_forward(b, st), "batch/forward")) return e;
  if (stages & CPP_STAGE_BACKTRACK)
    if (cpp_status e = cuda_status(launch_dp_batch(b->src, CPP_STAGE_BACKTRACK, b->params.dp_objective,
                                                   b->n, b->count, b->max_T, b->max_Kp, st),
                                   "batch/backtrack"))
      return e;
  if (stages & CPP_STAGE_LM)
    if (cpp_status e = cuda_status(launch_lm_batch_geo(b->src, b->n, b->count, b->max_T, b->params,
                                                       b->any_geo, st), "batch/lm"))
      return e;
  if (stages & CPP_STAGE_CHECK)
    return cuda_status(launch_check_batch(b->src, b->count, b->params, st), "batch/check");
  return CPP_OK;
}

// Key of a batch in the tuning table: joints, objective, and coarse buckets of the
// batch's shape (request count and longest T as powers of two, the cluster sizes
// present, and how far the largest lattice stands above the mean, log2).
std::string tune_key(const cpp_batch* b) {
  long long total = 0, mx = 0;
  unsigned cs_mask = 0;
  for (int r = 0; r < b->count; ++r) {
    total += b->edges[r];
    mx = std::max(mx, b->edges[r]);
    cs_mask |= 1u << cluster_size(b->reqs[r].Kp, 0);
  }
  auto lg2 = [](double v) { return v > 0 ? (int)std::lround(std::log2(v)) : -99; };
  const double mean = (double)total / b->count;
  char buf[160];
  snprintf(buf, sizeof(buf), "n%d_obj%d_count%d_tmax%d_cs%x_skew%d_sms%d", b->n,
           b->params.dp_objective, lg2(b->count), lg2(b->max_T), cs_mask, lg2(mx / mean),
           device_sm_count());
  return buf;
}

// One line per entry: "key alpha cands_per_cta ms [mask_tasks_per_warp [min_kp
// [budget_ms]]]" (fields absent in older tables: the defaults; budget_ms > 0
// selects per-request forms within that time); the last entry of a key wins.
bool table_lookup(const char* path, const std::string& key, double* alpha, int* cpc, int* tpw,
                  int* min_kp, double* budget_ms) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512], k[200];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    double a, ms, bud = 0.0;
    int c, t = 0, m = 0;
    const int got = sscanf(line, "%199s %lf %d %lf %d %d %lf", k, &a, &c, &ms, &t, &m, &bud);
    if (got < 4 || key != k) continue;
    *alpha = a;
    *cpc = c;
    *tpw = got >= 5 && t >= 1 && t <= 64 ? t : 0;
    *min_kp = got >= 6 && m >= 0 ? m : 0;
    *budget_ms = got == 7 && std::isfinite(bud) && bud > 0 ? bud : 0.0;
    found = true;
  }
  fclose(f);
  return found;
}

}  // namespace

extern "C" {

cpp_status cpp_batch_create(const cpp_robot_t* robots, int32_t n_robots, const cpp_params_t* params,
                            const cpp_plan_desc_t* descs, int32_t count, void* workspace,
                            size_t ws_bytes, int32_t* dev_status, cpp_stream_t stream,
                            cpp_batch_t** out) {
  if (!out) return fail(CPP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!robots || n_robots < 1) return fail(CPP_ERR_INVALID_ARG, "no robots");
  for (int k = 0; k < n_robots; ++k)
    if (cpp_status s = check_robot(&robots[k])) return s;
  if (cpp_status s = check_params(params)) return s;
  if (!descs || count < 1) return fail(CPP_ERR_INVALID_ARG, "no requests");
  const int n = robots[0].n;
  int max_T = 0, max_Kp = 0;
  long long max_tasks = 0;
  for (int r = 0; r < count; ++r) {
    const cpp_plan_desc_t& d = descs[r];
    if (d.robot < 0 || d.robot >= n_robots)
      return fail(CPP_ERR_INVALID_ARG, "request %d: robot index %d out of range", r, d.robot);
    if (robots[d.robot].n != n)
      return fail(CPP_ERR_INVALID_ARG, "request %d: all robots of one batch need the same n", r);
    if (cpp_status s = check_lattice(d.T, d.K, d.Kp, n)) return s;
    if (cpp_status s = check_smooth(params, d.T, n)) return s;
    if (!d.cand || !d.targets || !d.sel || !d.q_out || !d.best_cost)
      return fail(CPP_ERR_INVALID_ARG, "request %d: NULL buffer", r);
    if (!aligned(d.cand, 16)) return fail(CPP_ERR_INVALID_ARG, "request %d: cand misaligned", r);
    max_T = std::max(max_T, d.T);
    max_Kp = std::max(max_Kp, d.Kp);
    max_tasks = std::max(max_tasks, mask_tasks(d.T, d.Kp));
  }
  if (!dp_supported(n, max_Kp)) return fail(CPP_ERR_INVALID_ARG, "Kp too large for shared memory");
  const BatchLayout B = batch_layout(descs, count, n_robots, robots);
  if (!workspace || ws_bytes < B.total || !aligned(workspace, 256))
    return fail(CPP_ERR_INVALID_ARG, "workspace needs %zu bytes, 256-byte aligned", B.total);
  char* ws = static_cast<char*>(workspace);
  std::vector<Req> reqs(count);
  std::vector<long long> edges(count);
  std::vector<std::vector<char>> geos;  // device forms of the requests' collision models
  std::vector<char*> geo_dst;
  for (int r = 0; r < count; ++r) {
    const cpp_plan_desc_t& d = descs[r];
    const PlanLayout& L = B.L[r];
    char* b = ws + B.off[r];
    Req q = empty_req();
    q.T = d.T; q.K = d.K; q.Kp = d.Kp; q.n = n; q.robot = d.robot; q.Kb = bp_stride(d.Kp);
    q.cand = d.cand; q.targets = d.targets;
    q.mask = reinterpret_cast<uint8_t*>(b + L.mask);
    q.pen = reinterpret_cast<float*>(b + L.pen);
    q.pen_min = reinterpret_cast<float*>(b + L.dp_base + L.dp.pen_min);
    q.bp = reinterpret_cast<uint16_t*>(b + L.dp_base + L.dp.bp);
    q.costT = reinterpret_cast<float*>(b + L.dp_base + L.dp.costT);
    q.sel = d.sel; q.best_cost = d.best_cost;
    q.q_seed = reinterpret_cast<float*>(b + L.q_seed);
    q.q_in = q.q_seed; q.q_out = d.q_out; q.pose_err = d.pose_err; q.report = d.report;
    q.smooth_ws = reinterpret_cast<double*>(b + L.smooth);
    q.status = dev_status ? dev_status + r : nullptr;
    if (d.geometry) {
      geos.emplace_back(geo_bytes());
      char msg[160];
      if (!make_geo(*d.geometry, n, geos.back().data(), msg))
        return fail(CPP_ERR_INVALID_ARG, "request %d: %s", r, msg);
      geo_dst.push_back(b + L.geo);
      q.geo = reinterpret_cast<const GeoF*>(b + L.geo);
    }
    reqs[r] = q;
    edges[r] = (long long)(d.T - 1) * d.Kp * d.Kp;
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (size_t k = 0; k < geos.size(); ++k)  // pageable: staged before the call returns
    if (cpp_status e = cuda_status(cudaMemcpyAsync(geo_dst[k], geos[k].data(), geo_bytes(),
                                                   cudaMemcpyHostToDevice, st), "cpp_batch_create"))
      return e;
  // pageable sources: the copies are staged before cudaMemcpyAsync returns
  if (cpp_status e = cuda_status(cudaMemcpyAsync(ws + B.reqs, reqs.data(), sizeof(Req) * count,
                                                 cudaMemcpyHostToDevice, st), "cpp_batch_create"))
    return e;
  if (cpp_status e = cuda_status(cudaMemcpyAsync(ws + B.robots, robots,
                                                 sizeof(cpp_robot_t) * n_robots,
                                                 cudaMemcpyHostToDevice, st), "cpp_batch_create"))
    return e;
  // the LM's work distribution: waypoint prefix sums and robot views
  std::vector<int> wp(count + 1);
  const int wp_total = lm_prefix(reqs.data(), count, wp.data());
  if (cpp_status e = cuda_status(cudaMemcpyAsync(ws + B.lm + B.lm_layout.wp, wp.data(),
                                                 sizeof(int) * (count + 1), cudaMemcpyHostToDevice,
                                                 st), "cpp_batch_create"))
    return e;
  if (cpp_status e = cuda_status(
          launch_robot_views(reinterpret_cast<const cpp_robot_t*>(ws + B.robots), n_robots,
                             reinterpret_cast<RobotViews*>(ws + B.lm + B.lm_layout.views), st),
          "cpp_batch_create"))
    return e;
  cpp_batch* b = new (std::nothrow) cpp_batch;
  if (!b) return fail(CPP_ERR_OOM, "host allocation failed");
  b->src = BatchSrc{reinterpret_cast<const Req*>(ws + B.reqs),
                    reinterpret_cast<const cpp_robot_t*>(ws + B.robots),
                    lm_aux_at(ws + B.lm, B.lm_layout, count, wp_total)};
  b->params = *params;
  b->n = n; b->count = count; b->max_T = max_T; b->max_Kp = max_Kp; b->max_tasks = max_tasks;
  b->d_sched = reinterpret_cast<Req*>(ws + B.sched);
  b->d_robots = reinterpret_cast<const cpp_robot_t*>(ws + B.robots);
  b->reqs = std::move(reqs);
  b->edges = std::move(edges);
  b->any_geo = !geos.empty();
  b->alpha = 0;
  b->cpc = 0;
  b->budget_ms = 0.0;
  b->mask_tpw = 0;
  b->min_kp = 0;
  b->heavy = 0;
  for (int g = 0; g < kMaxGroups; ++g) { b->aux[g] = nullptr; b->join[g] = nullptr; }
  b->fork = nullptr;
  b->graph = nullptr;
  b->graph_stages = 0;
  if (cpp_status e = set_schedule(b, kDefaultAlpha, 0, st)) {
    cpp_batch_destroy(b);
    return e;
  }
  *out = b;
  return CPP_OK;
}

cpp_status cpp_batch_run(cpp_batch_t* b, uint32_t stages, cpp_stream_t stream) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  return run_stages(b, stages, (cudaStream_t)stream);
}

int32_t cpp_batch_launches(const cpp_batch_t* b, uint32_t stages) {
  if (!b) return 0;
  int c = 0;
  for (unsigned s = 1; s <= CPP_STAGE_CHECK; s <<= 1) {
    if (!(stages & s)) continue;
    if (s == CPP_STAGE_LM) { c += lm_launches(b->params, b->any_geo); continue; }
    if (s != CPP_STAGE_DP_FORWARD) { ++c; continue; }
    for (const SchedGroup& g : b->groups) c += g.count > 0 ? 1 : 0;
  }
  return c;
}

cpp_status cpp_batch_set_split(cpp_batch_t* b, double alpha, int32_t cands_per_cta,
                               cpp_stream_t stream) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  if (!std::isfinite(alpha) || alpha < 0) return fail(CPP_ERR_INVALID_ARG, "alpha must be >= 0");
  if (cands_per_cta != 0 && cands_per_cta != 32 && cands_per_cta != 64 && cands_per_cta != 128 &&
      cands_per_cta != 256 && cands_per_cta != 512)
    return fail(CPP_ERR_INVALID_ARG, "cands_per_cta must be 0, 32, 64, 128, 256 or 512");
  return set_schedule(b, alpha, cands_per_cta, (cudaStream_t)stream);
}

cpp_status cpp_batch_set_budget(cpp_batch_t* b, double budget_ms, cpp_stream_t stream) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  if (!std::isfinite(budget_ms) || budget_ms <= 0)
    return fail(CPP_ERR_INVALID_ARG, "budget_ms must be > 0");
  if (schedule_groups(b, budget_forms(b, budget_ms)) > kMaxGroups)
    return fail(CPP_ERR_INVALID_ARG, "budget %.3g ms gives more than %d cluster groups", budget_ms,
                kMaxGroups);
  return set_budget(b, budget_ms, (cudaStream_t)stream);
}

cpp_status cpp_batch_set_cluster_min_kp(cpp_batch_t* b, int32_t min_kp, cpp_stream_t stream) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  if (min_kp < 0) return fail(CPP_ERR_INVALID_ARG, "min_kp must be >= 0");
  b->min_kp = min_kp;
  return b->budget_ms > 0 ? set_budget(b, b->budget_ms, (cudaStream_t)stream)
                          : set_schedule(b, b->alpha, b->cpc, (cudaStream_t)stream);
}

cpp_status cpp_batch_set_mask_tasks(cpp_batch_t* b, int32_t tasks_per_warp) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  if (tasks_per_warp < 0 || tasks_per_warp > 64)
    return fail(CPP_ERR_INVALID_ARG, "tasks_per_warp must be in [0, 64]");
  b->mask_tpw = tasks_per_warp;
  drop_graph(b);
  return CPP_OK;
}

cpp_status cpp_batch_tune(cpp_batch_t* b, const char* table_path, cpp_stream_t stream,
                          cpp_tune_result_t* res) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cpp_tune_result_t out;
  memset(&out, 0, sizeof(out));
  out.dp_ms = out.dp_ms_unsplit = out.mask_ms = out.mask_ms_default = -1.f;
  const std::string key = tune_key(b);
  double alpha = 0, budget = 0;
  int cpc = 0, tpw = 0, mk = 0;
  if (table_lookup(table_path, key, &alpha, &cpc, &tpw, &mk, &budget)) {
    b->min_kp = mk;
    if (cpp_status e = budget > 0 ? set_budget(b, budget, st) : set_schedule(b, alpha, cpc, st))
      return e;
    b->mask_tpw = tpw;
    out.from_table = 1;
  } else {
    // node costs first: the sweeps read them
    if (cpp_status e = run_stages(b, CPP_STAGE_MASK | CPP_STAGE_LAYER_MIN, st)) return e;
    static const double kAlphas[] = {8.0, 4.0, 3.0, 2.0, 1.5, 1.0, 0.75, 0.5,
                                     0.35, 0.25, 0.15, 0.1, 0.05, 1e-9};
    // the smallest Kp that may run as a cluster: any, or each Kp of the batch above
    // its smallest (long requests of small K then stay one CTA each, longest first)
    std::vector<int> kps;
    for (const Req& q : b->reqs) kps.push_back(q.Kp);
    std::sort(kps.begin(), kps.end());
    kps.erase(std::unique(kps.begin(), kps.end()), kps.end());
    std::vector<int> mks{0};
    for (size_t i = 1; i < kps.size(); ++i) mks.push_back(kps[i]);
    // and per-request forms within a search-time budget (ms), the budgets that
    // give distinct schedules with at most kMaxGroups cluster groups
    struct Cand { double alpha; int cpc, mk; double budget; };
    std::vector<Cand> cands{{0.0, 0, 0, 0.0}};
    for (int c : {64, 128, 256, 512})
      for (int m : mks)
        for (double a : kAlphas) cands.push_back({a, c, m, 0.0});
    {
      std::vector<std::vector<int>> seen;
      for (double bud : {1.0, 1.5, 2.0, 3.0, 4.0, 5.0, 6.0, 8.0, 10.0, 12.0, 16.0, 24.0}) {
        const std::vector<int> f = budget_forms(b, bud);
        if (schedule_groups(b, f) > kMaxGroups) continue;
        if (std::find(seen.begin(), seen.end(), f) != seen.end()) continue;
        seen.push_back(f);
        cands.push_back({0.0, 0, 0, bud});
      }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cpp_status e = cuda_status(cudaEventCreate(&e0), "cpp_batch_tune")) return e;
    if (cpp_status e = cuda_status(cudaEventCreate(&e1), "cpp_batch_tune")) {
      cudaEventDestroy(e0);
      return e;
    }
    float best_ms = HUGE_VALF;
    Cand best{0.0, 0, 0, 0.0};
    int last_heavy = -1, last_cpc = -1, last_mk = -1;
    cpp_status err = CPP_OK;
    for (const Cand& c : cands) {
      b->min_kp = c.mk;
      if ((err = c.budget > 0 ? set_budget(b, c.budget, st) : set_schedule(b, c.alpha, c.cpc, st)) !=
          CPP_OK)
        break;
      // same split as before (the heavy set only grows down the ladder)
      if (c.budget <= 0 && b->heavy == last_heavy && c.cpc == last_cpc && c.mk == last_mk)
        continue;
      last_heavy = b->heavy;
      last_cpc = c.cpc;
      last_mk = c.mk;
      if (c.budget <= 0 && c.alpha > 0 && b->heavy == 0) continue;  // same as alpha = 0
      if (c.budget > 0 && b->heavy == 0) continue;                  // same as alpha = 0
      float ms = HUGE_VALF;
      for (int rep = 0; rep < 3 && err == CPP_OK; ++rep) {  // the first run warms up
        cudaError_t ce = cudaEventRecord(e0, st);
        if (ce == cudaSuccess) ce = run_forward(b, st);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float t = 0;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
        err = cuda_status(ce, "cpp_batch_tune");
        if (rep > 0) ms = std::min(ms, t);
      }
      if (err != CPP_OK) break;
      ++out.timed;
      if (c.alpha == 0.0) out.dp_ms_unsplit = ms;
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
    // the mask stage: 128-candidate tasks per warp (how many waypoints a warp
    // covers at each K), same timing rule
    float best_mask = HUGE_VALF;
    int best_tpw = 0;
    for (int t : {1, 2, 4, 8, 16}) {
      if (err != CPP_OK) break;
      b->mask_tpw = t;
      float ms = HUGE_VALF;
      for (int rep = 0; rep < 3 && err == CPP_OK; ++rep) {
        cudaError_t ce = cudaEventRecord(e0, st);
        if (ce == cudaSuccess)
          ce = launch_mask_batch(b->src, b->n, b->count, b->max_tasks, b->params, b->any_geo, st, t);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float tm = 0;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&tm, e0, e1);
        err = cuda_status(ce, "cpp_batch_tune");
        if (rep > 0) ms = std::min(ms, tm);
      }
      if (err != CPP_OK) break;
      ++out.timed;
      if (t == 4) out.mask_ms_default = ms;
      if (ms < best_mask) { best_mask = ms; best_tpw = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != CPP_OK) return err;
    b->mask_tpw = best_tpw;
    out.mask_ms = best_mask;
    b->min_kp = best.mk;
    if (cpp_status e = best.budget > 0 ? set_budget(b, best.budget, st)
                                       : set_schedule(b, best.alpha, best.cpc, st))
      return e;
    out.dp_ms = best_ms;
    if (table_path) {
      FILE* f = fopen(table_path, "a");
      if (!f) return fail(CPP_ERR_INVALID_ARG, "cannot append to tuning table %s", table_path);
      fprintf(f, "%s %.9g %d %.4f %d %d %.9g\n", key.c_str(), best.alpha, best.cpc, best_ms,
              best_tpw, best.mk, best.budget);
      fclose(f);
    }
  }
  out.alpha = b->alpha;
  out.cands_per_cta = b->cpc;
  out.mask_tasks_per_warp = b->mask_tpw > 0 ? b->mask_tpw : 4;
  out.cluster_min_kp = b->min_kp;
  out.budget_ms = (float)b->budget_ms;
  out.heavy = b->heavy;
  out.forward_launches = 0;
  for (const SchedGroup& g : b->groups) out.forward_launches += g.count > 0 ? 1 : 0;
  if (res) *res = out;
  return CPP_OK;
}

cpp_status cpp_batch_capture(cpp_batch_t* b, uint32_t stages, cpp_stream_t stream) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return fail(CPP_ERR_INVALID_ARG, "capture needs a created stream, not the default stream");
  drop_graph(b);
  if (cpp_status e = cuda_status(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal),
                                 "cpp_batch_capture"))
    return e;
  const cpp_status run = run_stages(b, stages, st);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(st, &g);
  if (run != CPP_OK) {
    if (g) cudaGraphDestroy(g);
    return run;
  }
  if (cpp_status e = cuda_status(ee, "cpp_batch_capture")) return e;
  cudaGraphExec_t x = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (cpp_status e = cuda_status(ie, "cpp_batch_capture")) return e;
  b->graph = x;
  b->graph_stages = stages;
  return CPP_OK;
}

cpp_status cpp_batch_replay(cpp_batch_t* b, cpp_stream_t stream) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  if (!b->graph) return fail(CPP_ERR_INVALID_ARG, "no captured graph (cpp_batch_capture first)");
  return cuda_status(cudaGraphLaunch(b->graph, (cudaStream_t)stream), "cpp_batch_replay");
}

void cpp_batch_destroy(cpp_batch_t* b) {
  if (!b) return;
  drop_graph(b);
  for (int g = 0; g < kMaxGroups; ++g) {
    if (b->aux[g]) cudaStreamDestroy(b->aux[g]);
    if (b->join[g]) cudaEventDestroy(b->join[g]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

cpp_status cpp_plan_batch(const cpp_robot_t* robots, int32_t n_robots, const cpp_params_t* params,
                          const cpp_plan_desc_t* descs, int32_t count, void* workspace,
                          size_t ws_bytes, int32_t* dev_status, cpp_stream_t stream) {
  cpp_batch_t* b = nullptr;
  if (cpp_status e = cpp_batch_create(robots, n_robots, params, descs, count, workspace, ws_bytes,
                                      dev_status, stream, &b))
    return e;
  const cpp_status e = cpp_batch_run(b, CPP_STAGE_ALL, stream);
  cpp_batch_destroy(b);
  return e;
}

}  // extern "C"
