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

static cpp_status mask_impl(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                            const double* targets, int32_t T, int32_t K, int32_t Kp,
                            int32_t k_begin, uint8_t* mask, float* pen, float* err,
                            int32_t* dev_status, cpp_stream_t stream) {
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  if (cpp_status s = check_lattice(T, K, Kp, robot->n)) return s;
  if (k_begin < 0 || k_begin > K || k_begin % 4 != 0)
    return fail(CPP_ERR_INVALID_ARG, "k_begin = %d must be a multiple of 4 in [0, K]", k_begin);
  if (!cand || !targets || !mask || !pen) return fail(CPP_ERR_INVALID_ARG, "NULL buffer");
  if (!aligned(cand, 16) || !aligned(pen, 16) || !aligned(mask, 4) || (err && !aligned(err, 16)))
    return fail(CPP_ERR_INVALID_ARG, "cand/pen/err must be 16-byte and mask 4-byte aligned");
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.K = K; s.r.Kp = Kp; s.r.n = robot->n; s.r.k_begin = k_begin;
  s.r.cand = cand; s.r.targets = targets; s.r.mask = mask; s.r.pen = pen; s.r.err = err;
  s.r.status = dev_status;
  s.robot = *robot;
  return cuda_status(launch_mask(s, *params, (cudaStream_t)stream), "cpp_mask");
}

cpp_status cpp_mask(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                    const double* targets, int32_t T, int32_t K, int32_t Kp, uint8_t* mask,
                    float* pen, float* err, int32_t* dev_status, cpp_stream_t stream) {
  return mask_impl(robot, params, cand, targets, T, K, Kp, 0, mask, pen, err, dev_status, stream);
}

cpp_status cpp_mask_range(const cpp_robot_t* robot, const cpp_params_t* params,
                          const float* cand, const double* targets, int32_t T, int32_t K,
                          int32_t Kp, int32_t k_begin, uint8_t* mask, float* pen, float* err,
                          int32_t* dev_status, cpp_stream_t stream) {
  return mask_impl(robot, params, cand, targets, T, K, Kp, k_begin, mask, pen, err, dev_status,
                   stream);
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
  SingleSrc s;
  s.r = empty_req();
  s.r.T = T; s.r.n = robot->n;
  s.r.q_in = q_in; s.r.q_out = q_out; s.r.targets = targets; s.r.pose_err = pose_err;
  s.r.status = dev_status;
  s.robot = *robot;
  return cuda_status(launch_lm(s, *params, true, (cudaStream_t)stream), "cpp_lm_refine");
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
  if (cpp_status s = check_robot(robot)) return s;
  if (cpp_status s = check_params(params)) return s;
  const int n = robot->n;
  if (cpp_status s = check_lattice(T, K, Kp, n)) return s;
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
  s.r.status = dev_status;
  s.robot = *robot;
  if (cpp_status e = cuda_status(launch_mask(s, *params, st), "cpp_plan/mask")) return e;
  if (cpp_status e = cuda_status(launch_dp(s, CPP_STAGE_LAYER_MIN | CPP_STAGE_DP_FORWARD |
                                                   CPP_STAGE_BACKTRACK, params->dp_objective, st),
                                 "cpp_plan/dp"))
    return e;
  // the check below writes the FP64 pose errors
  if (cpp_status e = cuda_status(launch_lm(s, *params, false, st), "cpp_plan/lm")) return e;
  return cuda_status(launch_check(s, *params, st), "cpp_plan/check");
}

// ------------------------------------------------------------------ many requests
namespace {
struct BatchLayout {
  size_t reqs, robots, per_req_base, total;
  std::vector<PlanLayout> L;
  std::vector<size_t> off;
};
BatchLayout batch_layout(const cpp_plan_desc_t* d, int count, int n_robots, const cpp_robot_t* robots) {
  BatchLayout B;
  size_t o = 0;
  B.reqs = o;   o += align256(sizeof(Req) * (size_t)count);
  B.robots = o; o += align256(sizeof(cpp_robot_t) * (size_t)n_robots);
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

struct cpp_batch {
  BatchSrc src;
  cpp_params_t params;
  int n, count, max_T, max_Kp;
  long long max_tasks;
};

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
    q.status = dev_status ? dev_status + r : nullptr;
    reqs[r] = q;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // pageable sources: the copies are staged before cudaMemcpyAsync returns
  if (cpp_status e = cuda_status(cudaMemcpyAsync(ws + B.reqs, reqs.data(), sizeof(Req) * count,
                                                 cudaMemcpyHostToDevice, st), "cpp_batch_create"))
    return e;
  if (cpp_status e = cuda_status(cudaMemcpyAsync(ws + B.robots, robots,
                                                 sizeof(cpp_robot_t) * n_robots,
                                                 cudaMemcpyHostToDevice, st), "cpp_batch_create"))
    return e;
  cpp_batch* b = new (std::nothrow) cpp_batch;
  if (!b) return fail(CPP_ERR_OOM, "host allocation failed");
  b->src = BatchSrc{reinterpret_cast<const Req*>(ws + B.reqs),
                    reinterpret_cast<const cpp_robot_t*>(ws + B.robots)};
  b->params = *params;
  b->n = n; b->count = count; b->max_T = max_T; b->max_Kp = max_Kp; b->max_tasks = max_tasks;
  *out = b;
  return CPP_OK;
}

cpp_status cpp_batch_run(cpp_batch_t* b, uint32_t stages, cpp_stream_t stream) {
  if (!b) return fail(CPP_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (stages & CPP_STAGE_MASK)
    if (cpp_status e = cuda_status(launch_mask_batch(b->src, b->n, b->count, b->max_tasks,
                                                     b->params, st), "batch/mask"))
      return e;
  const unsigned dp = stages & (CPP_STAGE_LAYER_MIN | CPP_STAGE_DP_FORWARD | CPP_STAGE_BACKTRACK);
  if (dp)
    if (cpp_status e = cuda_status(launch_dp_batch(b->src, dp, b->params.dp_objective, b->n,
                                                   b->count, b->max_T, b->max_Kp, st), "batch/dp"))
      return e;
  if (stages & CPP_STAGE_LM)
    if (cpp_status e = cuda_status(launch_lm_batch(b->src, b->n, b->count, b->max_T, b->params, st),
                                   "batch/lm"))
      return e;
  if (stages & CPP_STAGE_CHECK)
    return cuda_status(launch_check_batch(b->src, b->count, b->params, st), "batch/check");
  return CPP_OK;
}

int32_t cpp_batch_launches(const cpp_batch_t* b, uint32_t stages) {
  if (!b) return 0;
  int c = 0;
  for (unsigned s = 1; s <= CPP_STAGE_CHECK; s <<= 1)
    if (stages & s) ++c;
  return c;
}

void cpp_batch_destroy(cpp_batch_t* b) { delete b; }

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
