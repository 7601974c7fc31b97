// server.cu -- continuous-batching request loop (cpp_server_*, cpp_plan_submit /
// poll / wait / cancel). Not in the paper: it serves the planner core to many
// clients at once.
//
// Structure
//  * a device arena of hbm_budget_bytes, sub-allocated first-fit per request:
//    a request is admitted only when its whole footprint (lattice, targets,
//    plan scratch, outputs) fits, so lattices and search tables stay resident
//    on the device for the request's lifetime on the GPU;
//  * a pinned host pool for copied inputs (pageable fallback) and, per launch,
//    the request table's mirror and the staging of its results: the worker moves
//    each result into its request when the launch retires, so pinned memory
//    holds only what is in flight, however late the clients collect, and no
//    copy to or from pageable memory stalls the worker while launches run;
//  * one worker thread: it retires finished launches (event query), then forms
//    the next batch from the queue -- requests of the oldest request's size
//    class (joint count, K bucket, T bucket) in arrival order, while the class
//    cap, slots and arena space allow -- stages it (H2D copies of its inputs
//    and request table on a copy stream) and enqueues the six stage launches and
//    the D2H copy of results on one of max_inflight streams. When every stream
//    is busy and a full batch is queued, one batch is formed and staged ahead,
//    so its copies overlap the running launches instead of idling a stream.
//    Requests that arrive while earlier batches run are admitted into the next
//    batch as memory frees up, and the batches overlap on the device.
//  * two regimes. At light load (few requests queued or on the device) a batch
//    holds requests of one size class (joint count, K bucket, T bucket) and each
//    search runs in the latency form (the smallest tile: clusters of up to 16
//    CTAs), the fastest for a lone request. Under load a batch takes requests of
//    every K whose searches take about as long (one joint count and a factor-2
//    band of estimated search time, so short requests never wait for long
//    ones), and each search runs in the form with the highest edge rate per SM
//    that stays within search_budget_ms (one CTA, wide clusters of 512 or 256
//    successors per CTA, clusters of 128, else of 64; pick_search_form): the
//    search is launched once per K bucket and form, the launches forked onto
//    auxiliary streams of the batch's stream so they run side by side.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace cppflow;
using Clock = std::chrono::steady_clock;

namespace {

cpp_status sfail(cpp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

// First-fit allocator over [0, size) in 256-byte units.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = high_ = 0;
    size_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t start = it->first + bytes, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[start] = rest;
      used_ += bytes;
      high_ = std::max(high_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
    used_ -= bytes;
  }
  size_t used() const { return used_; }
  size_t high_water() const { return high_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, high_ = 0, size_ = 0;
};

enum class St { Queued, Running, Improving, Done, Failed, Cancelled };

struct Request {
  uint64_t ticket = 0;
  cpp_robot_t robot;
  int T = 0, K = 0, Kp = 0, n = 0;
  // inputs on the host (borrowed, pinned copy or pageable copy)
  const float* cand = nullptr;
  const double* targets = nullptr;
  std::vector<char> own_in;
  // results on the host: copied here from the launch's pinned staging when the
  // launch retires (for an anytime request, the latest pass's result)
  std::vector<char> own_out;
  std::vector<char> geo;  // device form of the collision model (empty: none)
  size_t pin_off = 0, pin_bytes = 0;
  bool pinned = false;
  // device slot: [cand][targets][outputs][plan scratch]
  size_t dev_off = 0, dev_bytes = 0;
  size_t o_cand = 0, o_tgt = 0, o_out = 0, o_ws = 0;
  size_t out_bytes = 0, o_sel = 0, o_q = 0, o_err = 0, o_rep = 0, o_best = 0;
  St state = St::Queued;
  cpp_status result = CPP_OK;
  int32_t dev_status = 0;
  Clock::time_point t_submit, t_done;
  // anytime planning: improvement rounds after the first pass, best result so far
  bool anytime = false, stop_improving = false, have_best = false;
  int rounds_left = 0, rounds_done = 0, best_rounds = 0;
  double best_len = 0.0;
  std::vector<char> best_out;  // host copy of the best published result (out_bytes)
};

struct Layout {
  size_t cand, tgt, out, ws, total;
  size_t sel, q, err, rep, best, out_bytes;
};

Layout slot_layout(int T, int Kp, int n) {
  Layout L;
  size_t o = 0;
  L.cand = o; o += align256((size_t)T * n * Kp * sizeof(float));
  L.tgt = o;  o += align256((size_t)T * 7 * sizeof(double));
  L.out = o;
  size_t u = 0;
  L.err = u;  u += (size_t)T * 2 * sizeof(double);
  L.rep = u;  u += sizeof(cpp_report_t);
  L.q = u;    u += (size_t)T * n * sizeof(float);
  L.sel = u;  u += (size_t)T * sizeof(int32_t);
  L.best = u; u += sizeof(float);
  L.out_bytes = u;
  o += align256(u);
  L.ws = o;   o += plan_layout(T, Kp, n).total;
  L.total = o;
  return L;
}

struct SearchGroup {  // requests of one K bucket and search form in a launch's table:
                     // [begin, begin + count)
  int begin = 0, count = 0, max_Kp = 0;
  int form = 0, cpc = 0;  // the forward sweep's form and successors per CTA
};

struct Launch {
  std::vector<Request*> reqs;
  bool improve = false;  // an anytime improvement round (slots already resident)
  bool latency = true;   // search in the latency form (light load) or the throughput form
  std::vector<SearchGroup> groups;  // the search's launches (throughput form)
  int stream = -1;       // compute stream, set when the kernels are enqueued
  cudaEvent_t copied = nullptr;  // inputs and table on the device (copy stream)
  cudaEvent_t done = nullptr;
  int n = 0, max_T = 0, max_Kp = 0;
  long long max_tasks = 0;
  bool any_geo = false;
  size_t tab_off = 0, tab_bytes = 0;      // device: Req[] | robots[] | status[] | LM aux
  int wp_total = 0;                       // waypoints of the launch's requests
  size_t tab_pin = 0, tab_pin_bytes = 0;  // pinned host mirror, then the results' staging
  bool tab_pinned = false;
  std::vector<char> tab_host;             // pageable fallback
  char* tab_h = nullptr;
  std::vector<size_t> out_off;            // per request (table order): its results' offset
                                          // in tab_h, set when the launch is enqueued
};

}  // namespace

struct cpp_server {
  cpp_server_config_t cfg;
  char* d_arena = nullptr;
  Arena darena;
  char* h_pinned = nullptr;
  Arena parena;
  std::vector<cudaStream_t> streams;
  std::vector<bool> stream_busy;
  // per compute stream: auxiliary streams and events that fork the search of a
  // mixed-K launch into one launch per K bucket and join it back
  static constexpr int kBuckets = 8;  // auxiliary streams per compute stream
  std::vector<cudaStream_t> aux;       // [max_inflight][kBuckets]
  std::vector<cudaEvent_t> aux_done;   // [max_inflight][kBuckets]
  std::vector<cudaEvent_t> fork_ev;    // [max_inflight]
  cudaStream_t copy_stream = nullptr;  // host-to-device copies of formed launches
  std::deque<Launch*> staged;          // formed, inputs copying, waiting for a stream
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::deque<Request*> improve_q;  // anytime requests waiting for their next round
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<Launch*> inflight;
  int resident = 0;
  int sms = 152;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  cpp_server_stats_t stats;
  std::string fatal;

  void run();
  bool form_batch(Launch* L);
  bool form_improve(Launch* L);
  bool alloc_table(Launch* L);
  void finish(Request* r);
  void anytime_step(Request* r, bool improve_round, const char* res);
  cpp_status stage(Launch* L);
  cpp_status enqueue(Launch* L);
  cudaError_t search(Launch* L, const BatchSrc& src, cudaStream_t st);
  void retire(Launch* L, cudaError_t e);
  void release_host(Request* r);
};

void cpp_server::release_host(Request* r) {
  if (r->pinned) {
    parena.release(r->pin_off, r->pin_bytes);
    r->pinned = false;
  }
  r->own_in.clear();
  r->own_in.shrink_to_fit();
}

// K bucket of a request (the search's launch groups) and T bucket.
static int k_bucket(const Request* r) {
  return r->Kp <= 128 ? 0 : r->Kp <= 256 ? 1 : r->Kp <= 512 ? 2 : 3;
}
static int t_bucket(const Request* r) { return r->T <= 256 ? 0 : r->T <= 1024 ? 1 : 2; }

// The search form of a request under load (the library's measured-rate policy).
static SearchForm throughput_form(const Request* r, double budget_ms) {
  return pick_search_form(r->T, r->Kp, budget_ms);
}

// Search time class under load: requests whose estimated search times (in their
// throughput forms) fall in the same factor-2 band finish at about the same time.
static int time_class(const Request* r, double budget_ms) {
  const double ms = throughput_form(r, budget_ms).est_ms;
  return std::max(0, std::min(31, (int)std::floor(std::log2(std::max(ms, 1e-3)) + 10.0)));
}

// Size class of a request. At light load: joint count, K bucket and T bucket --
// a launch holds one class only, so a small request never waits for a large one
// in its batch (a batch completes as a whole) and a K = 1024 request never widens
// the kernel of K = 128 ones. Under load: joint count and search time class --
// every K shares the launch (its search runs one launch per K bucket), and the
// requests of a launch finish their searches at about the same time, so few of
// them wait for the others.
static int size_class(const Request* r, bool latency, double budget_ms) {
  if (latency) return (r->n * 4 + k_bucket(r)) * 3 + t_bucket(r);
  return 1000 + r->n * 32 + time_class(r, budget_ms);
}

// Largest batch of a class under light load: heavy classes (K > 512 or T > 1024)
// are capped so the batch runs as clusters (8 CTAs per request, lower latency per
// request); the others up to max_batch. Under load (the throughput form, whose
// clusters are formed per request whatever the batch size) every class takes
// up to max_batch.
static int class_cap(const Request* r, int max_batch, int sms, bool latency) {
  if (!latency) return max_batch;
  const bool heavy = r->Kp > 512 || r->T > 1024;
  const int cs = cluster_size(r->Kp, 0);
  return heavy ? std::max(1, std::min(max_batch, sms / std::max(1, cs))) : max_batch;
}

// Take requests of the oldest request's size class, in arrival order, while the
// class cap, slots and arena allow. The launch takes the latency form while the
// requests queued and on the device are few, the throughput form otherwise.
bool cpp_server::form_batch(Launch* L) {
  if (queue.empty()) return false;
  L->latency = (int)queue.size() + resident <= cfg.latency_requests;
  const double budget = cfg.search_budget_ms;
  const int cls = size_class(queue.front(), L->latency, budget);
  const int cap = class_cap(queue.front(), cfg.max_batch, sms, L->latency);
  for (auto it = queue.begin(); it != queue.end();) {
    Request* r = *it;
    if ((int)L->reqs.size() >= cap || resident >= cfg.max_slots) break;
    if (size_class(r, L->latency, budget) != cls) { ++it; continue; }
    size_t off;
    if (!darena.alloc(r->dev_bytes, &off)) break;  // keep arrival order within the class
    r->dev_off = off;
    r->state = St::Running;
    ++resident;
    L->reqs.push_back(r);
    it = queue.erase(it);
  }
  if (L->reqs.empty()) return false;
  if (!alloc_table(L)) {
    // no room for the table: give the requests back
    for (Request* r : L->reqs) {
      darena.release(r->dev_off, r->dev_bytes);
      r->state = St::Queued;
      --resident;
    }
    for (auto it = L->reqs.rbegin(); it != L->reqs.rend(); ++it) queue.push_front(*it);
    L->reqs.clear();
    return false;
  }
  return true;
}

// Device table of a launch: Req[] | robots[] | status[] | the LM's work
// distribution (robot views, waypoint prefix sums, counter); the host mirror
// holds the same bytes (the views are formed on the device after the copy).
static size_t tab_robots(int count) { return align256(sizeof(Req) * count); }
static size_t tab_status(int count) { return tab_robots(count) + align256(sizeof(cpp_robot_t) * count); }
static size_t tab_lm(int count) { return tab_status(count) + align256(sizeof(int32_t) * count); }
static size_t tab_total(int count) { return tab_lm(count) + lm_aux_layout(count, count).total; }

// The host side is pinned: the table's mirror, then every request's results
// (the device-to-host copies land there; the worker moves them into the request
// when the launch retires). A copy to or from pageable memory would block the
// worker until the stream's earlier work is done, so without pinned room the
// launch waits for launches in flight to retire; with none in flight it takes
// pageable memory.
bool cpp_server::alloc_table(Launch* L) {
  const int count = (int)L->reqs.size();
  L->tab_bytes = tab_total(count);
  size_t o = align256(L->tab_bytes);
  for (const Request* r : L->reqs) o += align256(r->out_bytes);
  L->tab_pin_bytes = o;
  const bool pin = h_pinned && parena.alloc(L->tab_pin_bytes, &L->tab_pin);
  if (!pin && (!inflight.empty() || !staged.empty())) return false;
  if (!darena.alloc(L->tab_bytes, &L->tab_off)) {
    if (pin) parena.release(L->tab_pin, L->tab_pin_bytes);
    return false;
  }
  if (pin) {
    L->tab_pinned = true;
    L->tab_h = h_pinned + L->tab_pin;
  } else {
    L->tab_host.resize(L->tab_pin_bytes);
    L->tab_h = L->tab_host.data();
  }
  return true;
}

// An improvement launch: anytime requests of one joint count, in queue order.
bool cpp_server::form_improve(Launch* L) {
  if (improve_q.empty()) return false;
  const int n = improve_q.front()->n;
  for (auto it = improve_q.begin(); it != improve_q.end();) {
    if ((int)L->reqs.size() >= cfg.max_batch) break;
    if ((*it)->n != n) { ++it; continue; }
    (*it)->state = St::Running;
    L->reqs.push_back(*it);
    it = improve_q.erase(it);
  }
  L->improve = true;
  if (!alloc_table(L)) {
    for (auto it = L->reqs.rbegin(); it != L->reqs.rend(); ++it) {
      (*it)->state = St::Improving;
      improve_q.push_front(*it);
    }
    L->reqs.clear();
    return false;
  }
  return true;
}

// A finished request: its best published result (anytime) becomes the result;
// the device slot is freed.
void cpp_server::finish(Request* r) {
  if (r->have_best) r->own_out = r->best_out;
  darena.release(r->dev_off, r->dev_bytes);
  --resident;
  r->t_done = Clock::now();
  r->state = St::Done;
  r->result = r->dev_status == 0 ? CPP_OK : (cpp_status)r->dev_status;
  ++stats.completed;
}

// After a pass or an improvement round of an anytime request (its results at
// `res`): publish the result when it is valid and (after the first) shorter;
// queue the next round or finish.
void cpp_server::anytime_step(Request* r, bool improve_round, const char* res) {
  if (improve_round) {
    ++r->rounds_done;
    --r->rounds_left;
    ++stats.improve_rounds;
  }
  cpp_report_t rep;
  memcpy(&rep, res + r->o_rep, sizeof(rep));
  r->own_out.assign(res, res + r->out_bytes);
  if (r->dev_status == 0 && rep.valid && (!r->have_best || rep.traj_len < r->best_len)) {
    r->best_out.assign(res, res + r->out_bytes);
    r->have_best = true;
    r->best_len = rep.traj_len;
    r->best_rounds = r->rounds_done;
    ++stats.published;
  }
  if (r->rounds_left > 0 && !r->stop_improving && r->dev_status == 0) {
    r->state = St::Improving;
    improve_q.push_back(r);
  } else {
    finish(r);
  }
}

// The host-to-device part of a launch, on the copy stream: the requests'
// inputs (not for improvement rounds, whose inputs are resident) and the request
// table; `copied` marks the end. Launches staged while every compute stream is
// busy thus copy while the earlier launches compute.
cpp_status cpp_server::stage(Launch* L) {
  const cudaStream_t st = copy_stream;
  const int count = (int)L->reqs.size();
  if (!L->latency && !L->improve) {
    // the table in K buckets (largest first), each bucket longest request first:
    // one contiguous sub-table per search launch, and the one-CTA bucket hands
    // its longest requests to the block scheduler first
    const double budget = cfg.search_budget_ms;
    auto key = [budget](const Request* r) {  // search launch group of a request
      return 8 * k_bucket(r) + throughput_form(r, budget).rank;
    };
    std::stable_sort(L->reqs.begin(), L->reqs.end(), [&](const Request* a, const Request* b) {
      const int ka = key(a), kb = key(b);
      return ka != kb ? ka > kb : a->T > b->T;
    });
    L->groups.clear();
    for (int i = 0; i < count; ++i) {
      if (L->groups.empty() || key(L->reqs[L->groups.back().begin]) != key(L->reqs[i])) {
        const SearchForm f = throughput_form(L->reqs[i], budget);
        L->groups.push_back(SearchGroup{i, 0, 0, f.form, f.cpc});
      }
      SearchGroup& g = L->groups.back();
      ++g.count;
      g.max_Kp = std::max(g.max_Kp, L->reqs[i]->Kp);
    }
  }
  const int n = L->reqs[0]->n;
  char* tab_d = d_arena + L->tab_off;
  Req* tq = reinterpret_cast<Req*>(L->tab_h);
  cpp_robot_t* trob = reinterpret_cast<cpp_robot_t*>(L->tab_h + tab_robots(count));
  int32_t* tst = reinterpret_cast<int32_t*>(L->tab_h + align256(sizeof(Req) * count) +
                                            align256(sizeof(cpp_robot_t) * count));
  int32_t* tst_d = reinterpret_cast<int32_t*>(tab_d + align256(sizeof(Req) * count) +
                                              align256(sizeof(cpp_robot_t) * count));
  int max_T = 0, max_Kp = 0;
  long long max_tasks = 0;
  bool any_geo = false;
  for (int i = 0; i < count; ++i) {
    Request* r = L->reqs[i];
    char* b = d_arena + r->dev_off;
    cudaError_t e = cudaSuccess;
    if (!L->improve) {  // an improvement round finds its inputs resident
      e = cudaMemcpyAsync(b + r->o_cand, r->cand, (size_t)r->T * r->n * r->Kp * sizeof(float),
                          cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + r->o_tgt, r->targets, (size_t)r->T * 7 * sizeof(double),
                            cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return sfail(CPP_ERR_CUDA, "server H2D: %s", cudaGetErrorString(e));
    }
    Req q;
    memset(&q, 0, sizeof(q));
    q.T = r->T; q.K = r->K; q.Kp = r->Kp; q.n = r->n; q.robot = i; q.Kb = bp_stride(r->Kp);
    q.cand = reinterpret_cast<const float*>(b + r->o_cand);
    q.targets = reinterpret_cast<const double*>(b + r->o_tgt);
    const PlanLayout PL = plan_layout(r->T, r->Kp, r->n);
    carve_plan(q, b + r->o_ws, PL);
    if (!r->geo.empty()) {  // pageable source: staged before the call returns
      if (!L->improve) {
        e = cudaMemcpyAsync(b + r->o_ws + PL.geo, r->geo.data(), r->geo.size(),
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return sfail(CPP_ERR_CUDA, "server H2D: %s", cudaGetErrorString(e));
      }
      q.geo = reinterpret_cast<const GeoF*>(b + r->o_ws + PL.geo);
      any_geo = true;
    }
    char* out = b + r->o_out;
    q.sel = reinterpret_cast<int32_t*>(out + r->o_sel);
    q.q_out = reinterpret_cast<float*>(out + r->o_q);
    q.pose_err = reinterpret_cast<double*>(out + r->o_err);
    q.report = reinterpret_cast<cpp_report_t*>(out + r->o_rep);
    q.best_cost = reinterpret_cast<float*>(out + r->o_best);
    q.status = tst_d + i;
    tq[i] = q;
    trob[i] = r->robot;
    tst[i] = 0;
    max_T = std::max(max_T, r->T);
    max_Kp = std::max(max_Kp, r->Kp);
    max_tasks = std::max(max_tasks, mask_tasks(r->T, r->Kp));
  }
  // the LM's work distribution: waypoint prefix sums (copied with the table) and
  // robot views (formed on the device after it)
  const LmAuxLayout LA = lm_aux_layout(count, count);
  L->wp_total = lm_prefix(tq, count, reinterpret_cast<int*>(L->tab_h + tab_lm(count) + LA.wp));
  cudaError_t e = cudaMemcpyAsync(tab_d, L->tab_h, L->tab_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_robot_views(reinterpret_cast<const cpp_robot_t*>(tab_d + tab_robots(count)), count,
                           reinterpret_cast<RobotViews*>(tab_d + tab_lm(count) + LA.views), st);
  if (e == cudaSuccess) e = cudaEventRecord(L->copied, st);
  if (e != cudaSuccess) return sfail(CPP_ERR_CUDA, "server H2D table: %s", cudaGetErrorString(e));
  L->n = n;
  L->max_T = max_T;
  L->max_Kp = max_Kp;
  L->max_tasks = max_tasks;
  L->any_geo = any_geo;
  return CPP_OK;
}

// The search of a launch on its compute stream. Light load: one launch in the
// latency form. Under load: layer minima over the whole table, then one forward
// launch per K bucket in the throughput form -- a single bucket on the stream
// itself, several forked onto the stream's auxiliary streams and joined back --
// then the backtracking over the whole table.
cudaError_t cpp_server::search(Launch* L, const BatchSrc& src, cudaStream_t st) {
  const int count = (int)L->reqs.size(), n = L->n;
  const int obj = cfg.params.dp_objective;
  if (L->latency || L->groups.size() <= 1) {
    const int form = L->latency ? kFormAuto : L->groups[0].form;
    const int cpc = L->latency ? 0 : L->groups[0].cpc;
    return launch_dp_batch_form(src, CPP_STAGE_LAYER_MIN | CPP_STAGE_DP_FORWARD | CPP_STAGE_BACKTRACK,
                                obj, n, count, L->max_T, L->max_Kp, form, cpc, st);
  }
  cudaError_t e = launch_dp_batch_form(src, CPP_STAGE_LAYER_MIN, obj, n, count, L->max_T, L->max_Kp,
                                       kFormAuto, 0, st);
  if (e != cudaSuccess) return e;
  const int s = L->stream;
  if ((e = cudaEventRecord(fork_ev[s], st)) != cudaSuccess) return e;
  for (size_t g = 0; g < L->groups.size(); ++g) {
    const SearchGroup& G = L->groups[g];
    const size_t slot = (size_t)s * kBuckets + g % kBuckets;  // groups beyond kBuckets share
    const cudaStream_t a = aux[slot];
    if ((e = cudaStreamWaitEvent(a, fork_ev[s], 0)) != cudaSuccess) return e;
    // the forward sweep reads the request table only (Req::robot indexes the full table)
    const BatchSrc sub{src.r + G.begin, src.robots};
    if ((e = launch_forward(sub, obj, n, G.count, G.max_Kp, G.form, G.cpc, a)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(aux_done[slot], a)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, aux_done[slot], 0)) != cudaSuccess) return e;
  }
  return launch_dp_batch_form(src, CPP_STAGE_BACKTRACK, obj, n, count, L->max_T, L->max_Kp,
                              kFormAuto, 0, st);
}

// The device part of a staged launch on its compute stream: wait for its copies,
// the stage kernels, the device-to-host copies of the results, `done`.
cpp_status cpp_server::enqueue(Launch* L) {
  const cudaStream_t st = streams[L->stream];
  const int count = (int)L->reqs.size();
  const int n = L->n, max_T = L->max_T;
  const long long max_tasks = L->max_tasks;
  const bool any_geo = L->any_geo;
  char* tab_d = d_arena + L->tab_off;
  int32_t* tst = reinterpret_cast<int32_t*>(L->tab_h + align256(sizeof(Req) * count) +
                                            align256(sizeof(cpp_robot_t) * count));
  int32_t* tst_d = reinterpret_cast<int32_t*>(tab_d + align256(sizeof(Req) * count) +
                                              align256(sizeof(cpp_robot_t) * count));
  cudaError_t e = cudaStreamWaitEvent(st, L->copied, 0);
  if (e != cudaSuccess) return sfail(CPP_ERR_CUDA, "server launch: %s", cudaGetErrorString(e));
  BatchSrc src{reinterpret_cast<const Req*>(tab_d),
               reinterpret_cast<const cpp_robot_t*>(tab_d + tab_robots(count)),
               lm_aux_at(tab_d + tab_lm(count), lm_aux_layout(count, count), count, L->wp_total)};
  if (L->improve) {
    if ((e = launch_improve_batch(src, n, count, max_T, cfg.params, any_geo, st)) != cudaSuccess)
      return sfail(CPP_ERR_CUDA, "server launch: %s", cudaGetErrorString(e));
  } else if ((e = launch_mask_batch(src, n, count, max_tasks, cfg.params, any_geo, st)) !=
                 cudaSuccess ||
             (e = search(L, src, st)) != cudaSuccess ||
             (e = launch_lm_batch_geo(src, n, count, max_T, cfg.params, any_geo, st)) !=
                 cudaSuccess ||
             (e = launch_check_batch(src, count, cfg.params, st)) != cudaSuccess) {
    return sfail(CPP_ERR_CUDA, "server launch: %s", cudaGetErrorString(e));
  }
  // results staging after the table, in table order (stage() may have reordered reqs)
  L->out_off.resize(count);
  size_t o = align256(L->tab_bytes);
  for (int i = 0; i < count; ++i) {
    L->out_off[i] = o;
    o += align256(L->reqs[i]->out_bytes);
  }
  for (int i = 0; i < count; ++i) {
    Request* r = L->reqs[i];
    e = cudaMemcpyAsync(L->tab_h + L->out_off[i], d_arena + r->dev_off + r->o_out, r->out_bytes,
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return sfail(CPP_ERR_CUDA, "server D2H: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(tst, tst_d, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(L->done, st);
  if (e != cudaSuccess) return sfail(CPP_ERR_CUDA, "server D2H: %s", cudaGetErrorString(e));
  return CPP_OK;
}

void cpp_server::retire(Launch* L, cudaError_t e) {
  const int count = (int)L->reqs.size();
  const int32_t* tst = reinterpret_cast<const int32_t*>(
      L->tab_h + align256(sizeof(Req) * count) + align256(sizeof(cpp_robot_t) * count));
  const auto now = Clock::now();
  for (int i = 0; i < count; ++i) {
    Request* r = L->reqs[i];
    if (e != cudaSuccess) {
      darena.release(r->dev_off, r->dev_bytes);
      --resident;
      r->t_done = now;
      r->state = St::Failed;
      r->result = CPP_ERR_CUDA;
      ++stats.failed;
      release_host(r);
      continue;
    }
    r->dev_status = tst[i];
    release_host(r);  // the inputs were copied long before
    const char* res = L->tab_h + L->out_off[i];
    if (r->anytime) {
      anytime_step(r, L->improve, res);
      continue;
    }
    r->own_out.assign(res, res + r->out_bytes);
    darena.release(r->dev_off, r->dev_bytes);
    --resident;
    r->t_done = now;
    r->state = St::Done;
    r->result = tst[i] == 0 ? CPP_OK : (cpp_status)tst[i];
    ++stats.completed;
  }
  darena.release(L->tab_off, L->tab_bytes);
  if (L->tab_pinned) parena.release(L->tab_pin, L->tab_pin_bytes);
  if (L->stream >= 0) stream_busy[L->stream] = false;
}

static void drop_launch(Launch* L) {
  if (L->copied) cudaEventDestroy(L->copied);
  if (L->done) cudaEventDestroy(L->done);
  delete L;
}

void cpp_server::run() {
  cudaSetDevice(cfg.device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // retire finished launches
    for (size_t k = 0; k < inflight.size();) {
      Launch* L = inflight[k];
      const cudaError_t q = cudaEventQuery(L->done);
      if (q == cudaErrorNotReady) { ++k; continue; }
      retire(L, q);
      drop_launch(L);
      inflight.erase(inflight.begin() + k);
      cv_done.notify_all();
    }
    if (stop && inflight.empty() && staged.empty()) break;
    int sidx = -1;
    if ((int)inflight.size() < cfg.max_inflight)
      for (int k = 0; k < (int)streams.size(); ++k)
        if (!stream_busy[k]) { sidx = k; break; }
    // form and stage a launch: when a stream is free, or ahead of time (one
    // launch) when every stream is busy and a full batch is waiting, so its
    // copies overlap the running launches
    bool progressed = false;
    const bool ahead = sidx < 0 && staged.empty() && (int)queue.size() >= cfg.max_batch;
    if (!stop && ((sidx >= 0 && staged.empty()) || ahead) && (!queue.empty() || !improve_q.empty())) {
      Launch* L = new Launch;
      // new plans first; anytime improvement rounds fill the remaining capacity
      bool formed = false;
      if (!queue.empty()) formed = form_batch(L);
      if (!formed && !ahead && !improve_q.empty()) formed = form_improve(L);
      if (formed) {
        cudaEventCreateWithFlags(&L->copied, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
        ++stats.batches;
        if (L->improve) ++stats.improve_batches;
        stats.max_batch_seen = std::max<int32_t>(stats.max_batch_seen, (int32_t)L->reqs.size());
        stats.sum_batch += L->reqs.size();
        lk.unlock();
        const cpp_status st = stage(L);
        lk.lock();
        if (st != CPP_OK) {
          fatal = cpp_last_error();
          retire(L, cudaErrorUnknown);
          drop_launch(L);
          cv_done.notify_all();
        } else {
          staged.push_back(L);
        }
        progressed = true;
      } else {
        delete L;
      }
    }
    // enqueue the oldest staged launch on a free stream
    if (sidx >= 0 && !staged.empty()) {
      Launch* L = staged.front();
      staged.pop_front();
      L->stream = sidx;
      stream_busy[sidx] = true;
      lk.unlock();
      const cpp_status st = enqueue(L);
      lk.lock();
      if (st != CPP_OK) {
        fatal = cpp_last_error();
        retire(L, cudaErrorUnknown);
        drop_launch(L);
        cv_done.notify_all();
      } else {
        inflight.push_back(L);
      }
      progressed = true;
    }
    if (progressed) continue;
    if (inflight.empty() && staged.empty()) {
      cv_work.wait(lk, [&] { return stop || !queue.empty() || !improve_q.empty(); });
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
  // anytime requests between rounds finish with their best so far
  for (Request* r : improve_q) finish(r);
  improve_q.clear();
  // cancel what never ran
  for (Request* r : queue) {
    r->state = St::Cancelled;
    r->result = CPP_ERR_CANCELLED;
    release_host(r);
  }
  queue.clear();
  cv_done.notify_all();
}

extern "C" {

void cpp_server_config_default(cpp_server_config_t* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->device = 0;
  c->max_slots = 1024;
  c->max_batch = 512;
  c->max_inflight = 8;
  c->hbm_budget_bytes = (size_t)40 << 30;
  c->pinned_bytes = (size_t)1 << 30;
  cpp_params_default(&c->params);
  c->latency_requests = 8;
  c->search_budget_ms = 12.0;
}

cpp_status cpp_server_create(const cpp_server_config_t* cfg, cpp_server_t** out) {
  if (!out) return sfail(CPP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return sfail(CPP_ERR_INVALID_ARG, "config is NULL");
  if (cfg->max_slots < 1 || cfg->max_batch < 1 || cfg->max_inflight < 1 || cfg->max_inflight > 32)
    return sfail(CPP_ERR_INVALID_ARG, "max_slots, max_batch >= 1 and max_inflight in [1, 32]");
  if (cfg->latency_requests < 0) return sfail(CPP_ERR_INVALID_ARG, "latency_requests must be >= 0");
  if (!(std::isfinite(cfg->search_budget_ms) && cfg->search_budget_ms >= 0))
    return sfail(CPP_ERR_INVALID_ARG, "search_budget_ms must be finite and >= 0");
  if (cfg->hbm_budget_bytes < 4096) return sfail(CPP_ERR_INVALID_ARG, "hbm_budget_bytes too small");
  const cpp_params_t& P = cfg->params;
  if (P.lm_iters < 0 || P.smooth_rounds < 0 || P.smooth_rounds > 1000 ||
      !(std::isfinite(P.smooth_lambda) && P.smooth_lambda > 0) ||
      !(std::isfinite(P.pen_collide) && P.pen_collide >= 0) ||
      !(std::isfinite(P.coll_margin) && P.coll_margin >= 0) ||
      !(std::isfinite(P.coll_weight) && P.coll_weight >= 0) ||
      (P.dp_objective != CPP_DP_SUM && P.dp_objective != CPP_DP_MINMAX))
    return sfail(CPP_ERR_INVALID_ARG, "invalid params (lm_iters, smooth_rounds, smooth_lambda, "
                                      "dp_objective)");
  cpp_server* s = new (std::nothrow) cpp_server;
  if (!s) return sfail(CPP_ERR_OOM, "host allocation failed");
  s->cfg = *cfg;
  memset(&s->stats, 0, sizeof(s->stats));
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_arena, cfg->hbm_budget_bytes);
  if (e != cudaSuccess) {
    delete s;
    return sfail(e == cudaErrorMemoryAllocation ? CPP_ERR_OOM : CPP_ERR_CUDA,
                 "server device arena: %s", cudaGetErrorString(e));
  }
  s->darena.reset(cfg->hbm_budget_bytes);
  {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, cfg->device) == cudaSuccess && v > 0)
      s->sms = v;
  }
  if (cfg->pinned_bytes) {
    if (cudaHostAlloc(&s->h_pinned, cfg->pinned_bytes, cudaHostAllocDefault) == cudaSuccess)
      s->parena.reset(cfg->pinned_bytes);
    else
      s->h_pinned = nullptr;
  }
  s->streams.resize(cfg->max_inflight);
  s->stream_busy.assign(cfg->max_inflight, false);
  for (auto& st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  s->aux.resize((size_t)cfg->max_inflight * cpp_server::kBuckets);
  s->aux_done.resize(s->aux.size());
  s->fork_ev.resize(cfg->max_inflight);
  for (auto& st : s->aux) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (auto& ev : s->aux_done) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (auto& ev : s->fork_ev) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return CPP_OK;
}

cpp_status cpp_plan_submit(cpp_server_t* s, const cpp_plan_req_t* rq, uint64_t* ticket) {
  if (!s || !rq || !ticket) return sfail(CPP_ERR_INVALID_ARG, "NULL argument");
  if (!rq->robot) return sfail(CPP_ERR_INVALID_ARG, "robot is NULL");
  const cpp_robot_t& rb = *rq->robot;
  if (rb.n < 1 || rb.n > CPP_MAX_JOINTS) return sfail(CPP_ERR_INVALID_ARG, "robot.n out of range");
  for (int j = 0; j < rb.n; ++j)
    if (!std::isfinite(rb.a[j]) || !std::isfinite(rb.d[j]) || !std::isfinite(rb.alpha[j]) ||
        !std::isfinite(rb.theta0[j]) || !(rb.lo[j] <= rb.hi[j]))
      return sfail(CPP_ERR_INVALID_ARG, "robot joint %d malformed", j);
  const int T = rq->T, K = rq->K, Kp = rq->Kp, n = rb.n;
  if (T < 1 || K < 1 || K > 65535 || Kp < K || Kp % 4)
    return sfail(CPP_ERR_INVALID_ARG, "invalid lattice T=%d K=%d Kp=%d", T, K, Kp);
  if (!dp_supported(n, Kp)) return sfail(CPP_ERR_INVALID_ARG, "Kp too large for shared memory");
  if (s->cfg.params.smooth_rounds > 0 && smooth_smem_bytes(T, n) > 227u * 1024u)
    return sfail(CPP_ERR_INVALID_ARG, "smooth_rounds > 0 needs (n + 1) * T * 8 <= 227 KB");
  if (!rq->cand || !rq->targets) return sfail(CPP_ERR_INVALID_ARG, "NULL input");
  for (int i = 0; i < T; ++i) {
    const double* t = rq->targets + 7 * (size_t)i;
    double qn = 0;
    for (int k = 0; k < 7; ++k)
      if (!std::isfinite(t[k])) return sfail(CPP_ERR_INVALID_ARG, "target %d is not finite", i);
    for (int k = 3; k < 7; ++k) qn += t[k] * t[k];
    if (std::fabs(std::sqrt(qn) - 1.0) > 1e-6)
      return sfail(CPP_ERR_INVALID_ARG, "target %d: quaternion norm %.9f is not 1", i, std::sqrt(qn));
  }
  const Layout L = slot_layout(T, Kp, n);
  const size_t table = tab_total(1);
  if (L.total + table > s->cfg.hbm_budget_bytes)
    return sfail(CPP_ERR_BUDGET, "request needs %zu bytes of device memory; the budget is %zu",
                 L.total + table, s->cfg.hbm_budget_bytes);
  std::vector<char> geo;
  if (rq->geometry) {
    geo.resize(geo_bytes());
    char msg[160];
    if (!make_geo(*rq->geometry, n, geo.data(), msg)) return sfail(CPP_ERR_INVALID_ARG, "%s", msg);
  }
  const bool anytime = (rq->flags & CPP_REQ_ANYTIME) != 0;
  if (anytime && (rq->anytime_rounds < 0 || rq->anytime_rounds > 100000))
    return sfail(CPP_ERR_INVALID_ARG, "anytime_rounds outside [0, 100000]");
  if (anytime && smooth_smem_bytes(T, n) > 227u * 1024u)
    return sfail(CPP_ERR_INVALID_ARG, "anytime needs (n + 1) * T * 8 <= 227 KB");
  Request* r = new (std::nothrow) Request;
  if (!r) return sfail(CPP_ERR_OOM, "host allocation failed");
  r->robot = rb;
  r->geo = std::move(geo);
  r->anytime = anytime;
  r->rounds_left = anytime ? rq->anytime_rounds : 0;
  r->T = T; r->K = K; r->Kp = Kp; r->n = n;
  r->dev_bytes = L.total;
  r->o_cand = L.cand; r->o_tgt = L.tgt; r->o_out = L.out; r->o_ws = L.ws;
  r->out_bytes = L.out_bytes; r->o_sel = L.sel; r->o_q = L.q; r->o_err = L.err;
  r->o_rep = L.rep; r->o_best = L.best;
  const size_t cand_b = (size_t)T * n * Kp * sizeof(float), tgt_b = (size_t)T * 7 * sizeof(double);
  const bool borrow = (rq->flags & CPP_REQ_BORROW) != 0;
  const size_t in_b = borrow ? 0 : align256(cand_b) + align256(tgt_b);
  std::unique_lock<std::mutex> lk(s->mu);
  if (borrow) {
    r->cand = rq->cand;
    r->targets = rq->targets;
  } else if (s->h_pinned && s->parena.alloc(in_b, &r->pin_off)) {
    r->pinned = true;
    r->pin_bytes = in_b;
    char* base = s->h_pinned + r->pin_off;
    lk.unlock();
    memcpy(base, rq->cand, cand_b);
    memcpy(base + align256(cand_b), rq->targets, tgt_b);
    lk.lock();
    r->cand = reinterpret_cast<const float*>(base);
    r->targets = reinterpret_cast<const double*>(base + align256(cand_b));
  } else {
    r->own_in.resize(align256(cand_b) + tgt_b);
    memcpy(r->own_in.data(), rq->cand, cand_b);
    memcpy(r->own_in.data() + align256(cand_b), rq->targets, tgt_b);
    r->cand = reinterpret_cast<const float*>(r->own_in.data());
    r->targets = reinterpret_cast<const double*>(r->own_in.data() + align256(cand_b));
  }
  if (s->stop) {
    s->release_host(r);
    delete r;
    return sfail(CPP_ERR_CANCELLED, "server is shutting down");
  }
  r->ticket = s->next_ticket++;
  r->t_submit = Clock::now();
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  ++s->stats.submitted;
  *ticket = r->ticket;
  lk.unlock();
  s->cv_work.notify_one();
  return CPP_OK;
}

static cpp_status collect(cpp_server_t* s, Request* r, cpp_plan_result_t* res) {
  const cpp_status st = r->result;
  if (res) {
    res->latency_ms =
        std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    res->dev_status = r->dev_status;
    res->rounds = r->have_best ? r->best_rounds : r->rounds_done;
    if (r->state == St::Done) {
      const char* o = r->own_out.data();
      if (res->sel) memcpy(res->sel, o + r->o_sel, (size_t)r->T * sizeof(int32_t));
      if (res->q) memcpy(res->q, o + r->o_q, (size_t)r->T * r->n * sizeof(float));
      if (res->pose_err) memcpy(res->pose_err, o + r->o_err, (size_t)r->T * 2 * sizeof(double));
      if (res->report) memcpy(res->report, o + r->o_rep, sizeof(cpp_report_t));
      if (res->best_cost) memcpy(res->best_cost, o + r->o_best, sizeof(float));
    }
  }
  s->release_host(r);
  s->reqs.erase(r->ticket);
  delete r;
  return st;
}

cpp_status cpp_plan_poll(cpp_server_t* s, uint64_t ticket, cpp_plan_result_t* res) {
  if (!s) return sfail(CPP_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(CPP_ERR_NOT_FOUND, "unknown ticket %llu",
                                        (unsigned long long)ticket);
  Request* r = it->second;
  if (r->state == St::Queued || r->state == St::Running || r->state == St::Improving)
    return CPP_PENDING;
  return collect(s, r, res);
}

cpp_status cpp_plan_peek(cpp_server_t* s, uint64_t ticket, cpp_plan_result_t* res) {
  if (!s) return sfail(CPP_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(CPP_ERR_NOT_FOUND, "unknown ticket %llu",
                                        (unsigned long long)ticket);
  Request* r = it->second;
  const char* o = nullptr;
  if (r->have_best) o = r->best_out.data();
  else if (r->state == St::Done) o = r->own_out.data();
  else if (r->state == St::Failed || r->state == St::Cancelled) return r->result;
  else return CPP_PENDING;
  if (res) {
    const bool done = r->state == St::Done || r->state == St::Failed || r->state == St::Cancelled;
    res->latency_ms = std::chrono::duration<double, std::milli>(
                          (done ? r->t_done : Clock::now()) - r->t_submit).count();
    res->dev_status = r->dev_status;
    res->rounds = r->have_best ? r->best_rounds : r->rounds_done;
    if (res->sel) memcpy(res->sel, o + r->o_sel, (size_t)r->T * sizeof(int32_t));
    if (res->q) memcpy(res->q, o + r->o_q, (size_t)r->T * r->n * sizeof(float));
    if (res->pose_err) memcpy(res->pose_err, o + r->o_err, (size_t)r->T * 2 * sizeof(double));
    if (res->report) memcpy(res->report, o + r->o_rep, sizeof(cpp_report_t));
    if (res->best_cost) memcpy(res->best_cost, o + r->o_best, sizeof(float));
  }
  return r->have_best ? CPP_OK : r->result;
}

cpp_status cpp_plan_wait(cpp_server_t* s, uint64_t ticket, cpp_plan_result_t* res,
                         int64_t timeout_us) {
  if (!s) return sfail(CPP_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  for (;;) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(CPP_ERR_NOT_FOUND, "unknown ticket %llu",
                                          (unsigned long long)ticket);
    Request* r = it->second;
    if (r->state != St::Queued && r->state != St::Running && r->state != St::Improving)
      return collect(s, r, res);
    if (timeout_us >= 0 && Clock::now() >= deadline) return CPP_PENDING;
    if (timeout_us < 0) s->cv_done.wait(lk);
    else s->cv_done.wait_until(lk, deadline);
  }
}

cpp_status cpp_plan_cancel(cpp_server_t* s, uint64_t ticket) {
  if (!s) return sfail(CPP_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(CPP_ERR_NOT_FOUND, "unknown ticket");
  Request* r = it->second;
  if (r->anytime && r->state == St::Improving) {  // between rounds: finish with the best
    for (auto q = s->improve_q.begin(); q != s->improve_q.end(); ++q)
      if (*q == r) { s->improve_q.erase(q); break; }
    r->stop_improving = true;
    s->finish(r);
    s->cv_done.notify_all();
    return CPP_OK;
  }
  if (r->anytime && r->state == St::Running) {  // stops after the launch in flight
    r->stop_improving = true;
    return CPP_OK;
  }
  if (r->state != St::Queued) return CPP_PENDING;  // already on the device or finished
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == r) { s->queue.erase(q); break; }
  r->state = St::Cancelled;
  r->result = CPP_ERR_CANCELLED;
  r->t_done = Clock::now();
  ++s->stats.cancelled;
  s->release_host(r);
  return CPP_OK;
}

cpp_status cpp_server_get_stats(cpp_server_t* s, cpp_server_stats_t* out) {
  if (!s || !out) return sfail(CPP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->resident = s->resident;
  out->queued = (int32_t)s->queue.size();
  out->hbm_used = s->darena.used();
  out->hbm_high_water = s->darena.high_water();
  return CPP_OK;
}

void cpp_server_destroy(cpp_server_t* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->reqs) {
    s->release_host(kv.second);
    delete kv.second;
  }
  s->reqs.clear();
  for (auto st : s->streams) cudaStreamDestroy(st);
  for (auto st : s->aux) cudaStreamDestroy(st);
  for (auto ev : s->aux_done) cudaEventDestroy(ev);
  for (auto ev : s->fork_ev) cudaEventDestroy(ev);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->d_arena) cudaFree(s->d_arena);
  if (s->h_pinned) cudaFreeHost(s->h_pinned);
  delete s;
}

}  // extern "C"
