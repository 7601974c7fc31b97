/*
 * cppflow.h -- C ABI of the GB300-native CppFlow planner core.
 *
 * The problem (paper §II, "Problem Specification"): given a target path
 * Y = [y_1 .. y_T] of end-effector poses in SE(3) and, for every waypoint, K
 * candidate joint configurations (the paper draws them from IKFlow, §III-A;
 * here they come from the caller), return a joint trajectory
 * xi = [q_1 .. q_T] whose end effector follows Y within a pose threshold,
 * inside the joint limits and without large joint jumps.
 *
 * Pipeline (each stage is a hand-written sm_103a CUDA kernel):
 *   cpp_mask       FK of every candidate, pose error vs y_i, joint-limit and
 *                  pose masks, additive node costs              (§II, §III-B)
 *   cpp_dp_search  dynamic programme over the T x K x K lattice minimising
 *                  the summed per-step L-inf joint jump + node costs (§III-B)
 *   cpp_lm_refine  Levenberg-Marquardt on the pose residual, one damped n x n
 *                  problem per waypoint, clamped to the limits     (§III-C)
 *   cpp_check      FP64 pose error, limits, jumps, mjac, trajectory length (§II)
 *   cpp_plan       all of the above for one request, back to back on a stream
 *   cpp_plan_batch all of the above for many requests of different T and K in
 *                  one launch per stage
 *   cpp_server_*   continuous-batching request loop (submit / poll)
 *
 * Conventions
 *  - Ownership: the caller owns every buffer. Stage calls take DEVICE pointers
 *    and a cudaStream_t (pass 0 for the legacy default stream) and return as
 *    soon as the work is enqueued; results are valid once the stream reaches
 *    that point. cpp_plan_submit / cpp_plan_poll take HOST buffers.
 *  - Errors: every call returns a cpp_status. Arguments are validated on the
 *    host before anything is enqueued (CPP_ERR_INVALID_ARG, with a message
 *    from cpp_last_error(), which is thread-local). Conditions found on the
 *    device (an infeasible lattice) are written to the caller's int32
 *    dev_status word (may be NULL): kernels only ever raise it, never clear
 *    it, so the caller zeroes it before the first call.
 *  - Layouts: candidates are structure-of-arrays [T][n][Kp] FP32 (k fastest),
 *    Kp >= K, Kp a multiple of 4, lanes k >= K are padding and never chosen.
 *    Targets are [T][7] FP64: position x, y, z (m) then a unit quaternion
 *    w, x, y, z. Joint vectors are [T][n]. Angles are radians.
 *  - Robots: revolute serial chains in standard (distal) DH form,
 *    A_j = Rz(q_j + theta0_j) Tz(d_j) Tx(a_j) Rx(alpha_j), identity base and
 *    tool (the paper names no convention), 1 <= n <= 16.
 */
#ifndef CPPFLOW_H
#define CPPFLOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cpp_stream_t; /* = cudaStream_t */

typedef enum cpp_status {
    CPP_OK = 0,
    CPP_PENDING = 1,          /* cpp_plan_poll: not finished yet */
    CPP_ERR_INVALID_ARG = 2,  /* rejected on the host; nothing enqueued */
    CPP_ERR_INFEASIBLE = 3,   /* every path has infinite cost */
    CPP_ERR_OOM = 4,          /* a device or pinned allocation failed */
    CPP_ERR_BUDGET = 5,       /* the request alone exceeds the server's HBM budget */
    CPP_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    CPP_ERR_CUDA = 7,         /* a CUDA runtime call failed (see cpp_last_error) */
    CPP_ERR_NOT_FOUND = 8,    /* unknown or already collected ticket */
    CPP_ERR_CANCELLED = 9     /* the request was cancelled before it ran */
} cpp_status;

#define CPP_MAX_JOINTS 16

/* Mask bits written by cpp_mask (one byte per candidate). */
#define CPP_MASK_OUT 1u       /* some joint outside its limits (§II "Joint limits") */
#define CPP_MASK_NEAR 2u      /* some joint within near_margin of a limit (§III-B) */
#define CPP_MASK_POSE 4u      /* pose error above tau_pos or tau_rot (§II "Pose error") */
#define CPP_MASK_NONFINITE 8u /* some joint value is NaN or inf: cost +inf, no other bit */
#define CPP_MASK_PAD 16u      /* padding lane k >= K: cost +inf */
#define CPP_MASK_COLLIDE 32u  /* a capsule pair or a capsule and a box overlap (§III-B, with a
                                 collision model only; cost + pen_collide) */

/* Collision model of a request (§III-B collision cost, §III-C capsule and cuboid
 * distances): the robot as capsules (segment + radius) fixed to its DH frames
 * (frame 0 = base, frame j = the frame after joint j), the self-collision pairs
 * to test, and cuboid obstacles; every capsule is tested against every box.
 * Clearance of a pair = segment distance - r_u - r_v; of a capsule and a box =
 * segment-box distance - r_u; a candidate collides when its smallest clearance
 * is negative. Host struct; the calls below copy it. */
#define CPP_MAX_CAPSULES 12
#define CPP_MAX_PAIRS 64
#define CPP_MAX_BOXES 8
typedef struct cpp_capsule {
    int32_t frame;            /* 0..n */
    int32_t reserved;
    double a[3], b[3];        /* segment end points in the frame (m) */
    double radius;            /* >= 0 (m) */
} cpp_capsule_t;
typedef struct cpp_cuboid {
    double R[9], p[3];        /* box frame -> world, row-major: x_w = R x_b + p */
    double half[3];           /* half extents >= 0: the box is [-half, half] in its frame */
} cpp_cuboid_t;
typedef struct cpp_geometry {
    int32_t n_caps, n_pairs, n_boxes, reserved;
    cpp_capsule_t caps[CPP_MAX_CAPSULES];
    int32_t pairs[CPP_MAX_PAIRS][2];   /* capsule indices, u != v */
    cpp_cuboid_t boxes[CPP_MAX_BOXES];
} cpp_geometry_t;

typedef struct cpp_robot {
    int32_t n;                      /* joints */
    int32_t reserved;
    double a[CPP_MAX_JOINTS];       /* link length (m) */
    double d[CPP_MAX_JOINTS];       /* link offset (m) */
    double alpha[CPP_MAX_JOINTS];   /* link twist (rad) */
    double theta0[CPP_MAX_JOINTS];  /* joint offset (rad) */
    double lo[CPP_MAX_JOINTS];      /* lower limit (rad) */
    double hi[CPP_MAX_JOINTS];      /* upper limit (rad) */
} cpp_robot_t;

typedef struct cpp_params {
    double tau_pos;      /* pose-valid position threshold, m (default 1e-3, Table I) */
    double tau_rot;      /* pose-valid rotation threshold, rad (default 0.1 deg, §II) */
    double near_margin;  /* near-limit band, rad (default 1.5 deg, §III-B) */
    double pen_limit;    /* node cost for out-of / near-limit configs (default 10, §III-B) */
    double pen_pose;     /* node cost for pose-invalid configs (default 100) */
    double jump_max;     /* discontinuity bound per step, rad (default 7 deg, §II) */
    double lambda0;      /* initial LM damping (default 1e-3) */
    double lambda_up;    /* damping factor after a rejected step (default 10) */
    double lambda_down;  /* damping divisor after an accepted step (default 10) */
    double lambda_min;   /* default 1e-12 */
    double lambda_max;   /* default 1e12 */
    double freeze_step;  /* a waypoint stops when max|delta| < this (default 1e-10) */
    double freeze_cost;  /* a waypoint stops when F = |e|^2/2 < this (default 1e-13: |e| ~ 4.5e-7,
                            the resolution of FP32 forward kinematics) */
    int32_t lm_iters;    /* LM iterations per waypoint (default 20) */
    uint32_t free_mask;  /* bit j set: LM may move joint j (default all) */
    int32_t lm_fp64;     /* 0: FP32 FK/Jacobian + FP64 normal equations and Cholesky;
                            1: everything in FP64 (for near-singular chains) */
    int32_t dp_objective; /* CPP_DP_SUM (default) or CPP_DP_MINMAX, see cpp_dp_search_ex */
    int32_t smooth_rounds; /* §III-C non-stationary objective: trajectory-length steps
                              alternated with pose phases (default 0: pose only), see
                              cpp_smooth_step; at most 1000 */
    int32_t reserved_;
    double smooth_lambda;  /* damping of the trajectory-length step (default 1; > 0) */
    double pen_collide;    /* node cost of a colliding candidate (default 100, §III-B) */
    double coll_margin;    /* collision rows of the trajectory-length step: active where the
                              clearance is below this (m, default 0.02, >= 0) */
    double coll_weight;    /* their weight w: residual w (coll_margin - clearance) (default 1) */
} cpp_params_t;

#define CPP_DP_SUM 0     /* minimise the summed per-step L-inf joint jump */
#define CPP_DP_MINMAX 1  /* the paper's objective: minimise the largest per-step jump (mjac) */

/* Trajectory report of cpp_check (device or host struct, FP64). */
typedef struct cpp_report {
    double max_pos;        /* worst waypoint position error (m) */
    double max_rot;        /* worst waypoint rotation error (rad) */
    double mjac;           /* max over steps and joints of |dq| (§III-B) */
    double sum_linf;       /* sum over steps of the per-step L-inf jump */
    double traj_len;       /* sum over steps and joints of |dq| (§II) */
    int32_t n_pose_fail;   /* waypoints with pos > tau_pos or rot > tau_rot */
    int32_t n_limit_fail;  /* waypoints with a joint outside [lo, hi] */
    int32_t n_jump_fail;   /* steps with an L-inf jump > jump_max (§II) */
    int32_t valid;         /* 1 when every check passes */
} cpp_report_t;

/* ------------------------------------------------------------------ misc */
const char* cpp_last_error(void);          /* thread-local message of the last failure */
const char* cpp_status_string(int status);
int32_t cpp_version(void);                 /* major * 10000 + minor * 100 + patch */
void cpp_params_default(cpp_params_t* p);  /* fills the defaults listed above */
/* Diagnostic (not in the paper): a bounded device wait that nothing completes.
 * One thread waits up to limit_ns (1e3 .. 1e10) on an mbarrier that never
 * completes, with the CTA-scope (cluster_scope = 0) or the cluster-scope
 * (cluster_scope = 1) bounded wait that the search kernels use, and records
 * CPP_ERR_TIMEOUT in *dev_status (device int32) when the limit runs out: a
 * stuck wait ends with a status the host reads, the context stays usable.
 * Asynchronous on `stream`. INVALID_ARG for a limit outside the range or a
 * NULL status. */
cpp_status cpp_wait_selftest(int64_t limit_ns, int32_t cluster_scope, int32_t* dev_status,
                             cpp_stream_t stream);

/* ------------------------------------------------------------------ FK (§II)
 * FK(q): R^n -> SE(3) for N configurations in FP32.
 * q: [n][N] SoA (joint-major), R: [9][N] row-major rotation entries, p: [3][N].
 * INVALID_ARG if N < 0 or the robot is malformed. */
cpp_status cpp_fk_batch(const cpp_robot_t* robot, const float* q, int64_t N, float* R,
                        float* p, cpp_stream_t stream);

/* FP64 FK to poses: q [N][n] FP64 -> pose [N][7] (x, y, z, qw, qx, qy, qz, with qw >= 0). */
cpp_status cpp_fk_pose_f64(const cpp_robot_t* robot, const double* q, int64_t N,
                           double* pose, cpp_stream_t stream);

/* ------------------------------------------------------------------ masking (§II, §III-B)
 * Per candidate (i, k): FP32 FK, position error |p - p_t|, rotation error =
 * geodesic angle of R_t^T R (§II "Pose error"), and
 *   NONFINITE (cost +inf), OUT / NEAR against the FP32-rounded limits lo, hi,
 *   lo + near_margin, hi - near_margin (each formed in FP64, rounded once),
 *   POSE (pos > tau_pos or rot > tau_rot, both compared in FP32),
 *   pen = pen_limit * [OUT or NEAR] + pen_pose * [POSE]     (§III-B).
 * cand [T][n][Kp] FP32, targets [T][7] FP64 -> mask [T][Kp] u8, pen [T][Kp] FP32,
 * err [T][Kp][2] FP32 (position m, rotation rad; NaN on padding) or NULL.
 * INVALID_ARG: T < 1, K < 1, Kp < K, Kp % 4 != 0, n mismatch, NULL buffers. */
cpp_status cpp_mask(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                    const double* targets, int32_t T, int32_t K, int32_t Kp, uint8_t* mask,
                    float* pen, float* err, int32_t* dev_status, cpp_stream_t stream);

/* cpp_mask with the collision model `geometry` (host pointer, copied; NULL =
 * none): COLLIDE bit and + pen_collide per colliding candidate (the node's costs
 * are summed in FP64 in the order limit, pose, collision and rounded once).
 * clearance [T][Kp] FP32 (or NULL) receives the smallest clearance of every
 * candidate (+inf without a model, NaN on padding and non-finite lanes). Distances
 * are solved in FP32 (errors ~1e-6 m). INVALID_ARG also for a model with counts
 * above the limits, frames above n, pair indices out of range or equal,
 * non-finite values, negative radii or half extents. */
cpp_status cpp_mask_geo(const cpp_robot_t* robot, const cpp_params_t* params,
                        const cpp_geometry_t* geometry, const float* cand,
                        const double* targets, int32_t T, int32_t K, int32_t Kp, uint8_t* mask,
                        float* pen, float* err, float* clearance, int32_t* dev_status,
                        cpp_stream_t stream);

/* cpp_mask on the candidate lanes [k_begin, K) only (k_begin a multiple of 4); the
 * lanes below k_begin keep the mask and cost they already have. This is how a
 * re-search reuses a resident lattice: allocate Kp for the largest K expected,
 * mask and search the first K0 lanes, and when the search path's mjac is too
 * large (§III-B: 12 deg) write more candidates into lanes [K0, K1), mask just
 * those, and search again with K = K1; as in §III-B, the checks already made
 * on the first candidates are kept, not redone. */
cpp_status cpp_mask_range(const cpp_robot_t* robot, const cpp_params_t* params,
                          const float* cand, const double* targets, int32_t T, int32_t K,
                          int32_t Kp, int32_t k_begin, uint8_t* mask, float* pen, float* err,
                          int32_t* dev_status, cpp_stream_t stream);

/* ------------------------------------------------------------------ search (§III-B)
 * Dynamic programme over the layered graph whose nodes are the K candidates of
 * each waypoint and whose edges join every node of step i to every node of
 * step i+1. Node costs enter relative to the cheapest node of their waypoint
 * (r_i = pen_i - min_k pen_i; a per-waypoint constant changes no path's rank):
 *   C_0 = r_0;  C_{i+1}[k'] = min_k (C_i[k] + max_j |q_{i+1,k',j} - q_{i,k,j}|) + r_{i+1}[k']
 * in FP32 with one rounding per operation, ties to the lowest k, then
 * backtracking from the lowest argmin of C_{T-1}.
 * Outputs: sel [T] int32 (chosen k per waypoint), best_cost [1] FP32 (min of
 * C_{T-1}), q_seed [T][n] FP32 (the chosen candidates) or NULL.
 * workspace: device scratch of at least cpp_dp_workspace_size(T, Kp) bytes,
 * 256-byte aligned, owned by the caller, not read before it is written.
 * dev_status is raised to CPP_ERR_INFEASIBLE when min C_{T-1} is +inf.
 * INVALID_ARG: T < 1, K < 1, K > 65535, Kp < K, Kp % 4 != 0, n < 1, n > 16,
 * workspace too small or misaligned. */
size_t cpp_dp_workspace_size(int32_t T, int32_t Kp);

/* The search with a choice of objective (§III-B). CPP_DP_SUM is cpp_dp_search.
 * CPP_DP_MINMAX is the paper's own cost: a node costs the smallest mjac that any
 * path through it can reach. C_0 = r_0, C_{i+1}[k'] = max(min_k max(C_i[k], d(k, k')), r_{i+1}[k']),
 * so a path costs the larger of its largest per-step L-inf jump and its largest
 * relative node cost (a near-limit cost of 10 outweighs any revolute jump); max
 * and min are exact, so it involves no rounding. search_mjac [1] FP32 (or NULL)
 * receives the mjac of the selected path, max over steps and joints of |dq|, for
 * the paper's re-search test (more candidates when it exceeds 12 deg). Other
 * arguments as cpp_dp_search; INVALID_ARG for another objective. */
cpp_status cpp_dp_search_ex(const float* cand, const float* pen, int32_t T, int32_t K,
                            int32_t Kp, int32_t n, int32_t objective, void* workspace,
                            size_t ws_bytes, int32_t* sel, float* best_cost, float* q_seed,
                            float* search_mjac, int32_t* dev_status, cpp_stream_t stream);
cpp_status cpp_dp_search(const float* cand, const float* pen, int32_t T, int32_t K,
                         int32_t Kp, int32_t n, void* workspace, size_t ws_bytes,
                         int32_t* sel, float* best_cost, float* q_seed, int32_t* dev_status,
                         cpp_stream_t stream);

/* ------------------------------------------------------------------ search without allocation
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory when they plan: real-time control loops that
 * forbid allocation after start-up (an allocation can block for an unbounded
 * time), and plug-ins whose host application owns every device allocation. It
 * computes exactly what cpp_dp_search computes, but
 * its scratch (layer minima, backpointers, final costs) lives in one
 * file-scope device array of CPP_DP_STATIC_SCRATCH_BYTES inside the library.
 * That array is reserved on every GPU that loads the library and held until the
 * process exits; the call itself allocates nothing (no cudaMalloc, no cudaFree,
 * no allocating library routine). The caller still passes inputs and outputs.
 * Limit: scratch = align256(4T) + align256(2 T Kb) + align256(4 Kp) bytes with
 * Kb = Kp rounded up to 8 -- e.g. T = 2000, Kp = 1024 fits, T = 2000, Kp = 2048
 * does not; larger lattices are rejected with CPP_ERR_INVALID_ARG and a message
 * (use cpp_dp_search with a caller workspace for them).
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture. Every call uses the same array and leaves its
 * contents behind, so calls that overlap on the GPU (other streams, other host
 * threads) race with each other. Each call writes every scratch word it reads,
 * so nothing needs clearing between calls (after a CPP_ERR_TIMEOUT the unfinished
 * rows keep older values; the backtracking clamps what it reads from them to
 * [0, K)). The cached address does not survive a device reset (cudaDeviceReset
 * or a primary-context reset): do not call this entry point on a device after
 * resetting it. Arguments, layouts and errors otherwise as cpp_dp_search. */
#define CPP_DP_STATIC_SCRATCH_BYTES (8u << 20)
cpp_status cpp_dp_search_static(const float* cand, const float* pen, int32_t T, int32_t K,
                                int32_t Kp, int32_t n, int32_t* sel, float* best_cost,
                                float* q_seed, int32_t* dev_status, cpp_stream_t stream);

/* ------------------------------------------------------------------ LM (§III-C)
 * Per waypoint independently (the pose residual of waypoint i depends on q_i
 * only, so J is block diagonal): residual e = [p_t - p(q); log(R_t R(q)^T)]
 * (world-frame rotation vector), geometric Jacobian J (6 x n), step
 * (J^T J + lambda I) delta = J^T e solved by FP64 Cholesky, q' = clamp(q + delta,
 * lo, hi); accept when F(q') < F(q) (lambda /= lambda_down) else reject
 * (lambda *= lambda_up). lm_iters iterations; a waypoint stops early when
 * F < freeze_cost or max|delta| < freeze_step. Joints outside free_mask stay.
 * q_in, q_out [T][n] FP32 (may alias), targets [T][7] FP64,
 * pose_err [T][2] FP64 (FP64 position / rotation error of q_out) or NULL. */
cpp_status cpp_lm_refine(const cpp_robot_t* robot, const cpp_params_t* params,
                         const float* q_in, const double* targets, int32_t T, float* q_out,
                         double* pose_err, int32_t* dev_status, cpp_stream_t stream);

/* §III-C non-stationary objective. The paper alternates pose-only LM phases with
 * single steps on the trajectory-length residual r_diff = [q_{i+1} - q_i]
 * (differences of consecutive configurations; its collision rows are not
 * built), taking such a step only once every waypoint is within tau_pos /
 * tau_rot. cpp_smooth_step is one such step on q [T][n] FP32 in place: if the
 * FP64 FK of every waypoint is within tau it applies
 *   delta = -(J^T J + smooth_lambda I)^{-1} J^T r_diff,  q = clamp(q + delta, lo, hi),
 * solved in FP64 (J^T J is block tridiagonal with blocks that are multiples of
 * I, so the block Thomas recursion splits into one scalar recursion per joint),
 * else it leaves q unchanged. With params->smooth_rounds = R > 0, cpp_lm_refine
 * (and cpp_plan, batches, the server) run a pose phase, then R times this step
 * followed by another pose phase (starting from the previous phase's q_out);
 * pose_err then belongs to the last phase. Limit: (n + 1) * T * 8 bytes of shared
 * memory per request, at most 227 KB (T <= 3632 at n = 7, 2905 at n = 9);
 * INVALID_ARG beyond it. */
cpp_status cpp_smooth_step(const cpp_robot_t* robot, const cpp_params_t* params, float* q,
                           const double* targets, int32_t T, int32_t* dev_status,
                           cpp_stream_t stream);

/* The trajectory-length step with the collision rows of r_diff (§III-C): for
 * every listed pair and capsule-box combination with clearance d below
 * coll_margin, a residual coll_weight * (coll_margin - d) with its gradient
 * (closest-point direction times the point Jacobians). Each row touches one
 * waypoint, so the normal equations stay block tridiagonal with full n x n
 * diagonal blocks; the block Thomas recursion runs in FP64 (rows and gradients
 * in FP32). Gate, clamp and in-place update as cpp_smooth_step. geometry: host
 * pointer (copied); NULL gives cpp_smooth_step. workspace: device scratch of
 * cpp_smooth_workspace_size(T, n) bytes, 256-byte aligned. In cpp_plan_geo,
 * batches and the server a request with a collision model takes these steps
 * whenever smooth_rounds > 0. */
size_t cpp_smooth_workspace_size(int32_t T, int32_t n);
cpp_status cpp_smooth_step_geo(const cpp_robot_t* robot, const cpp_params_t* params,
                               const cpp_geometry_t* geometry, float* q, const double* targets,
                               int32_t T, void* workspace, size_t ws_bytes, int32_t* dev_status,
                               cpp_stream_t stream);

/* ------------------------------------------------------------------ check (§II)
 * FP64 FK of q [T][n] FP32 -> pose_err [T][2] FP64 (or NULL) and a report
 * (device pointer to one cpp_report_t): worst errors, mjac, summed L-inf jump,
 * trajectory length, counts of pose / limit / jump (> jump_max) failures. */
cpp_status cpp_check(const cpp_robot_t* robot, const cpp_params_t* params, const float* q,
                     const double* targets, int32_t T, double* pose_err,
                     cpp_report_t* report, cpp_stream_t stream);

/* ------------------------------------------------------------------ one request
 * mask -> search -> LM -> check on one stream (the plain per-request path).
 * Device buffers: cand, targets in; sel [T], q_out [T][n], pose_err [T][2],
 * report [1], best_cost [1] out; dev_status as above; workspace of
 * cpp_plan_workspace_size(T, K, Kp, n) bytes, 256-byte aligned. */
size_t cpp_plan_workspace_size(int32_t T, int32_t K, int32_t Kp, int32_t n);
cpp_status cpp_plan(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                    const double* targets, int32_t T, int32_t K, int32_t Kp,
                    void* workspace, size_t ws_bytes, int32_t* sel, float* best_cost,
                    float* q_out, double* pose_err, cpp_report_t* report,
                    int32_t* dev_status, cpp_stream_t stream);
/* cpp_plan with a collision model (host pointer, copied; NULL = none): the mask
 * adds the collision cost of §III-B, so the search avoids colliding candidates. */
cpp_status cpp_plan_geo(const cpp_robot_t* robot, const cpp_params_t* params,
                        const cpp_geometry_t* geometry, const float* cand,
                        const double* targets, int32_t T, int32_t K, int32_t Kp,
                        void* workspace, size_t ws_bytes, int32_t* sel, float* best_cost,
                        float* q_out, double* pose_err, cpp_report_t* report,
                        int32_t* dev_status, cpp_stream_t stream);

/* The plain per-request path from HOST memory: copies cand [T][n][Kp] FP32 and
 * targets [T][7] FP64 from host buffers to the device, runs cpp_plan on `stream`,
 * copies sel [T], best_cost [1], q_out [T][n], pose_err [T][2] and report [1] back
 * into host buffers (each may be NULL) and waits for the stream. This is the path a
 * single client with host data takes, one request at a time. Pinned host buffers
 * make the copies direct DMA; pageable ones work (slower). workspace: DEVICE
 * scratch of cpp_plan_host_workspace_size(T, K, Kp, n) bytes, 256-byte aligned
 * (the device copies of inputs and outputs, a status word and the plan's scratch).
 * Returns INVALID_ARG as cpp_plan, CUDA on a failed copy or launch, otherwise the
 * plan's device status after the wait (OK, INFEASIBLE or TIMEOUT). */
size_t cpp_plan_host_workspace_size(int32_t T, int32_t K, int32_t Kp, int32_t n);
cpp_status cpp_plan_host(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                         const double* targets, int32_t T, int32_t K, int32_t Kp,
                         void* workspace, size_t ws_bytes, int32_t* sel, float* best_cost,
                         float* q_out, double* pose_err, cpp_report_t* report,
                         cpp_stream_t stream);

/* ------------------------------------------------------------------ diagnostics (not in the paper)
 * Arithmetic throughput probe, the measured peak the kernels are compared with.
 * CPP_PROBE_FP32: every thread runs 8 independent chains x = max(x + a, b), one
 * FP32 add and one FP32 max per link (the two operations of the search's inner
 * loop, each one FP32 lane operation); CPP_PROBE_FP64: 8 chains x = fma(x, a, b)
 * in FP64 (2 flops per link). One launch of blocks_per_sm * SMs blocks of 256
 * threads, `iters` links per chain, on `stream`; time it with events on that
 * stream. *lane_ops (host) receives the operations one launch performs (FP32 lane
 * operations, or FP64 flops). sink: device buffer of one double that keeps the
 * chains from being removed (its value is meaningless). INVALID_ARG for another
 * kind, blocks_per_sm outside [1, 8], iters outside [1, 1e9]. */
#define CPP_PROBE_FP32 0
#define CPP_PROBE_FP64 1
cpp_status cpp_peak_probe(int32_t kind, int32_t blocks_per_sm, int64_t iters, double* sink,
                          double* lane_ops, cpp_stream_t stream);

/* Work counters of the LM stage (S5), accumulated over every LM launch of the
 * process on the current device: waypoints refined and LM iterations that built
 * and solved a damped system (accepted or rejected; a waypoint stops early at
 * F < freeze_cost or max|delta| < freeze_step). cpp_counters_reset zeroes them on
 * `stream`; cpp_counters_read copies them to the host once every earlier launch has
 * completed (synchronize the streams that ran them first). */
typedef struct cpp_counters {
    uint64_t lm_waypoints;
    uint64_t lm_iterations;
} cpp_counters_t;
cpp_status cpp_counters_reset(cpp_stream_t stream);
cpp_status cpp_counters_read(cpp_counters_t* out);

/* FP64 geometric Jacobian in the world frame (§III-C, the matrix of the LM step):
 * q [N][n] FP64 -> J [N][6][n] FP64, rows 0..2 the linear part z_{j-1} x (p_e - o_{j-1}),
 * rows 3..5 the angular part z_{j-1} (frame 0 = base). For conditioning reports
 * (the smallest singular value along a path). INVALID_ARG if N < 0 or the robot
 * is malformed. */
cpp_status cpp_jacobian_f64(const cpp_robot_t* robot, const double* q, int64_t N, double* J,
                            cpp_stream_t stream);

/* ------------------------------------------------------------------ cpf-BatchOpt
 * The paper's fastest planner variant (§III, in its commented text): refine the
 * smoothest of the K candidate trajectories directly instead of searching. Lane
 * k across the waypoints is one candidate trajectory; its smoothness is its mjac,
 * max over steps and joints of |q_{i+1,k,j} - q_{i,k,j}| in FP32 (+inf if it holds
 * a non-finite value). The `lanes` smoothest (ascending mjac, lowest index first
 * among equals; the paper uses 5) are refined as separate trajectories by the LM
 * of cpp_lm_refine (with params->smooth_rounds alternation) and checked as by
 * cpp_check. Device buffers out: lane_sel [lanes] (lane indices, smoothest
 * first), lane_mjac [lanes], q_out [lanes][T][n], pose_err [lanes][T][2] (or
 * NULL), reports [lanes], best [1] (position in lane_sel of the first valid plan,
 * -1 if none). Workspace: cpp_batch_opt_workspace_size(T, K, n, lanes) bytes,
 * 256-byte aligned. INVALID_ARG: lanes outside [1, K], lattice and params as
 * cpp_plan. Meaningful on lane-coherent candidates (a generative model's plans);
 * on independently drawn candidates the search (cpp_plan) is the planner. */
size_t cpp_batch_opt_workspace_size(int32_t T, int32_t K, int32_t n, int32_t lanes);
cpp_status cpp_batch_opt(const cpp_robot_t* robot, const cpp_params_t* params, const float* cand,
                         const double* targets, int32_t T, int32_t K, int32_t Kp, int32_t lanes,
                         void* workspace, size_t ws_bytes, int32_t* lane_sel, float* lane_mjac,
                         float* q_out, double* pose_err, cpp_report_t* reports, int32_t* best,
                         int32_t* dev_status, cpp_stream_t stream);

/* ------------------------------------------------------------------ many requests
 * One launch per stage for `count` requests of different T, K, Kp (same params).
 * Each descriptor holds DEVICE pointers; robots are read from the host array
 * `robots` (copied into the workspace). The workspace must hold
 * cpp_plan_batch_workspace_size(descs, count) bytes. dev_status [count] int32. */
typedef struct cpp_plan_desc {
    int32_t T, K, Kp, robot;   /* robot = index into the robots array */
    const float* cand;         /* [T][n][Kp] */
    const double* targets;     /* [T][7] */
    int32_t* sel;              /* [T] */
    float* q_out;              /* [T][n] */
    double* pose_err;          /* [T][2] */
    cpp_report_t* report;      /* [1] */
    float* best_cost;          /* [1] */
    const cpp_geometry_t* geometry;  /* host pointer, copied at batch creation; NULL = none */
} cpp_plan_desc_t;

size_t cpp_plan_batch_workspace_size(const cpp_plan_desc_t* descs, int32_t count,
                                     const cpp_robot_t* robots, int32_t n_robots);
cpp_status cpp_plan_batch(const cpp_robot_t* robots, int32_t n_robots,
                          const cpp_params_t* params, const cpp_plan_desc_t* descs,
                          int32_t count, void* workspace, size_t ws_bytes,
                          int32_t* dev_status, cpp_stream_t stream);

/* ------------------------------------------------------------------ prepared batches
 * cpp_batch_create validates a batch exactly like cpp_plan_batch, copies its
 * request table into the workspace (enqueued on `stream`; the host arrays may be
 * freed on return) and returns a host handle. cpp_batch_run then enqueues any
 * subset of the stages below, in pipeline order, on any stream; it launches
 * kernels only, so it can be repeated, timed stage by stage, or captured into a
 * CUDA graph. The workspace and every descriptor buffer must stay valid until
 * the handle is destroyed. cpp_plan_batch = create + run(CPP_STAGE_ALL) + destroy. */
#define CPP_STAGE_MASK 1u        /* S1+S2: FK, pose error, masks, node costs */
#define CPP_STAGE_LAYER_MIN 2u   /* per-waypoint cheapest node cost */
#define CPP_STAGE_DP_FORWARD 4u  /* S3: the min-plus sweep over the T x K x K lattice */
#define CPP_STAGE_BACKTRACK 8u   /* S4: final argmin, backtracking, seed gather */
#define CPP_STAGE_LM 16u         /* S5: Levenberg-Marquardt */
#define CPP_STAGE_CHECK 32u      /* S6: FP64 check and report */
#define CPP_STAGE_ALL 63u

typedef struct cpp_batch cpp_batch_t;
cpp_status cpp_batch_create(const cpp_robot_t* robots, int32_t n_robots,
                            const cpp_params_t* params, const cpp_plan_desc_t* descs,
                            int32_t count, void* workspace, size_t ws_bytes,
                            int32_t* dev_status, cpp_stream_t stream, cpp_batch_t** out);
cpp_status cpp_batch_run(cpp_batch_t* batch, uint32_t stages, cpp_stream_t stream);
/* Number of kernel launches cpp_batch_run(batch, stages, ...) enqueues. */
int32_t cpp_batch_launches(const cpp_batch_t* batch, uint32_t stages);
void cpp_batch_destroy(cpp_batch_t* batch);

/* Scheduling of the search stage (S3) for uneven batches. The search is serial
 * in T, so a batch's search time is at least that of its longest request on
 * whatever runs it. A request whose lattice ((T - 1) * Kp^2 edges) exceeds
 * alpha times the mean load of a CTA slot (total edges / (2 * SMs)) is "heavy"
 * and runs as a thread-block cluster (one launch per cluster size, each on an
 * internal stream forked from and joined back into the caller's stream by
 * events); the others run one CTA per request, longest first. alpha = 0 sends
 * every request to the one-launch form (clusters only when one wave of them
 * covers the whole batch). cpp_batch_create applies alpha = 2.
 *
 * The cluster form gives each CTA cands_per_cta successor candidates of a
 * waypoint (32, 64 or 128: the CTAs exchange whole records [-q, C] every step;
 * 256 or 512: the wide form, in which every CTA stages each layer's joint values
 * itself and only the node costs C cross the cluster; 0 = 64 up to Kp = 512 and
 * 128 above, as long as the cluster has 2..8 CTAs; an explicit 32 or 64 also
 * allows the non-portable sizes of 9..16 CTAs): fewer per CTA shorten a long
 * request's latency, more raise the edge rate per SM (fewer exchanges and waits
 * per candidate). The automatic form
 * (alpha = 0, single-request calls, the server) takes the smallest tile (32 per
 * CTA up to Kp = 512, 64 above, clusters of up to 16 CTAs) when the device holds
 * all the requests' clusters at once with one CTA per SM.
 *
 * cpp_batch_set_split sets alpha (>= 0) and cands_per_cta and uploads the new
 * schedule on `stream`. cpp_batch_tune picks both by measurement on the batch
 * itself: it enqueues the mask and node-cost stages, then times the forward
 * sweep (CUDA events, best of two runs after one warm-up) for alpha = 0 and,
 * for each cands_per_cta in {64, 128, 256, 512} and each smallest clustered Kp (any, or
 * each Kp of the batch above its smallest), a ladder of alpha values from 8 down
 * to 1e-9 (every cluster-capable request heavy), skipping values that give the
 * same split, and keeps the fastest; then it times the mask stage the same way for
 * 1, 2, 4, 8 and 16 tasks per warp and keeps the fastest. With a
 * non-NULL table_path the choice is looked up first under a key of the batch's
 * shape (joints, objective, request count and longest T in powers of two,
 * cluster sizes present, skew of the largest lattice over the mean, SM count;
 * plain text, one "key alpha cands_per_cta ms mask_tasks_per_warp min_kp" line
 * per entry, the last entry wins; missing trailing fields mean the defaults)
 * and, when
 * missing, appended after tuning. The call synchronizes `stream`; the batch's
 * outputs are undefined until its next cpp_batch_run. A new schedule drops any
 * captured graph. */
typedef struct cpp_tune_result {
    double alpha;            /* heavy threshold in use */
    int32_t cands_per_cta;   /* successor candidates per CTA of the cluster form (0: default) */
    int32_t heavy;           /* requests run as clusters */
    int32_t forward_launches;/* launches of the forward sweep */
    int32_t timed;           /* configurations timed (0 when taken from the table) */
    int32_t from_table;      /* 1: alpha came from the tuning table */
    float dp_ms;             /* forward sweep time of the choice (-1 from the table) */
    float dp_ms_unsplit;     /* forward sweep time with alpha = 0 (-1 from the table) */
    int32_t mask_tasks_per_warp; /* 128-candidate tasks per warp of the mask stage in use */
    float mask_ms;           /* mask stage time of the choice (-1 from the table) */
    float mask_ms_default;   /* mask stage time with 4 tasks per warp (-1 from the table) */
    int32_t cluster_min_kp;  /* smallest Kp allowed to run as a cluster (0: any) */
    float budget_ms;         /* > 0: per-request forms within this time (cpp_batch_set_budget);
                                0: the alpha split */
} cpp_tune_result_t;
cpp_status cpp_batch_set_split(cpp_batch_t* batch, double alpha, int32_t cands_per_cta,
                               cpp_stream_t stream);
/* The search schedule of the serving loop under load: each request runs in the
 * form with the highest edge rate per SM whose estimated search time is at most
 * budget_ms (one CTA, clusters of 512, 256, 128 or 64 successors per CTA; rates
 * measured on GB300, stated in the library source), else in the fastest of them.
 * Cluster requests are grouped by tile and cluster size, one launch per group.
 * Results are identical in every schedule. INVALID_ARG if budget_ms <= 0 or the
 * choice makes more than 8 cluster groups; cpp_batch_set_split returns to the
 * alpha split. Drops any captured graph. */
cpp_status cpp_batch_set_budget(cpp_batch_t* batch, double budget_ms, cpp_stream_t stream);
/* Smallest Kp that may run as a cluster (0: any): heavier requests of smaller K
 * then stay one CTA each, longest first. Re-applies the current alpha and
 * cands_per_cta and uploads the schedule on `stream`. INVALID_ARG if negative. */
cpp_status cpp_batch_set_cluster_min_kp(cpp_batch_t* batch, int32_t min_kp, cpp_stream_t stream);
/* Tasks per warp of the mask stage (S1+S2): a task is one waypoint and 128
 * candidates, so a warp covers tasks_per_warp * 128 / Kp waypoints of a request
 * (0: the default, 4). Results do not depend on it. INVALID_ARG outside [0, 64]. */
cpp_status cpp_batch_set_mask_tasks(cpp_batch_t* batch, int32_t tasks_per_warp);
cpp_status cpp_batch_tune(cpp_batch_t* batch, const char* table_path, cpp_stream_t stream,
                          cpp_tune_result_t* result);

/* CUDA graph of a prepared batch: cpp_batch_capture records the launches of
 * cpp_batch_run(batch, stages) on `stream` (a created stream, not the legacy
 * default stream; the batch's internal streams join the capture through its
 * events) into an executable graph held by the batch, replacing any earlier
 * one; nothing runs during the capture. cpp_batch_replay launches that graph on
 * any stream: the same kernels, arguments and buffers, one host call. */
cpp_status cpp_batch_capture(cpp_batch_t* batch, uint32_t stages, cpp_stream_t stream);
cpp_status cpp_batch_replay(cpp_batch_t* batch, cpp_stream_t stream);

/* ------------------------------------------------------------------ serving
 * A continuous-batching request loop (not in the paper). Clients submit plans
 * with HOST buffers from any thread; a worker thread admits queued requests
 * while request slots and the HBM budget allow (each admitted request keeps its
 * lattice, targets, search tables and results resident in a device arena of
 * hbm_budget_bytes), groups requests of one size class (joint count, K bucket,
 * T bucket) into one batched launch per stage, and keeps up to max_inflight
 * launches on the device at once,
 * so requests that arrive while others run are admitted as memory frees up and
 * their work overlaps. Every request runs with the server's params. */
typedef struct cpp_server cpp_server_t;

typedef struct cpp_server_config {
    int32_t device;           /* CUDA device ordinal */
    int32_t max_slots;        /* requests resident on the device at once (default 1024) */
    int32_t max_batch;        /* requests per launch (default 512) */
    int32_t max_inflight;     /* launches in flight, 1..32 (default 8) */
    size_t hbm_budget_bytes;  /* device arena for resident requests (default 40 GiB) */
    size_t pinned_bytes;      /* pinned host staging (default 1 GiB): copied inputs until
                                 their launch retires, each launch's table and results
                                 while in flight (results then move to the request, so
                                 uncollected results hold no pinned memory); a launch
                                 that finds no room waits for earlier ones to retire.
                                 0 = pageable only: each launch's copies then block the
                                 worker */
    cpp_params_t params;      /* settings of every request */
    /* Search form by load. While at most latency_requests requests are queued or on
     * the device, a launch runs each request's search in the latency form (the
     * smallest tile: clusters of up to 16 CTAs, 32 or 64 successors per CTA), the
     * fastest for one request. Above it, a launch takes requests of every K whose
     * searches take about as long, and runs each search in the form with the
     * highest edge rate per SM whose estimated time is at most search_budget_ms:
     * one CTA, clusters of 512 or of 256 successors per CTA (the wide form of
     * cpp_batch_set_split), clusters of 128 successors per CTA, else clusters of 64
     * (estimates from rates measured on GB300, stated in the server source).
     * Results are identical in every form. (defaults 8 and 12 ms; latency_requests >= 0,
     * search_budget_ms >= 0) */
    int32_t latency_requests;
    int32_t reserved_;
    double search_budget_ms;
} cpp_server_config_t;

#define CPP_REQ_BORROW 1  /* inputs stay valid and unchanged until the plan is collected:
                             no copy at submit (pinned inputs then go straight to the device) */
/* Anytime planning (§III-C: the latest valid solution is kept and can be taken
 * while the optimiser goes on improving it). After the plan's first pass the
 * request keeps its device slot and runs up to anytime_rounds improvement
 * rounds, each one trajectory-length step (cpp_smooth_step, with the collision
 * rows when the request has a model) and one pose phase from the current
 * trajectory, then the check. A result is published as the best so far when it
 * is valid and, after the first, shorter (trajectory length) than the last one
 * published. cpp_plan_peek reads the best so far at any time; poll / wait
 * complete when the rounds are used up (or cancel stops them) and return the
 * best so far, or the last result if none was valid. */
#define CPP_REQ_ANYTIME 2

typedef struct cpp_plan_req {
    const cpp_robot_t* robot;  /* host */
    int32_t T, K, Kp;          /* lattice shape, as for cpp_plan */
    int32_t flags;             /* CPP_REQ_BORROW | CPP_REQ_ANYTIME, or 0 */
    const float* cand;         /* host [T][n][Kp] */
    const double* targets;     /* host [T][7] */
    const cpp_geometry_t* geometry;  /* host, copied at submit; NULL = no collision model */
    int32_t anytime_rounds;    /* improvement rounds of an anytime request (0..100000) */
    int32_t reserved;
} cpp_plan_req_t;

typedef struct cpp_plan_result {  /* caller-owned HOST buffers; any pointer may be NULL */
    int32_t* sel;           /* [T] */
    float* q;               /* [T][n] */
    double* pose_err;       /* [T][2] */
    cpp_report_t* report;   /* [1] */
    float* best_cost;       /* [1] */
    double latency_ms;      /* out: submit -> completion seen by the server (peek: -> now) */
    int32_t dev_status;     /* out: device status word of the request */
    int32_t rounds;         /* out: improvement rounds run when this result was published */
} cpp_plan_result_t;

typedef struct cpp_server_stats {
    uint64_t submitted, completed, failed, cancelled, batches, sum_batch;
    int32_t max_batch_seen, resident, queued, reserved;
    size_t hbm_used, hbm_high_water;
    uint64_t improve_batches;  /* launches of anytime improvement rounds */
    uint64_t improve_rounds;   /* improvement rounds run (over all requests) */
    uint64_t published;        /* best-so-far results published */
} cpp_server_stats_t;

void cpp_server_config_default(cpp_server_config_t* cfg);
/* Allocates the device arena and pinned pool and starts the worker.
 * OOM if the arena cannot be allocated. CUDA loads each kernel on its first
 * launch (lazy module loading), so the first launch of each search form and
 * size stalls the worker briefly: plan a few requests of each expected shape,
 * singly and together, before serving latency-sensitive traffic (or run the
 * process with CUDA_MODULE_LOADING=EAGER). The launches in flight run on up to
 * max_inflight streams, each forking its search groups onto side streams; CUDA
 * maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 by default)
 * that run in order, so a serving process should set it to 32 before its first
 * CUDA call (measured on the serving mix: burst capacity 3-5k -> 5-6.3k plans/s). */
cpp_status cpp_server_create(const cpp_server_config_t* cfg, cpp_server_t** out);
/* Validates on the host (robot, lattice shape, finite targets with unit
 * quaternions within 1e-6), copies the inputs unless CPP_REQ_BORROW, queues the
 * request and returns its ticket. BUDGET if the request alone exceeds the arena.
 * Non-finite candidates are allowed (masked on the device). */
cpp_status cpp_plan_submit(cpp_server_t* srv, const cpp_plan_req_t* req, uint64_t* ticket);
/* PENDING until the plan is done; then copies the results into `res`, forgets the
 * ticket and returns the plan's status (OK, INFEASIBLE, CUDA, CANCELLED).
 * NOT_FOUND for an unknown or already collected ticket. */
cpp_status cpp_plan_poll(cpp_server_t* srv, uint64_t ticket, cpp_plan_result_t* res);
/* As poll, but blocks up to timeout_us (negative = no limit); PENDING on timeout. */
cpp_status cpp_plan_wait(cpp_server_t* srv, uint64_t ticket, cpp_plan_result_t* res,
                         int64_t timeout_us);
/* Removes a request that is still queued (OK; its poll returns CANCELLED); for
 * an anytime request on the device or improving, stops further rounds (OK; it
 * completes with its best so far); PENDING if it is on the device (not anytime)
 * or finished. */
cpp_status cpp_plan_cancel(cpp_server_t* srv, uint64_t ticket);
/* Anytime requests: copies the best-so-far result into `res` without collecting
 * the request and returns OK; PENDING while none is published; a finished
 * request that never published returns its status as poll would, still
 * uncollected. NOT_FOUND for an unknown ticket. */
cpp_status cpp_plan_peek(cpp_server_t* srv, uint64_t ticket, cpp_plan_result_t* res);
cpp_status cpp_server_get_stats(cpp_server_t* srv, cpp_server_stats_t* out);
/* Finishes the launches in flight, cancels queued requests, frees everything. */
void cpp_server_destroy(cpp_server_t* srv);

#ifdef __cplusplus
}
#endif
#endif
