/*
 * cppflow_oracle.h -- plain, slow FP64 CPU oracle for the CppFlow planner core.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or
 * call this code: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it. It shares no code, header, table or constant with
 * the CUDA library; the two meet only through seeded input arrays.
 *
 * Every routine follows a passage of "CppFlow: Generative Inverse Kinematics
 * for Efficient and Robust Cartesian Path Planning" (Morgan, Millard,
 * Sukhatme, arXiv 2309.09102), cited as "§II" (Problem Specification),
 * "§III-B" (Global discrete search) and "§III-C" (Levenberg-Marquardt for
 * trajectory optimization). Readings of silent or ambiguous passages are
 * stated beside the routine that adopts them.
 *
 * Every function here is pinned by a CPU test against something other than
 * itself (closed forms, library routines, brute force, invariants).
 */
#ifndef CPPFLOW_ORACLE_H
#define CPPFLOW_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXJ 16

/* Revolute serial chain in standard (distal) DH form, joint angles in rad. */
typedef struct orc_robot {
    int32_t n;               /* joints, 1..16 */
    int32_t pad_;
    double a[ORC_MAXJ];      /* link length along x_j (m) */
    double d[ORC_MAXJ];      /* link offset along z_{j-1} (m) */
    double alpha[ORC_MAXJ];  /* link twist about x_j (rad) */
    double theta0[ORC_MAXJ]; /* joint angle offset (rad) */
    double lo[ORC_MAXJ];     /* lower joint limit (rad) */
    double hi[ORC_MAXJ];     /* upper joint limit (rad) */
} orc_robot;

/* Thresholds, penalties and LM settings. Angles in rad. */
typedef struct orc_params {
    double tau_pos;       /* pose-valid position threshold (m) */
    double tau_rot;       /* pose-valid rotation threshold (rad) */
    double near_margin;   /* near-limit band (rad) */
    double pen_limit;     /* node cost for out-of/near-limit configs */
    double pen_pose;      /* node cost for pose-invalid configs */
    double jump_max;      /* discontinuity bound per step (rad) */
    double lambda0, lambda_up, lambda_down, lambda_min, lambda_max;
    double freeze_step;   /* stop a waypoint when max|delta| < this */
    double freeze_cost;   /* stop a waypoint when F < this */
    int32_t lm_iters;
    uint32_t free_mask;   /* bit j set: joint j may move in LM */
} orc_params;

/* mask bits */
#define ORC_OUT       1u
#define ORC_NEAR      2u
#define ORC_POSE      4u
#define ORC_NONFINITE 8u
#define ORC_PAD      16u

/* ---- §II: forward kinematics and pose error ---- */
void   orc_fk(const orc_robot* r, const double* q, double R[9], double p[3]);
void   orc_fk_frames(const orc_robot* r, const double* q, double z[][3], double o[][3],
                     double R[9], double p[3]);
void   orc_quat_to_R(const double quat_wxyz[4], double R[9]);
void   orc_R_to_quat(const double R[9], double quat_wxyz[4]);
double orc_rot_angle(const double Rt[9], const double R[9]);
void   orc_pose_error(const double Rt[9], const double pt[3], const double R[9],
                      const double p[3], double* pos, double* rot);
void   orc_fk_pose(const orc_robot* r, const double* q /*[N][n]*/, int64_t N,
                   double* pose /*[N][7] xyz wxyz*/);

/* ---- §II joint limits + §III-B node costs ---- */
void orc_mask(const orc_robot* r, const orc_params* P, const float* cand /*[T][n][Kp]*/,
              const double* targets /*[T][7]*/, int T, int K, int Kp,
              uint8_t* mask /*[T][Kp]*/, float* pen /*[T][Kp]*/, double* err /*[T][Kp][2] or 0*/);

/* ---- §III-B collision cost, §III-C collision distances ----
 * The robot as capsules (segment + radius) fixed to its DH frames, obstacles as
 * cuboids. Frame f of a capsule: 0 = base, j = the frame after joint j. */
#define ORC_MAX_CAPS 12
#define ORC_MAX_PAIRS 64
#define ORC_MAX_BOXES 8
#define ORC_COLLIDE  32u
typedef struct orc_capsule {
    int32_t frame, pad_;
    double a[3], b[3];       /* segment end points in the capsule's frame (m) */
    double radius;
} orc_capsule;
typedef struct orc_cuboid {
    double R[9], p[3];       /* box frame -> world: x_w = R x_b + p */
    double half[3];          /* the box is [-half, half] in its frame */
} orc_cuboid;
typedef struct orc_geometry {
    int32_t n_caps, n_pairs, n_boxes, pad_;
    orc_capsule caps[ORC_MAX_CAPS];
    int32_t pairs[ORC_MAX_PAIRS][2];   /* self-collision capsule pairs */
    orc_cuboid boxes[ORC_MAX_BOXES];   /* every capsule is checked against every box */
} orc_geometry;
double orc_seg_seg_dist2(const double a1[3], const double b1[3], const double a2[3],
                         const double b2[3], double* t1, double* t2);
double orc_seg_box_dist2(const double a[3], const double b[3], const double half[3], double* t);
void   orc_capsules_world(const orc_robot* r, const orc_geometry* g, const double* q,
                          double A[][3], double B[][3]);
void   orc_clearance(const orc_robot* r, const orc_geometry* g, const double* q,
                     double* self_min, double* env_min);
int    orc_collision_rows(const orc_robot* r, const orc_geometry* g, const double* q,
                          double d_safe, double w, double* res, double* J /*[rows][n]*/,
                          int max_rows);
int    orc_diff_step_geo(const orc_robot* r, const orc_geometry* g, const double* q_in, int T,
                         double lambda_d, double d_safe, double w, double* q_out,
                         int32_t* rows_out);
void   orc_lm_smooth_geo(const orc_robot* r, const orc_params* P, const orc_geometry* g,
                         const double* q_in, const double* targets, int T, int rounds,
                         double lambda_d, double d_safe, double w, double* q_out,
                         int32_t* taken);
void   orc_mask_geo(const orc_robot* r, const orc_params* P, const orc_geometry* g,
                    double pen_collide, const float* cand, const double* targets, int T, int K,
                    int Kp, uint8_t* mask, float* pen, double* err, double* clearance);

/* ---- §III-B: dynamic-programming search over the T x K x K lattice ---- */
int orc_dp_f32(const float* cand, const float* pen, int T, int K, int Kp, int n,
               int32_t* sel, float* best_cost, float* cost_T /*[Kp] or 0*/,
               uint16_t* bp /*[T][Kp] or 0*/);
int orc_dp_f32_ex(const float* cand, const float* pen, int T, int K, int Kp, int n,
                  int objective /* 0 sum, 1 min-max */, int32_t* sel, float* best_cost,
                  float* cost_T, uint16_t* bp);
float orc_path_mjac_f32(const float* cand, int T, int Kp, int n, const int32_t* sel);
int orc_dp_f64(const float* cand, const float* pen, int T, int K, int Kp, int n,
               int32_t* sel, double* best_cost);

/* ---- §III-C: Levenberg-Marquardt, one independent problem per waypoint ---- */
void   orc_log_rot(const double M[9], double w[3]);
void   orc_jacobian(const orc_robot* r, const double* q, double J[] /*[6][n]*/);
void   orc_residual(const orc_robot* r, const double* q, const double* target7,
                    double e[6]);
void   orc_lm(const orc_robot* r, const orc_params* P, const double* q_in /*[T][n]*/,
              const double* targets /*[T][7]*/, int T, double* q_out /*[T][n]*/,
              double* F_hist /*[T][lm_iters+1] or 0*/, int32_t* iters_run /*[T] or 0*/);

/* ---- §III-C non-stationary objective: trajectory-length (differencing) steps ---- */
int  orc_block_tridiag_solve(int T, int n, const double* Dg /*[T][n][n]*/,
                             const double* Off /*[T-1][n][n]*/, const double* b /*[T][n]*/,
                             double* x /*[T][n]*/);
int  orc_diff_step(const orc_robot* r, const double* q_in /*[T][n]*/, int T, double lambda_d,
                   double* q_out /*[T][n]*/);
void orc_lm_smooth(const orc_robot* r, const orc_params* P, const double* q_in,
                   const double* targets, int T, int rounds, double lambda_d,
                   double* q_out, int32_t* taken);

/* ---- §II report: errors, validity, mjac, jumps, trajectory length ---- */
typedef struct orc_report {
    double max_pos, max_rot;      /* worst waypoint error */
    double mjac;                  /* max over steps and joints of |dq| */
    double sum_linf;              /* sum over steps of the per-step L-inf jump */
    double traj_len;              /* sum over steps and joints of |dq| */
    int32_t n_pose_fail;          /* waypoints above tau */
    int32_t n_limit_fail;         /* waypoints outside joint limits */
    int32_t n_jump_fail;          /* steps above jump_max */
    int32_t valid;
} orc_report;
void orc_check(const orc_robot* r, const orc_params* P, const double* q /*[T][n]*/,
               const double* targets, int T, double* pose_err /*[T][2] or 0*/,
               orc_report* rep);

/* ---- cpf-BatchOpt: the smoothest candidate lanes refined directly ---- */
void orc_lane_mjac_f32(const float* cand, int T, int K, int Kp, int n, float* mjac /*[K]*/);
int  orc_batch_opt(const orc_robot* r, const orc_params* P, const float* cand,
                   const double* targets, int T, int K, int Kp, int lanes, int32_t* lane_sel,
                   float* lane_mjac, double* q_out /*[lanes][T][n]*/, orc_report* reps);

/* ---- whole post-generation pipeline for one request ---- */
int orc_plan(const orc_robot* r, const orc_params* P, const float* cand,
             const double* targets, int T, int K, int Kp,
             int32_t* sel, float* best_cost, double* q_out /*[T][n]*/,
             double* pose_err /*[T][2]*/, orc_report* rep);

#ifdef __cplusplus
}
#endif
#endif
