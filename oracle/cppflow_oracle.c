/*
 * cppflow_oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * use this file. It is written for a reader who checks it against the paper by
 * eye: no blocking, no fusion, no reordering beyond what each definition says.
 * Build: gcc -O2 -ffp-contract=off (no fast-math, no FMA contraction), so the
 * FP32 DP cost path rounds exactly once per IEEE operation.
 *
 * Paper: "CppFlow: Generative Inverse Kinematics for Efficient and Robust
 * Cartesian Path Planning", arXiv 2309.09102. Section tags: §II Problem
 * Specification, §III-B Global discrete search, §III-C Levenberg-Marquardt.
 *
 * Parity status: every routine is pinned by a CPU test (closed forms, SciPy
 * rotation routines, finite differences, brute-force enumeration, invariants).
 */
#include "cppflow_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* small 4x4 / 3x3 helpers (plain row-major loops)                           */
/* ------------------------------------------------------------------------- */
static void mat4_identity(double M[16]) {
    memset(M, 0, 16 * sizeof(double));
    M[0] = M[5] = M[10] = M[15] = 1.0;
}

static void mat4_mul(const double A[16], const double B[16], double C[16]) {
    double T[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[4 * r + k] * B[4 * k + c];
            T[4 * r + c] = s;
        }
    memcpy(C, T, sizeof(T));
}

static void rot_z(double th, double M[16]) {
    mat4_identity(M);
    M[0] = cos(th); M[1] = -sin(th);
    M[4] = sin(th); M[5] = cos(th);
}

static void rot_x(double al, double M[16]) {
    mat4_identity(M);
    M[5] = cos(al);  M[6] = -sin(al);
    M[9] = sin(al);  M[10] = cos(al);
}

static void trans_z(double d, double M[16]) { mat4_identity(M); M[11] = d; }
static void trans_x(double a, double M[16]) { mat4_identity(M); M[3] = a; }

/* §II: FK(q): R^d -> SE(3). Reading (the paper gives no convention): standard
 * (distal) DH, A_j = Rz(q_j + theta0_j) Tz(d_j) Tx(a_j) Rx(alpha_j), base and
 * tool frames are the identity. Returns A_j as a 4x4 homogeneous matrix. */
static void dh_link(const orc_robot* r, int j, double qj, double A[16]) {
    double M[16];
    rot_z(qj + r->theta0[j], A);
    trans_z(r->d[j], M);  mat4_mul(A, M, A);
    trans_x(r->a[j], M);  mat4_mul(A, M, A);
    rot_x(r->alpha[j], M); mat4_mul(A, M, A);
}

static void split_pose(const double M[16], double R[9], double p[3]) {
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = M[4 * r + c];
        p[r] = M[4 * r + 3];
    }
}

/* §II: T(q) = A_1 A_2 ... A_n. */
void orc_fk(const orc_robot* r, const double* q, double R[9], double p[3]) {
    double T[16], A[16];
    mat4_identity(T);
    for (int j = 0; j < r->n; ++j) {
        dh_link(r, j, q[j], A);
        mat4_mul(T, A, T);
    }
    split_pose(T, R, p);
}

/* Frames T_j = A_1..A_j for j = 0..n (T_0 = identity): z_j = third column of
 * the rotation of T_j, o_j = its origin. Joint j (0-based) turns about z_j. */
void orc_fk_frames(const orc_robot* r, const double* q, double z[][3], double o[][3],
                   double R[9], double p[3]) {
    double T[16], A[16];
    mat4_identity(T);
    for (int j = 0; j <= r->n; ++j) {
        for (int c = 0; c < 3; ++c) { z[j][c] = T[4 * c + 2]; o[j][c] = T[4 * c + 3]; }
        if (j == r->n) break;
        dh_link(r, j, q[j], A);
        mat4_mul(T, A, T);
    }
    split_pose(T, R, p);
}

/* Unit quaternion (w, x, y, z) -> rotation matrix (normalised first). */
void orc_quat_to_R(const double qq[4], double R[9]) {
    double nrm = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    double w = qq[0] / nrm, x = qq[1] / nrm, y = qq[2] / nrm, z = qq[3] / nrm;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Rotation matrix -> unit quaternion (w >= 0), by the largest-pivot branch. */
void orc_R_to_quat(const double R[9], double q[4]) {
    double tr = R[0] + R[4] + R[8];
    double w, x, y, z;
    if (tr > 0.0) {
        double s = sqrt(tr + 1.0) * 2.0;
        w = 0.25 * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
    } else if (R[0] > R[4] && R[0] > R[8]) {
        double s = sqrt(1.0 + R[0] - R[4] - R[8]) * 2.0;
        w = (R[7] - R[5]) / s; x = 0.25 * s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
    } else if (R[4] > R[8]) {
        double s = sqrt(1.0 + R[4] - R[0] - R[8]) * 2.0;
        w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; y = 0.25 * s; z = (R[5] + R[7]) / s;
    } else {
        double s = sqrt(1.0 + R[8] - R[0] - R[4]) * 2.0;
        w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; z = 0.25 * s;
    }
    if (w < 0.0) { w = -w; x = -x; y = -y; z = -z; }
    double nrm = sqrt(w * w + x * x + y * y + z * z);
    q[0] = w / nrm; q[1] = x / nrm; q[2] = y / nrm; q[3] = z / nrm;
}

/* §II "Pose error": the rotational error is the geodesic distance between the
 * rotations of FK(q) and the target, i.e. the angle of E = Rt^T R, computed as
 * atan2(|vee(E - E^T)| / 2, (tr E - 1) / 2) in [0, pi]. */
double orc_rot_angle(const double Rt[9], const double R[9]) {
    double E[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Rt[3 * k + r] * R[3 * k + c];
            E[3 * r + c] = s;
        }
    double vx = E[7] - E[5], vy = E[2] - E[6], vz = E[3] - E[1];
    double s = 0.5 * sqrt(vx * vx + vy * vy + vz * vz);
    double c = 0.5 * (E[0] + E[4] + E[8] - 1.0);
    return atan2(s, c);
}

/* §II "Pose error": position error is the Euclidean norm of the difference. */
void orc_pose_error(const double Rt[9], const double pt[3], const double R[9],
                    const double p[3], double* pos, double* rot) {
    double dx = p[0] - pt[0], dy = p[1] - pt[1], dz = p[2] - pt[2];
    *pos = sqrt(dx * dx + dy * dy + dz * dz);
    *rot = orc_rot_angle(Rt, R);
}

void orc_fk_pose(const orc_robot* r, const double* q, int64_t N, double* pose) {
    for (int64_t i = 0; i < N; ++i) {
        double R[9], p[3];
        orc_fk(r, q + i * r->n, R, p);
        pose[7 * i + 0] = p[0]; pose[7 * i + 1] = p[1]; pose[7 * i + 2] = p[2];
        orc_R_to_quat(R, pose + 7 * i + 3);
    }
}

static void target_pose(const double* t7, double Rt[9], double pt[3]) {
    pt[0] = t7[0]; pt[1] = t7[1]; pt[2] = t7[2];
    orc_quat_to_R(t7 + 3, Rt);
}

/* ------------------------------------------------------------------------- */
/* §II joint limits + §III-B node costs                                      */
/* ------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------- */
/* Collision geometry: §III-B (+100 node cost) and §III-C (distances)         */
/* ------------------------------------------------------------------------- */
static double dist2(const double x[3], const double y[3]) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    return d0 * d0 + d1 * d1 + d2 * d2;
}
static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Squared distance between segments P(s) = a1 + s (b1 - a1) and Q(t) = a2 +
 * t (b2 - a2), s, t in [0, 1]: the convex QP of §III-C solved by enumerating its
 * active sets. f(s, t) = |P(s) - Q(t)|^2 is convex on the unit square, so its
 * minimum is the interior stationary point when that lies in the square, else
 * the smallest of the four edge minima, each a 1-D convex problem solved by
 * clamping the edge's stationary point. Every candidate is evaluated directly
 * as |P - Q|^2 and the smallest wins (ties: first found). */
double orc_seg_seg_dist2(const double a1[3], const double b1[3], const double a2[3],
                         const double b2[3], double* t1, double* t2) {
    double d1[3], d2[3], r[3];
    for (int k = 0; k < 3; ++k) { d1[k] = b1[k] - a1[k]; d2[k] = b2[k] - a2[k]; r[k] = a1[k] - a2[k]; }
    const double A = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
    const double C = d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2];
    const double B = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
    const double D = d1[0] * r[0] + d1[1] * r[1] + d1[2] * r[2];
    const double E = d2[0] * r[0] + d2[1] * r[1] + d2[2] * r[2];
    double cs[5], ct[5];
    int m = 0;
    const double det = A * C - B * B;
    if (det > 1e-300) {
        const double s = (B * E - C * D) / det, t = (A * E - B * D) / det;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) { cs[m] = s; ct[m] = t; ++m; }
    }
    /* edges s = 0, s = 1 (t free), t = 0, t = 1 (s free) */
    cs[m] = 0.0; ct[m] = C > 0.0 ? clamp01(E / C) : 0.0; ++m;
    cs[m] = 1.0; ct[m] = C > 0.0 ? clamp01((B + E) / C) : 0.0; ++m;
    cs[m] = A > 0.0 ? clamp01(-D / A) : 0.0; ct[m] = 0.0; ++m;
    cs[m] = A > 0.0 ? clamp01((B - D) / A) : 0.0; ct[m] = 1.0; ++m;
    double best = INFINITY;
    for (int c = 0; c < m; ++c) {
        double P[3], Q[3];
        for (int k = 0; k < 3; ++k) { P[k] = a1[k] + cs[c] * d1[k]; Q[k] = a2[k] + ct[c] * d2[k]; }
        const double f = dist2(P, Q);
        if (f < best) { best = f; if (t1) *t1 = cs[c]; if (t2) *t2 = ct[c]; }
    }
    return best;
}

/* Squared distance between the segment x(t) = a + t (b - a), t in [0, 1], and
 * the box [-half, half] (both in the box's frame): the QP of §III-C over (t, p).
 * For fixed t the best p is x(t) clamped to the box, so the cost is
 * g(t) = sum_k dist(x_k(t), [-h_k, h_k])^2, convex and piecewise quadratic in t
 * with breakpoints where some x_k(t) crosses -h_k or h_k. On each piece g is one
 * quadratic (its active faces fixed by the piece's midpoint); its minimiser,
 * clamped to the piece, and the piece's ends are evaluated, the smallest wins. */
static double box_cost(const double a[3], const double d[3], const double h[3], double t) {
    double g = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double x = a[k] + t * d[k];
        if (x > h[k]) g += (x - h[k]) * (x - h[k]);
        else if (x < -h[k]) g += (x + h[k]) * (x + h[k]);
    }
    return g;
}
double orc_seg_box_dist2(const double a[3], const double b[3], const double half[3], double* tout) {
    double d[3], br[8];
    int nb = 0;
    for (int k = 0; k < 3; ++k) d[k] = b[k] - a[k];
    br[nb++] = 0.0;
    br[nb++] = 1.0;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) continue;
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            const double t = (sgn * half[k] - a[k]) / d[k];
            if (t > 0.0 && t < 1.0) br[nb++] = t;
        }
    }
    for (int i = 1; i < nb; ++i)      /* insertion sort */
        for (int j = i; j > 0 && br[j] < br[j - 1]; --j) { double x = br[j]; br[j] = br[j - 1]; br[j - 1] = x; }
    double best = INFINITY, tb = 0.0;
    for (int i = 0; i + 1 < nb; ++i) {
        const double ta = br[i], tz = br[i + 1], tm = 0.5 * (ta + tz);
        double num = 0.0, den = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double x = a[k] + tm * d[k];
            double c;
            if (x > half[k]) c = half[k];
            else if (x < -half[k]) c = -half[k];
            else continue;
            num += d[k] * (c - a[k]);
            den += d[k] * d[k];
        }
        double cand[3] = {ta, tz, ta};
        int nc = 2;
        if (den > 0.0) {
            double ts = num / den;
            if (ts < ta) ts = ta;
            if (ts > tz) ts = tz;
            cand[nc++] = ts;
        }
        for (int c = 0; c < nc; ++c) {
            const double g = box_cost(a, d, half, cand[c]);
            if (g < best) { best = g; tb = cand[c]; }
        }
    }
    if (tout) *tout = tb;
    return best;
}

/* World end points of every capsule: frame transforms T_0 = I, T_j = T_{j-1} A_j
 * (FP64 DH products as in orc_fk), x_w = R_f x + p_f. */
void orc_capsules_world(const orc_robot* r, const orc_geometry* g, const double* q,
                        double A[][3], double B[][3]) {
    double Tf[ORC_MAXJ + 1][16], L[16];
    mat4_identity(Tf[0]);
    for (int j = 0; j < r->n; ++j) {
        dh_link(r, j, q[j], L);
        mat4_mul(Tf[j], L, Tf[j + 1]);
    }
    for (int c = 0; c < g->n_caps; ++c) {
        const double* M = Tf[g->caps[c].frame];
        for (int k = 0; k < 3; ++k) {
            A[c][k] = M[4 * k] * g->caps[c].a[0] + M[4 * k + 1] * g->caps[c].a[1] +
                      M[4 * k + 2] * g->caps[c].a[2] + M[4 * k + 3];
            B[c][k] = M[4 * k] * g->caps[c].b[0] + M[4 * k + 1] * g->caps[c].b[1] +
                      M[4 * k + 2] * g->caps[c].b[2] + M[4 * k + 3];
        }
    }
}

/* Clearances of one configuration (§III-C): over the listed capsule pairs,
 * segment distance - r_u - r_v; over every capsule and box, segment-box distance
 * - r_u (the box frame: x_b = R^T (x_w - p)). +inf when a list is empty. */
void orc_clearance(const orc_robot* r, const orc_geometry* g, const double* q,
                   double* self_min, double* env_min) {
    double A[ORC_MAX_CAPS][3], B[ORC_MAX_CAPS][3];
    orc_capsules_world(r, g, q, A, B);
    double sm = INFINITY, em = INFINITY;
    for (int k = 0; k < g->n_pairs; ++k) {
        const int u = g->pairs[k][0], v = g->pairs[k][1];
        const double d = sqrt(orc_seg_seg_dist2(A[u], B[u], A[v], B[v], 0, 0)) -
                         g->caps[u].radius - g->caps[v].radius;
        if (d < sm) sm = d;
    }
    for (int o = 0; o < g->n_boxes; ++o) {
        const orc_cuboid* bx = &g->boxes[o];
        for (int c = 0; c < g->n_caps; ++c) {
            double a[3], b[3];
            for (int k = 0; k < 3; ++k) {
                a[k] = bx->R[k] * (A[c][0] - bx->p[0]) + bx->R[3 + k] * (A[c][1] - bx->p[1]) +
                       bx->R[6 + k] * (A[c][2] - bx->p[2]);
                b[k] = bx->R[k] * (B[c][0] - bx->p[0]) + bx->R[3 + k] * (B[c][1] - bx->p[1]) +
                       bx->R[6 + k] * (B[c][2] - bx->p[2]);
            }
            const double d = sqrt(orc_seg_box_dist2(a, b, bx->half, 0)) - g->caps[c].radius;
            if (d < em) em = d;
        }
    }
    *self_min = sm;
    *env_min = em;
}

/* Collision rows of r_diff for one configuration (§III-C; reading: a hinge on a
 * safety margin, since the distances themselves are to grow, not shrink): for
 * every listed pair and every capsule-box combination with clearance d <
 * d_safe, a residual w (d_safe - d) and its gradient row -w dd/dq. By the
 * envelope theorem dd/dq is the derivative at the QP's minimiser: with x_u, x_v
 * the closest points and n = (x_u - x_v) / |x_u - x_v|,
 *   dd/dq_j = n . (dx_u/dq_j - dx_v/dq_j),   dx/dq_j = z_j x (x - o_j)
 * for a point on a frame that joint j moves (frame > j), else 0; for a box the
 * box point is fixed. Rows whose closest points are within ORC_MIN_DIR (1e-6 m)
 * of each other are skipped: at zero distance (touching or interpenetrating
 * shapes, where the QP's minimum is 0) the direction is undefined, and below
 * 1e-6 m it is rounding noise. Returns the number of rows (at most max_rows);
 * J is [rows][n]. */
#define ORC_MIN_DIR 1e-6
static void point_rate(const double z[][3], const double o[][3], int frame, int n,
                       const double x[3], double out[][3]) {
    for (int j = 0; j < n; ++j) {
        if (frame > j) {
            const double dx = x[0] - o[j][0], dy = x[1] - o[j][1], dz = x[2] - o[j][2];
            out[j][0] = z[j][1] * dz - z[j][2] * dy;
            out[j][1] = z[j][2] * dx - z[j][0] * dz;
            out[j][2] = z[j][0] * dy - z[j][1] * dx;
        } else {
            out[j][0] = out[j][1] = out[j][2] = 0.0;
        }
    }
}

int orc_collision_rows(const orc_robot* r, const orc_geometry* g, const double* q,
                       double d_safe, double w, double* res, double* J, int max_rows) {
    const int n = r->n;
    double z[ORC_MAXJ + 1][3], o[ORC_MAXJ + 1][3], Re[9], pe[3];
    orc_fk_frames(r, q, z, o, Re, pe);
    double A[ORC_MAX_CAPS][3], B[ORC_MAX_CAPS][3];
    orc_capsules_world(r, g, q, A, B);
    int m = 0;
    for (int k = 0; k < g->n_pairs && m < max_rows; ++k) {
        const int u = g->pairs[k][0], v = g->pairs[k][1];
        double s, t;
        const double d2 = orc_seg_seg_dist2(A[u], B[u], A[v], B[v], &s, &t);
        const double dist = sqrt(d2);
        const double d = dist - g->caps[u].radius - g->caps[v].radius;
        if (!(d < d_safe) || dist <= ORC_MIN_DIR) continue;
        double xu[3], xv[3], nv[3], ru[ORC_MAXJ][3], rv[ORC_MAXJ][3];
        for (int c = 0; c < 3; ++c) {
            xu[c] = A[u][c] + s * (B[u][c] - A[u][c]);
            xv[c] = A[v][c] + t * (B[v][c] - A[v][c]);
            nv[c] = (xu[c] - xv[c]) / dist;
        }
        point_rate(z, o, g->caps[u].frame, n, xu, ru);
        point_rate(z, o, g->caps[v].frame, n, xv, rv);
        res[m] = w * (d_safe - d);
        for (int j = 0; j < n; ++j)
            J[(size_t)m * n + j] = -w * (nv[0] * (ru[j][0] - rv[j][0]) + nv[1] * (ru[j][1] - rv[j][1]) +
                                         nv[2] * (ru[j][2] - rv[j][2]));
        ++m;
    }
    for (int ob = 0; ob < g->n_boxes; ++ob) {
        const orc_cuboid* bx = &g->boxes[ob];
        for (int c = 0; c < g->n_caps && m < max_rows; ++c) {
            double a[3], b[3], t;
            for (int k = 0; k < 3; ++k) {
                a[k] = bx->R[k] * (A[c][0] - bx->p[0]) + bx->R[3 + k] * (A[c][1] - bx->p[1]) +
                       bx->R[6 + k] * (A[c][2] - bx->p[2]);
                b[k] = bx->R[k] * (B[c][0] - bx->p[0]) + bx->R[3 + k] * (B[c][1] - bx->p[1]) +
                       bx->R[6 + k] * (B[c][2] - bx->p[2]);
            }
            const double d2 = orc_seg_box_dist2(a, b, bx->half, &t);
            const double dist = sqrt(d2);
            const double d = dist - g->caps[c].radius;
            if (!(d < d_safe) || dist <= ORC_MIN_DIR) continue;
            double xb[3], pb[3], nb[3], nw[3], x[3], rc[ORC_MAXJ][3];
            for (int k = 0; k < 3; ++k) {
                xb[k] = a[k] + t * (b[k] - a[k]);
                pb[k] = xb[k] > bx->half[k] ? bx->half[k] : (xb[k] < -bx->half[k] ? -bx->half[k] : xb[k]);
                nb[k] = (xb[k] - pb[k]) / dist;
            }
            for (int k = 0; k < 3; ++k) {   /* back to the world: R (box) */
                nw[k] = bx->R[3 * k] * nb[0] + bx->R[3 * k + 1] * nb[1] + bx->R[3 * k + 2] * nb[2];
                x[k] = A[c][k] + t * (B[c][k] - A[c][k]);
            }
            point_rate(z, o, g->caps[c].frame, n, x, rc);
            res[m] = w * (d_safe - d);
            for (int j = 0; j < n; ++j)
                J[(size_t)m * n + j] = -w * (nw[0] * rc[j][0] + nw[1] * rc[j][1] + nw[2] * rc[j][2]);
            ++m;
        }
    }
    return m;
}

/* Per candidate (i, k):
 *   NONFINITE: some joint value is not finite -> node cost +inf, no other bit.
 *   OUT:  some q_j < lo_j or q_j > hi_j                (§II "Joint limits")
 *   NEAR: some q_j within near_margin of a limit       (§III-B, +10 band)
 *   POSE: position error > tau_pos or rotation error > tau_rot (§II)
 *   COLLIDE (orc_mask_geo only): the smaller clearance is negative (§III-B)
 *   pen = pen_limit * [OUT or NEAR] + pen_pose * [POSE] (+ pen_collide * [COLLIDE])
 *                                                      (§III-B additive costs)
 * Readings: limit comparisons are made in FP32 on the FP32 candidate against
 * the FP32-rounded thresholds (lo, hi, lo+m, hi-m, each formed in FP64 and
 * rounded once), so the OUT/NEAR bits are exact on any IEEE machine; a
 * configuration outside the limits is charged like one inside the band; the
 * pose bit takes its errors from FP64 forward kinematics of the upcast
 * candidate. Padding lanes k in [K, Kp) get PAD and +inf. */
/* Mask and node costs, with the collision cost of §III-B when g is given:
 * COLLIDE when the smaller clearance is negative, cost += pen_collide (the sum
 * of the node's costs formed in FP64 in the order limit, pose, collision, then
 * rounded to FP32 once). clearance [T][Kp] (or 0) receives the smaller
 * clearance (+inf without geometry, NaN for padding / non-finite). */
static void mask_core(const orc_robot* r, const orc_params* P, const orc_geometry* g,
                      double pen_collide, const float* cand, const double* targets, int T,
                      int K, int Kp, uint8_t* mask, float* pen, double* err, double* clearance) {
    const int n = r->n;
    float lo_f[ORC_MAXJ], hi_f[ORC_MAXJ], nlo_f[ORC_MAXJ], nhi_f[ORC_MAXJ];
    for (int j = 0; j < n; ++j) {
        lo_f[j] = (float)r->lo[j];
        hi_f[j] = (float)r->hi[j];
        nlo_f[j] = (float)(r->lo[j] + P->near_margin);
        nhi_f[j] = (float)(r->hi[j] - P->near_margin);
    }
    for (int i = 0; i < T; ++i) {
        double Rt[9], pt[3];
        target_pose(targets + 7 * i, Rt, pt);
        for (int k = 0; k < Kp; ++k) {
            size_t o = (size_t)i * Kp + k;
            if (k >= K) {
                mask[o] = ORC_PAD; pen[o] = INFINITY;
                if (err) { err[2 * o] = NAN; err[2 * o + 1] = NAN; }
                if (clearance) clearance[o] = NAN;
                continue;
            }
            float qf[ORC_MAXJ];
            double qd[ORC_MAXJ];
            int finite = 1;
            for (int j = 0; j < n; ++j) {
                qf[j] = cand[((size_t)i * n + j) * Kp + k];
                qd[j] = (double)qf[j];
                if (!isfinite(qf[j])) finite = 0;
            }
            if (!finite) {
                mask[o] = ORC_NONFINITE; pen[o] = INFINITY;
                if (err) { err[2 * o] = NAN; err[2 * o + 1] = NAN; }
                if (clearance) clearance[o] = NAN;
                continue;
            }
            unsigned bits = 0;
            for (int j = 0; j < n; ++j) {
                if (qf[j] < lo_f[j] || qf[j] > hi_f[j]) bits |= ORC_OUT;
                if (qf[j] < nlo_f[j] || qf[j] > nhi_f[j]) bits |= ORC_NEAR;
            }
            double R[9], p[3], pos, rot;
            orc_fk(r, qd, R, p);
            orc_pose_error(Rt, pt, R, p, &pos, &rot);
            if (pos > P->tau_pos || rot > P->tau_rot) bits |= ORC_POSE;
            double cl = INFINITY;
            if (g) {
                double sm, em;
                orc_clearance(r, g, qd, &sm, &em);
                cl = sm < em ? sm : em;
                if (cl < 0.0) bits |= ORC_COLLIDE;
            }
            double c = 0.0;
            if (bits & (ORC_OUT | ORC_NEAR)) c += P->pen_limit;
            if (bits & ORC_POSE) c += P->pen_pose;
            if (bits & ORC_COLLIDE) c += pen_collide;
            mask[o] = (uint8_t)bits;
            pen[o] = (float)c;
            if (err) { err[2 * o] = pos; err[2 * o + 1] = rot; }
            if (clearance) clearance[o] = cl;
        }
    }
}

void orc_mask(const orc_robot* r, const orc_params* P, const float* cand,
              const double* targets, int T, int K, int Kp,
              uint8_t* mask, float* pen, double* err) {
    mask_core(r, P, 0, 0.0, cand, targets, T, K, Kp, mask, pen, err, 0);
}

void orc_mask_geo(const orc_robot* r, const orc_params* P, const orc_geometry* g,
                  double pen_collide, const float* cand, const double* targets, int T, int K,
                  int Kp, uint8_t* mask, float* pen, double* err, double* clearance) {
    mask_core(r, P, g, pen_collide, cand, targets, T, K, Kp, mask, pen, err, clearance);
}

/* ------------------------------------------------------------------------- */
/* §III-B global discrete search                                             */
/* ------------------------------------------------------------------------- */
/* Nodes are the K candidates at each of the T waypoints; every node at step i
 * has an edge to every node at step i+1. Objective (reading of the search's
 * cost): the SUM over steps of the per-step L-inf joint jump
 *   d(k, k') = max_j |q_{i+1,k',j} - q_{i,k,j}|,
 * plus the node costs. Node costs enter relative to the cheapest node of their
 * waypoint, r_i[k] = fl(pen_i[k] - m_i) with m_i = min_{k<K} pen_i[k] (m_i = 0
 * when that min is +inf): a constant added to every node of one waypoint
 * changes no path's rank, and it keeps the running FP32 cost small enough to
 * resolve the joint jumps (a uniform +100 per waypoint would otherwise grow it
 * to 100 T). Recurrence, evaluated literally in FP32:
 *   C_0[k]      = r_0[k]
 *   C_{i+1}[k'] = fl( min_k fl(C_i[k] + d(k, k')) + r_{i+1}[k'] )
 *   bp[i+1][k'] = smallest k attaining that min (strict '<' scan from k = 0)
 * then k_{T-1} = smallest argmin of C_{T-1}, and backtracking k_i = bp[i+1][k_{i+1}].
 * best_cost is min_k C_{T-1}[k] (the relative cost). The max over joints uses
 * fmaxf (a NaN term is ignored). Returns 0, or 3 when every final cost is +inf
 * (no feasible path). */
static float layer_min_f32(const float* pen_i, int K) {
    float m = INFINITY;
    for (int k = 0; k < K; ++k) m = fminf(m, pen_i[k]);
    return isinf(m) ? 0.0f : m;
}

/* Objective 1 is the paper's own (§III-B): a node costs the smallest mjac that any
 * path through it can reach -- a bottleneck (min-max) path. With the node costs
 * it reads
 *   C_0[k] = r_0[k],  C_{i+1}[k'] = fmaxf( min_k fmaxf(C_i[k], d(k, k')), r_{i+1}[k'] ),
 * i.e. a path costs max(largest per-step L-inf jump, largest relative node cost);
 * a node cost of 10 exceeds any revolute jump (pi), as the paper intends. max
 * and min are exact, so this objective involves no rounding at all. */
int orc_dp_f32_ex(const float* cand, const float* pen, int T, int K, int Kp, int n,
                  int objective, int32_t* sel, float* best_cost, float* cost_T,
                  uint16_t* bp_out) {
    float* C = (float*)malloc(sizeof(float) * (size_t)Kp);
    float* Cn = (float*)malloc(sizeof(float) * (size_t)Kp);
    uint16_t* bp = (uint16_t*)calloc((size_t)T * Kp, sizeof(uint16_t));
    float m0 = layer_min_f32(pen, K);
    for (int k = 0; k < Kp; ++k) C[k] = (k < K) ? pen[k] - m0 : INFINITY;
    for (int i = 0; i + 1 < T; ++i) {
        const float* qa = cand + (size_t)i * n * Kp;        /* step i   */
        const float* qb = cand + (size_t)(i + 1) * n * Kp;  /* step i+1 */
        const float m1 = layer_min_f32(pen + (size_t)(i + 1) * Kp, K);
        for (int kp = 0; kp < Kp; ++kp) {
            if (kp >= K) { Cn[kp] = INFINITY; continue; }
            float best = INFINITY;
            int arg = 0;
            for (int k = 0; k < K; ++k) {
                float d = fabsf(qb[kp] - qa[k]);
                for (int j = 1; j < n; ++j)
                    d = fmaxf(d, fabsf(qb[(size_t)j * Kp + kp] - qa[(size_t)j * Kp + k]));
                float v = objective ? fmaxf(C[k], d) : C[k] + d;
                if (v < best) { best = v; arg = k; }
            }
            const float r = pen[(size_t)(i + 1) * Kp + kp] - m1;
            Cn[kp] = objective ? fmaxf(best, r) : best + r;
            bp[(size_t)(i + 1) * Kp + kp] = (uint16_t)arg;
        }
        float* t = C; C = Cn; Cn = t;
    }
    float best = INFINITY;
    int arg = 0;
    for (int k = 0; k < K; ++k)
        if (C[k] < best) { best = C[k]; arg = k; }
    sel[T - 1] = arg;
    for (int i = T - 1; i > 0; --i) sel[i - 1] = bp[(size_t)i * Kp + sel[i]];
    *best_cost = best;
    if (cost_T) memcpy(cost_T, C, sizeof(float) * (size_t)Kp);
    if (bp_out) memcpy(bp_out, bp, sizeof(uint16_t) * (size_t)T * Kp);
    free(C); free(Cn); free(bp);
    return isinf(best) ? 3 : 0;
}

int orc_dp_f32(const float* cand, const float* pen, int T, int K, int Kp, int n,
               int32_t* sel, float* best_cost, float* cost_T, uint16_t* bp_out) {
    return orc_dp_f32_ex(cand, pen, T, K, Kp, n, 0, sel, best_cost, cost_T, bp_out);
}

/* mjac of a selection (§III-B): max over steps and joints of |q_{i+1} - q_i|, in FP32. */
float orc_path_mjac_f32(const float* cand, int T, int Kp, int n, const int32_t* sel) {
    float m = 0.0f;
    for (int i = 0; i + 1 < T; ++i)
        for (int j = 0; j < n; ++j)
            m = fmaxf(m, fabsf(cand[((size_t)(i + 1) * n + j) * Kp + sel[i + 1]] -
                               cand[((size_t)i * n + j) * Kp + sel[i]]));
    return m;
}

/* The same recurrence in FP64 (used for the error report, not for indices),
 * with the same per-waypoint relative node costs. */
static double layer_min_f64(const float* pen_i, int K) {
    double m = INFINITY;
    for (int k = 0; k < K; ++k) m = fmin(m, (double)pen_i[k]);
    return isinf(m) ? 0.0 : m;
}

int orc_dp_f64(const float* cand, const float* pen, int T, int K, int Kp, int n,
               int32_t* sel, double* best_cost) {
    double* C = (double*)malloc(sizeof(double) * (size_t)Kp);
    double* Cn = (double*)malloc(sizeof(double) * (size_t)Kp);
    int32_t* bp = (int32_t*)calloc((size_t)T * Kp, sizeof(int32_t));
    double m0 = layer_min_f64(pen, K);
    for (int k = 0; k < Kp; ++k) C[k] = (k < K) ? (double)pen[k] - m0 : INFINITY;
    for (int i = 0; i + 1 < T; ++i) {
        const float* qa = cand + (size_t)i * n * Kp;
        const float* qb = cand + (size_t)(i + 1) * n * Kp;
        const double m1 = layer_min_f64(pen + (size_t)(i + 1) * Kp, K);
        for (int kp = 0; kp < K; ++kp) {
            double best = INFINITY;
            int arg = 0;
            for (int k = 0; k < K; ++k) {
                double d = fabs((double)qb[kp] - (double)qa[k]);
                for (int j = 1; j < n; ++j)
                    d = fmax(d, fabs((double)qb[(size_t)j * Kp + kp] - (double)qa[(size_t)j * Kp + k]));
                double v = C[k] + d;
                if (v < best) { best = v; arg = k; }
            }
            Cn[kp] = best + ((double)pen[(size_t)(i + 1) * Kp + kp] - m1);
            bp[(size_t)(i + 1) * Kp + kp] = arg;
        }
        double* t = C; C = Cn; Cn = t;
    }
    double best = INFINITY;
    int arg = 0;
    for (int k = 0; k < K; ++k)
        if (C[k] < best) { best = C[k]; arg = k; }
    sel[T - 1] = arg;
    for (int i = T - 1; i > 0; --i) sel[i - 1] = bp[(size_t)i * Kp + sel[i]];
    *best_cost = best;
    free(C); free(Cn); free(bp);
    return isinf(best) ? 3 : 0;
}

/* ------------------------------------------------------------------------- */
/* §III-C Levenberg-Marquardt                                                */
/* ------------------------------------------------------------------------- */
/* Matrix logarithm of a rotation as a rotation vector w (|w| = angle).
 * Reading of the r_pose rotation rows: the paper subtracts roll/pitch/yaw
 * elementwise; this oracle uses the world-frame rotation vector log(Rt R^T),
 * which matches the geometric Jacobian and has no gimbal or wrap issue.
 * Small angles (< 1e-6) use w = vee(M - M^T)/2 (theta/sin(theta) -> 1); angles
 * within 1e-6 of pi take the axis from the largest diagonal of (M + I)/2. */
void orc_log_rot(const double M[9], double w[3]) {
    double v[3] = {M[7] - M[5], M[2] - M[6], M[3] - M[1]};
    double s = 0.5 * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double c = 0.5 * (M[0] + M[4] + M[8] - 1.0);
    double th = atan2(s, c);
    if (th < 1e-6) {
        w[0] = 0.5 * v[0]; w[1] = 0.5 * v[1]; w[2] = 0.5 * v[2];
    } else if (th > M_PI - 1e-6) {
        /* M ~ 2 a a^T - I: pick the column of (M + I)/2 with the largest diagonal */
        int m = 0;
        if (M[4] > M[0]) m = 1;
        if (M[8] > M[3 * m + m]) m = 2;
        double col[3];
        for (int r = 0; r < 3; ++r) col[r] = 0.5 * (M[3 * r + m] + (r == m ? 1.0 : 0.0));
        double nrm = sqrt(col[0] * col[0] + col[1] * col[1] + col[2] * col[2]);
        double sgn = (col[0] * v[0] + col[1] * v[1] + col[2] * v[2]) < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < 3; ++r) w[r] = sgn * th * col[r] / nrm;
    } else {
        double f = th / (2.0 * s);
        w[0] = f * v[0]; w[1] = f * v[1]; w[2] = f * v[2];
    }
}

/* Geometric Jacobian in the world frame, 6 x n row-major:
 * column j = [z_j x (p_e - o_j); z_j] for revolute joint j (§III-C "kinematic
 * Jacobian"). */
void orc_jacobian(const orc_robot* r, const double* q, double J[]) {
    double z[ORC_MAXJ + 1][3], o[ORC_MAXJ + 1][3], R[9], p[3];
    const int n = r->n;
    orc_fk_frames(r, q, z, o, R, p);
    for (int j = 0; j < n; ++j) {
        double dx = p[0] - o[j][0], dy = p[1] - o[j][1], dz = p[2] - o[j][2];
        J[0 * n + j] = z[j][1] * dz - z[j][2] * dy;
        J[1 * n + j] = z[j][2] * dx - z[j][0] * dz;
        J[2 * n + j] = z[j][0] * dy - z[j][1] * dx;
        J[3 * n + j] = z[j][0];
        J[4 * n + j] = z[j][1];
        J[5 * n + j] = z[j][2];
    }
}

/* r_pose rows for one waypoint (§III-C), as target minus current:
 * e = [p_t - p(q); log(R_t R(q)^T)]. */
void orc_residual(const orc_robot* r, const double* q, const double* t7, double e[6]) {
    double R[9], p[3], Rt[9], pt[3], M[9];
    orc_fk(r, q, R, p);
    target_pose(t7, Rt, pt);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Rt[3 * a + k] * R[3 * b + k];
            M[3 * a + b] = s;
        }
    e[0] = pt[0] - p[0]; e[1] = pt[1] - p[1]; e[2] = pt[2] - p[2];
    orc_log_rot(M, e + 3);
}

static double half_sq(const double e[6]) {
    double s = 0.0;
    for (int a = 0; a < 6; ++a) s += e[a] * e[a];
    return 0.5 * s;
}

/* Solve (L L^T) x = b for SPD A (n x n, row-major) by Cholesky. Returns 0 on a
 * non-positive or non-finite pivot. */
static int chol_solve(int n, const double* A, const double* b, double* x) {
    double L[ORC_MAXJ * ORC_MAXJ];
    memset(L, 0, sizeof(L));
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0) || !isfinite(s)) return 0;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    double y[ORC_MAXJ];
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
        y[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
    return 1;
}

/* §III-C: LM on r_pose. Because each waypoint's pose residual depends on that
 * waypoint's configuration only, J is block diagonal and every waypoint is an
 * independent n x n problem (the paper's observation; its commented text).
 * Per waypoint, seeded with q_in[i], lambda = lambda0, F = |e|^2 / 2:
 *   repeat lm_iters times:
 *     stop if F < freeze_cost
 *     J = geometric Jacobian, columns of joints outside free_mask set to 0
 *     solve (J^T J + lambda I) delta = J^T e     (the paper's update, with the
 *                                                 transpose on J restored)
 *     stop if max_j |delta_j| < freeze_step
 *     q' = clamp(q + delta, lo, hi)              (§III-C "Joint limits")
 *     if F(q') < F(q): accept, lambda = max(lambda / lambda_down, lambda_min)
 *     else:            reject, lambda = min(lambda * lambda_up, lambda_max)
 * A failed factorisation counts as a rejection. */
void orc_lm(const orc_robot* r, const orc_params* P, const double* q_in,
            const double* targets, int T, double* q_out, double* F_hist,
            int32_t* iters_run) {
    const int n = r->n;
    const int N = P->lm_iters;
    for (int i = 0; i < T; ++i) {
        const double* t7 = targets + 7 * i;
        double q[ORC_MAXJ], e[6];
        for (int j = 0; j < n; ++j) q[j] = q_in[(size_t)i * n + j];
        orc_residual(r, q, t7, e);
        double F = half_sq(e);
        double lam = P->lambda0;
        int it = 0;
        if (F_hist) F_hist[(size_t)i * (N + 1)] = F;
        for (; it < N; ++it) {
            if (F < P->freeze_cost) break;
            double J[6 * ORC_MAXJ], A[ORC_MAXJ * ORC_MAXJ], g[ORC_MAXJ], dq[ORC_MAXJ];
            orc_jacobian(r, q, J);
            for (int j = 0; j < n; ++j)
                if (!((P->free_mask >> j) & 1u))
                    for (int a = 0; a < 6; ++a) J[a * n + j] = 0.0;
            for (int a = 0; a < n; ++a) {
                for (int b = 0; b < n; ++b) {
                    double s = 0.0;
                    for (int k = 0; k < 6; ++k) s += J[k * n + a] * J[k * n + b];
                    A[a * n + b] = s + (a == b ? lam : 0.0);
                }
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += J[k * n + a] * e[k];
                g[a] = s;
            }
            int ok = chol_solve(n, A, g, dq);
            if (ok) {
                double mx = 0.0;
                for (int j = 0; j < n; ++j) mx = fmax(mx, fabs(dq[j]));
                if (mx < P->freeze_step) break;
                double qn[ORC_MAXJ], en[6];
                for (int j = 0; j < n; ++j) {
                    double v = q[j] + dq[j];
                    if (v < r->lo[j]) v = r->lo[j];
                    if (v > r->hi[j]) v = r->hi[j];
                    qn[j] = v;
                }
                orc_residual(r, qn, t7, en);
                double Fn = half_sq(en);
                if (Fn < F) {
                    memcpy(q, qn, sizeof(double) * n);
                    memcpy(e, en, sizeof(e));
                    F = Fn;
                    lam = fmax(lam / P->lambda_down, P->lambda_min);
                } else {
                    lam = fmin(lam * P->lambda_up, P->lambda_max);
                }
            } else {
                lam = fmin(lam * P->lambda_up, P->lambda_max);
            }
            if (F_hist) F_hist[(size_t)i * (N + 1) + it + 1] = F;
        }
        if (F_hist)
            for (int k = it + 1; k <= N; ++k) F_hist[(size_t)i * (N + 1) + k] = F;
        if (iters_run) iters_run[i] = it;
        for (int j = 0; j < n; ++j) q_out[(size_t)i * n + j] = q[j];
    }
}

/* ------------------------------------------------------------------------- */
/* §II constraints and metrics on a finished trajectory                      */
/* ------------------------------------------------------------------------- */
/* Pose error per waypoint (FP64), joint-limit check on the exact limits, the
 * discontinuity bound per step (§II "Discontinuities", all joints revolute),
 * mjac = max over steps and joints of |dq| (§III-B, steps i = 1..n-1),
 * the summed per-step L-inf jump (the search objective), and trajectory length
 * = sum over steps and joints of |dq| (§II). valid = every check passes. */
void orc_check(const orc_robot* r, const orc_params* P, const double* q,
               const double* targets, int T, double* pose_err, orc_report* rep) {
    const int n = r->n;
    memset(rep, 0, sizeof(*rep));
    for (int i = 0; i < T; ++i) {
        double R[9], p[3], Rt[9], pt[3], pos, rot;
        orc_fk(r, q + (size_t)i * n, R, p);
        target_pose(targets + 7 * i, Rt, pt);
        orc_pose_error(Rt, pt, R, p, &pos, &rot);
        if (pose_err) { pose_err[2 * i] = pos; pose_err[2 * i + 1] = rot; }
        rep->max_pos = fmax(rep->max_pos, pos);
        rep->max_rot = fmax(rep->max_rot, rot);
        if (!(pos <= P->tau_pos && rot <= P->tau_rot)) rep->n_pose_fail++;
        int out = 0;
        for (int j = 0; j < n; ++j) {
            double v = q[(size_t)i * n + j];
            if (!(v >= r->lo[j] && v <= r->hi[j])) out = 1;
        }
        rep->n_limit_fail += out;
        if (i + 1 < T) {
            double linf = 0.0;
            for (int j = 0; j < n; ++j) {
                double dq = fabs(q[(size_t)(i + 1) * n + j] - q[(size_t)i * n + j]);
                linf = fmax(linf, dq);
                rep->traj_len += dq;
            }
            rep->mjac = fmax(rep->mjac, linf);
            rep->sum_linf += linf;
            if (linf > P->jump_max) rep->n_jump_fail++;
        }
    }
    rep->valid = (rep->n_pose_fail == 0 && rep->n_limit_fail == 0 && rep->n_jump_fail == 0);
}

/* ------------------------------------------------------------------------- */
/* §III-C non-stationary objective: the trajectory-length (differencing) step */
/* ------------------------------------------------------------------------- */

/* Cholesky factor L (lower, row-major) of an SPD n x n matrix; 0 on a
 * non-positive or non-finite pivot. */
static int chol_factor(int n, const double* A, double* L) {
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0) || !isfinite(s)) return 0;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / L[j * n + j];
        }
    }
    return 1;
}

/* x = (L L^T)^{-1} b */
static void chol_apply(int n, const double* L, const double* b, double* x) {
    double y[ORC_MAXJ];
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
        y[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
}

/* Block-tridiagonal SPD solve by block Cholesky (the block Thomas algorithm),
 * FP64. Diagonal blocks Dg[i] (i = 0..T-1), upper blocks Off[i] = A_{i,i+1} =
 * A_{i+1,i}^T (i = 0..T-2), all n x n row-major:
 *   S_0 = Dg[0],  S_i = Dg[i] - Off[i-1]^T S_{i-1}^{-1} Off[i-1]
 *   y_0 = b_0,    y_i = b_i  - Off[i-1]^T S_{i-1}^{-1} y_{i-1}
 *   x_{T-1} = S_{T-1}^{-1} y_{T-1},  x_i = S_i^{-1} (y_i - Off[i] x_{i+1})
 * Returns 0 if some S_i is not positive definite. */
int orc_block_tridiag_solve(int T, int n, const double* Dg, const double* Off, const double* b,
                            double* x) {
    const size_t nn = (size_t)n * n;
    double* Lf = (double*)malloc(sizeof(double) * nn * (size_t)T);
    double* y = (double*)malloc(sizeof(double) * (size_t)n * T);
    int ok = 1;
    for (int i = 0; i < T && ok; ++i) {
        double S[ORC_MAXJ * ORC_MAXJ];
        memcpy(S, Dg + nn * i, sizeof(double) * nn);
        memcpy(y + (size_t)n * i, b + (size_t)n * i, sizeof(double) * n);
        if (i > 0) {
            const double* B = Off + nn * (i - 1);      /* A_{i-1,i} */
            const double* Lp = Lf + nn * (i - 1);
            /* Z = S_{i-1}^{-1} B column by column; S -= B^T Z */
            double Z[ORC_MAXJ * ORC_MAXJ], col[ORC_MAXJ], zc[ORC_MAXJ];
            for (int c = 0; c < n; ++c) {
                for (int r = 0; r < n; ++r) col[r] = B[r * n + c];
                chol_apply(n, Lp, col, zc);
                for (int r = 0; r < n; ++r) Z[r * n + c] = zc[r];
            }
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < n; ++c) {
                    double t = 0.0;
                    for (int r = 0; r < n; ++r) t += B[r * n + a] * Z[r * n + c];
                    S[a * n + c] -= t;
                }
            /* y_i -= B^T S_{i-1}^{-1} y_{i-1} */
            double w[ORC_MAXJ];
            chol_apply(n, Lp, y + (size_t)n * (i - 1), w);
            for (int a = 0; a < n; ++a) {
                double t = 0.0;
                for (int r = 0; r < n; ++r) t += B[r * n + a] * w[r];
                y[(size_t)n * i + a] -= t;
            }
        }
        ok = chol_factor(n, S, Lf + nn * i);
    }
    if (ok) {
        for (int i = T - 1; i >= 0; --i) {
            double rhs[ORC_MAXJ];
            for (int a = 0; a < n; ++a) rhs[a] = y[(size_t)n * i + a];
            if (i + 1 < T) {
                const double* B = Off + nn * i;        /* A_{i,i+1} */
                for (int a = 0; a < n; ++a) {
                    double t = 0.0;
                    for (int c = 0; c < n; ++c) t += B[a * n + c] * x[(size_t)n * (i + 1) + c];
                    rhs[a] -= t;
                }
            }
            chol_apply(n, Lf + nn * i, rhs, x + (size_t)n * i);
        }
    }
    free(Lf);
    free(y);
    return ok;
}

/* §III-C "Trajectory length": one LM step on the differencing residual
 * r_diff = [q_{i+1} - q_i], i = 0..T-2 (the collision rows of r_diff are not
 * built). Row block i of its Jacobian holds -I at waypoint i and +I at i+1, so
 *   J^T J + lambda_d I: diagonal blocks (c_i + lambda_d) I with c_i the number
 *     of differences that touch waypoint i (1 at the ends, 2 inside, 0 if
 *     T = 1), off-diagonal blocks -I;
 *   J^T r_diff: block i = (q_i - q_{i-1}) - (q_{i+1} - q_i), absent terms 0;
 *   delta = -(J^T J + lambda_d I)^{-1} J^T r_diff   (orc_block_tridiag_solve),
 *   q' = clamp(q + delta, lo, hi).
 * The residual is linear, so before the clamp the step lowers |r_diff|^2 / 2
 * for any lambda_d > 0. Returns 0 if the solve failed (q' = q). */
int orc_diff_step(const orc_robot* r, const double* q_in, int T, double lambda_d,
                  double* q_out) {
    const int n = r->n;
    const size_t nn = (size_t)n * n;
    double* Dg = (double*)calloc(nn * (size_t)T, sizeof(double));
    double* Off = (double*)calloc(nn * (size_t)(T > 1 ? T - 1 : 1), sizeof(double));
    double* g = (double*)calloc((size_t)n * T, sizeof(double));
    double* d = (double*)calloc((size_t)n * T, sizeof(double));
    for (int i = 0; i < T; ++i) {
        const double c = (i > 0 ? 1.0 : 0.0) + (i + 1 < T ? 1.0 : 0.0);
        for (int a = 0; a < n; ++a) Dg[nn * i + (size_t)a * n + a] = c + lambda_d;
        if (i + 1 < T)
            for (int a = 0; a < n; ++a) Off[nn * i + (size_t)a * n + a] = -1.0;
        for (int a = 0; a < n; ++a) {
            double t = 0.0;
            if (i > 0) t += q_in[(size_t)i * n + a] - q_in[(size_t)(i - 1) * n + a];
            if (i + 1 < T) t -= q_in[(size_t)(i + 1) * n + a] - q_in[(size_t)i * n + a];
            g[(size_t)i * n + a] = -t;   /* right-hand side -J^T r_diff */
        }
    }
    const int ok = orc_block_tridiag_solve(T, n, Dg, Off, g, d);
    for (int i = 0; i < T; ++i)
        for (int a = 0; a < n; ++a) {
            double v = q_in[(size_t)i * n + a] + (ok ? d[(size_t)i * n + a] : 0.0);
            if (v < r->lo[a]) v = r->lo[a];
            if (v > r->hi[a]) v = r->hi[a];
            q_out[(size_t)i * n + a] = ok ? v : q_in[(size_t)i * n + a];
        }
    free(Dg); free(Off); free(g); free(d);
    return ok;
}

/* The trajectory-length step with the collision rows of r_diff (§III-C): one
 * damped Gauss-Newton step on |r_diff|^2 / 2 with r_diff = [differences;
 * collision rows of every waypoint]. The collision rows of waypoint i touch q_i
 * only, so they add J_c,i^T J_c,i to diagonal block i and J_c,i^T r_c,i to the
 * right-hand side; the system stays block tridiagonal (now with full diagonal
 * blocks) and is solved by orc_block_tridiag_solve. Returns 0 if the solve
 * failed (q' = q). rows_out (or 0) receives the number of collision rows. */
int orc_diff_step_geo(const orc_robot* r, const orc_geometry* g, const double* q_in, int T,
                      double lambda_d, double d_safe, double w, double* q_out, int32_t* rows_out) {
    const int n = r->n;
    const size_t nn = (size_t)n * n;
    const int max_rows = ORC_MAX_PAIRS + ORC_MAX_CAPS * ORC_MAX_BOXES;
    double* Dg = (double*)calloc(nn * (size_t)T, sizeof(double));
    double* Off = (double*)calloc(nn * (size_t)(T > 1 ? T - 1 : 1), sizeof(double));
    double* gr = (double*)calloc((size_t)n * T, sizeof(double));
    double* d = (double*)calloc((size_t)n * T, sizeof(double));
    double* res = (double*)malloc(sizeof(double) * max_rows);
    double* J = (double*)malloc(sizeof(double) * (size_t)max_rows * n);
    int32_t rows = 0;
    for (int i = 0; i < T; ++i) {
        const double c = (i > 0 ? 1.0 : 0.0) + (i + 1 < T ? 1.0 : 0.0);
        for (int a = 0; a < n; ++a) Dg[nn * i + (size_t)a * n + a] = c + lambda_d;
        if (i + 1 < T)
            for (int a = 0; a < n; ++a) Off[nn * i + (size_t)a * n + a] = -1.0;
        for (int a = 0; a < n; ++a) {
            double t = 0.0;
            if (i > 0) t += q_in[(size_t)i * n + a] - q_in[(size_t)(i - 1) * n + a];
            if (i + 1 < T) t -= q_in[(size_t)(i + 1) * n + a] - q_in[(size_t)i * n + a];
            gr[(size_t)i * n + a] = -t;
        }
        const int m = orc_collision_rows(r, g, q_in + (size_t)i * n, d_safe, w, res, J, max_rows);
        rows += m;
        for (int k = 0; k < m; ++k)
            for (int a = 0; a < n; ++a) {
                gr[(size_t)i * n + a] -= J[(size_t)k * n + a] * res[k];
                for (int b = 0; b < n; ++b)
                    Dg[nn * i + (size_t)a * n + b] += J[(size_t)k * n + a] * J[(size_t)k * n + b];
            }
    }
    const int ok = orc_block_tridiag_solve(T, n, Dg, Off, gr, d);
    for (int i = 0; i < T; ++i)
        for (int a = 0; a < n; ++a) {
            double v = q_in[(size_t)i * n + a] + (ok ? d[(size_t)i * n + a] : 0.0);
            if (v < r->lo[a]) v = r->lo[a];
            if (v > r->hi[a]) v = r->hi[a];
            q_out[(size_t)i * n + a] = ok ? v : q_in[(size_t)i * n + a];
        }
    if (rows_out) *rows_out = rows;
    free(Dg); free(Off); free(gr); free(d); free(res); free(J);
    return ok;
}

/* §III-C non-stationary objective: pose-only LM phases (orc_lm) alternate with
 * single trajectory-length steps; a trajectory-length step is taken only when
 * the pose phase before it left every waypoint within tau_pos / tau_rot (FP64
 * check), and the sequence ends with a pose phase:
 *   q = q_in
 *   repeat rounds times: q = lm(q); if every waypoint is within tau:
 *                        q = diff_step(q, lambda_d), taken += 1
 *   q = lm(q)
 * Each pose phase starts from lambda0 (orc_lm). */
void orc_lm_smooth(const orc_robot* r, const orc_params* P, const double* q_in,
                   const double* targets, int T, int rounds, double lambda_d, double* q_out,
                   int32_t* taken) {
    const int n = r->n;
    double* q = (double*)malloc(sizeof(double) * (size_t)T * n);
    double* w = (double*)malloc(sizeof(double) * (size_t)T * n);
    memcpy(q, q_in, sizeof(double) * (size_t)T * n);
    int32_t cnt = 0;
    for (int k = 0; k < rounds; ++k) {
        orc_lm(r, P, q, targets, T, w, 0, 0);
        orc_report rep;
        orc_check(r, P, w, targets, T, 0, &rep);
        if (rep.n_pose_fail == 0) {
            orc_diff_step(r, w, T, lambda_d, q);
            ++cnt;
        } else {
            memcpy(q, w, sizeof(double) * (size_t)T * n);
        }
    }
    orc_lm(r, P, q, targets, T, q_out, 0, 0);
    if (taken) *taken = cnt;
    free(q); free(w);
}

/* orc_lm_smooth with the collision rows in every trajectory-length step
 * (orc_diff_step_geo); g = 0 gives orc_lm_smooth. */
void orc_lm_smooth_geo(const orc_robot* r, const orc_params* P, const orc_geometry* g,
                       const double* q_in, const double* targets, int T, int rounds,
                       double lambda_d, double d_safe, double w, double* q_out, int32_t* taken) {
    const int n = r->n;
    double* q = (double*)malloc(sizeof(double) * (size_t)T * n);
    double* v = (double*)malloc(sizeof(double) * (size_t)T * n);
    memcpy(q, q_in, sizeof(double) * (size_t)T * n);
    int32_t cnt = 0;
    for (int k = 0; k < rounds; ++k) {
        orc_lm(r, P, q, targets, T, v, 0, 0);
        orc_report rep;
        orc_check(r, P, v, targets, T, 0, &rep);
        if (rep.n_pose_fail == 0) {
            if (g) orc_diff_step_geo(r, g, v, T, lambda_d, d_safe, w, q, 0);
            else orc_diff_step(r, v, T, lambda_d, q);
            ++cnt;
        } else {
            memcpy(q, v, sizeof(double) * (size_t)T * n);
        }
    }
    orc_lm(r, P, q, targets, T, q_out, 0, 0);
    if (taken) *taken = cnt;
    free(q); free(v);
}

/* ------------------------------------------------------------------------- */
/* cpf-BatchOpt (§III, commented text): optimise the smoothest lanes directly */
/* ------------------------------------------------------------------------- */
/* Lane k across the waypoints is one of the K candidate trajectories. Its
 * smoothness is its mjac, max over steps and joints of |q_{i+1,k,j} - q_{i,k,j}|,
 * formed in FP32 (an IEEE subtraction and exact max); a lane with a non-finite
 * value gets +inf. */
void orc_lane_mjac_f32(const float* cand, int T, int K, int Kp, int n, float* mjac) {
    for (int k = 0; k < K; ++k) {
        float m = 0.0f;
        int finite = 1;
        for (int i = 0; i < T; ++i)
            for (int j = 0; j < n; ++j) {
                const float v = cand[((size_t)i * n + j) * Kp + k];
                if (!isfinite(v)) finite = 0;
                if (i + 1 < T) {
                    const float d = fabsf(cand[((size_t)(i + 1) * n + j) * Kp + k] - v);
                    if (d > m) m = d;
                }
            }
        mjac[k] = finite ? m : INFINITY;
    }
}

/* The `lanes` smoothest lanes (ascending mjac, lowest index first among
 * equals), each refined by orc_lm as its own trajectory and checked by
 * orc_check; returns the position (in that order) of the first valid one, or -1.
 * q_out [lanes][T][n], reps [lanes]. */
int orc_batch_opt(const orc_robot* r, const orc_params* P, const float* cand,
                  const double* targets, int T, int K, int Kp, int lanes, int32_t* lane_sel,
                  float* lane_mjac, double* q_out, orc_report* reps) {
    const int n = r->n;
    float* m = (float*)malloc(sizeof(float) * (size_t)K);
    unsigned char* used = (unsigned char*)calloc((size_t)K, 1);
    double* seed = (double*)malloc(sizeof(double) * (size_t)T * n);
    orc_lane_mjac_f32(cand, T, K, Kp, n, m);
    int best = -1;
    for (int l = 0; l < lanes; ++l) {
        int arg = -1;
        for (int k = 0; k < K; ++k)   /* smallest unused, lowest index on ties (inf last) */
            if (!used[k] && (arg < 0 || m[k] < m[arg])) arg = k;
        used[arg] = 1;
        lane_sel[l] = arg;
        lane_mjac[l] = m[arg];
        for (int i = 0; i < T; ++i)
            for (int j = 0; j < n; ++j)
                seed[(size_t)i * n + j] = (double)cand[((size_t)i * n + j) * Kp + arg];
        double* q = q_out + (size_t)l * T * n;
        orc_lm(r, P, seed, targets, T, q, 0, 0);
        orc_check(r, P, q, targets, T, 0, &reps[l]);
        if (best < 0 && reps[l].valid) best = l;
    }
    free(m); free(used); free(seed);
    return best;
}

/* Mask -> FP32 search -> seed -> LM -> check, for one request. */
int orc_plan(const orc_robot* r, const orc_params* P, const float* cand,
             const double* targets, int T, int K, int Kp, int32_t* sel,
             float* best_cost, double* q_out, double* pose_err, orc_report* rep) {
    const int n = r->n;
    uint8_t* mask = (uint8_t*)malloc((size_t)T * Kp);
    float* pen = (float*)malloc(sizeof(float) * (size_t)T * Kp);
    double* seed = (double*)malloc(sizeof(double) * (size_t)T * n);
    orc_mask(r, P, cand, targets, T, K, Kp, mask, pen, 0);
    int st = orc_dp_f32(cand, pen, T, K, Kp, n, sel, best_cost, 0, 0);
    for (int i = 0; i < T; ++i)
        for (int j = 0; j < n; ++j)
            seed[(size_t)i * n + j] = (double)cand[((size_t)i * n + j) * Kp + sel[i]];
    orc_lm(r, P, seed, targets, T, q_out, 0, 0);
    orc_check(r, P, q_out, targets, T, pose_err, rep);
    free(mask); free(pen); free(seed);
    return st;
}
