// collide.cuh -- capsule / cuboid clearances of one configuration in FP32 (paper
// §III-B collision cost, §III-C "Robot-robot" and "Robot-environment collision
// avoidance"): the robot as capsules fixed to its DH frames, obstacles as boxes.
#pragma once

#include <math_constants.h>

#include "common.cuh"

namespace cppflow {

__device__ __forceinline__ float clamp01f(float v) { return fminf(fmaxf(v, 0.f), 1.f); }

__device__ __forceinline__ float d2_pts(const float* x, const float* y) {
  const float d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  return d0 * d0 + d1 * d1 + d2 * d2;
}

// Squared distance of segments a1 + s (b1 - a1), a2 + t (b2 - a2), s, t in [0, 1]:
// the convex QP solved by its active sets -- the interior stationary point when
// it lies in the unit square, and the four edges, each minimised by clamping its
// 1-D stationary point; the smallest directly evaluated |P - Q|^2 wins (s, t:
// its parameters).
__device__ __forceinline__ float seg_seg_d2_st(const float* a1, const float* b1, const float* a2,
                                               const float* b2, float& so, float& to) {
  float d1[3], d2[3], r[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) { d1[k] = b1[k] - a1[k]; d2[k] = b2[k] - a2[k]; r[k] = a1[k] - a2[k]; }
  const float A = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
  const float C = d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2];
  const float B = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
  const float D = d1[0] * r[0] + d1[1] * r[1] + d1[2] * r[2];
  const float E = d2[0] * r[0] + d2[1] * r[1] + d2[2] * r[2];
  float cs[5], ct[5];
  const float det = A * C - B * B;
  const float si = (B * E - C * D) / det, ti = (A * E - B * D) / det;
  const bool inner = det > 1e-12f * A * C && si >= 0.f && si <= 1.f && ti >= 0.f && ti <= 1.f;
  cs[0] = inner ? si : 0.f;                 ct[0] = inner ? ti : 0.f;
  cs[1] = 0.f;                              ct[1] = C > 0.f ? clamp01f(E / C) : 0.f;
  cs[2] = 1.f;                              ct[2] = C > 0.f ? clamp01f((B + E) / C) : 0.f;
  cs[3] = A > 0.f ? clamp01f(-D / A) : 0.f; ct[3] = 0.f;
  cs[4] = A > 0.f ? clamp01f((B - D) / A) : 0.f; ct[4] = 1.f;
  float best = CUDART_INF_F;
  so = to = 0.f;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float P[3], Q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { P[k] = a1[k] + cs[c] * d1[k]; Q[k] = a2[k] + ct[c] * d2[k]; }
    const float f = d2_pts(P, Q);
    if (f < best) { best = f; so = cs[c]; to = ct[c]; }
  }
  return best;
}

__device__ __forceinline__ float seg_seg_d2(const float* a1, const float* b1, const float* a2,
                                            const float* b2) {
  float s, t;
  return seg_seg_d2_st(a1, b1, a2, b2, s, t);
}

__device__ __forceinline__ float box_g(const float* a, const float* d, const float* h, float t) {
  float g = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float x = a[k] + t * d[k];
    const float e = x > h[k] ? x - h[k] : (x < -h[k] ? x + h[k] : 0.f);
    g += e * e;
  }
  return g;
}

__device__ __forceinline__ void cswap(float& x, float& y) {
  const float lo = fminf(x, y), hi = fmaxf(x, y);
  x = lo;
  y = hi;
}

// Squared distance of the segment a + t (b - a), t in [0, 1], to the box [-h, h]
// (box frame): for fixed t the nearest box point is the clamped point, so the
// cost is convex and piecewise quadratic in t with breakpoints where a
// coordinate crosses a face plane; each piece's quadratic (faces fixed by its
// midpoint) is minimised by clamping its stationary point to the piece, and the
// piece's ends are evaluated too (to: the minimiser). The eight breakpoints
// (0, 1 and the six crossings, those outside (0, 1) moved to 1) are sorted by a
// fixed network in registers; empty pieces cost nothing but an evaluation.
__device__ __forceinline__ float seg_box_d2_t(const float* a, const float* b, const float* h,
                                              float& to) {
  float d[3], br[8];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = b[k] - a[k];
  br[0] = 0.f;
  br[1] = 1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float t0 = d[k] != 0.f ? (-h[k] - a[k]) / d[k] : 1.f;
    const float t1 = d[k] != 0.f ? (h[k] - a[k]) / d[k] : 1.f;
    br[2 + 2 * k] = (t0 > 0.f && t0 < 1.f) ? t0 : 1.f;
    br[3 + 2 * k] = (t1 > 0.f && t1 < 1.f) ? t1 : 1.f;
  }
  // Batcher's odd-even merge sort for 8 keys (19 compare-exchanges)
  cswap(br[0], br[1]); cswap(br[2], br[3]); cswap(br[4], br[5]); cswap(br[6], br[7]);
  cswap(br[0], br[2]); cswap(br[1], br[3]); cswap(br[4], br[6]); cswap(br[5], br[7]);
  cswap(br[1], br[2]); cswap(br[5], br[6]);
  cswap(br[0], br[4]); cswap(br[1], br[5]); cswap(br[2], br[6]); cswap(br[3], br[7]);
  cswap(br[2], br[4]); cswap(br[3], br[5]);
  cswap(br[1], br[2]); cswap(br[3], br[4]); cswap(br[5], br[6]);
  float best = box_g(a, d, h, 0.f);
  to = 0.f;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const float ta = br[i], tz = br[i + 1], tm = 0.5f * (ta + tz);
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float x = a[k] + tm * d[k];
      const float c = x > h[k] ? h[k] : (x < -h[k] ? -h[k] : x);
      const float on = x != c ? 1.f : 0.f;   // the face of coordinate k is active
      num += on * d[k] * (c - a[k]);
      den += on * d[k] * d[k];
    }
    const float gz = box_g(a, d, h, tz);
    if (gz < best) { best = gz; to = tz; }
    const float ts = den > 0.f ? fminf(fmaxf(num / den, ta), tz) : tz;
    const float gs = box_g(a, d, h, ts);
    if (gs < best) { best = gs; to = ts; }
  }
  return best;
}

__device__ __forceinline__ float seg_box_d2(const float* a, const float* b, const float* h) {
  float t;
  return seg_box_d2_t(a, b, h, t);
}

// World end points of the capsules of frame f, given that frame's pose.
__device__ __forceinline__ void place_caps(const GeoF& g, int f, const float R[9], const float p[3],
                                           float (*cA)[3], float (*cB)[3]) {
  for (int c = g.frame_begin[f]; c < g.frame_begin[f + 1]; ++c) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cA[c][k] = R[3 * k] * g.a[c][0] + R[3 * k + 1] * g.a[c][1] + R[3 * k + 2] * g.a[c][2] + p[k];
      cB[c][k] = R[3 * k] * g.b[c][0] + R[3 * k + 1] * g.b[c][1] + R[3 * k + 2] * g.b[c][2] + p[k];
    }
  }
}

// Bounding spheres of capsule c (about its segment midpoint m) and of box o
// overlap, widened by `extra`; otherwise their clearance is at least `extra`.
__device__ __forceinline__ bool spheres_meet(const float* mu, float Ru, const float* mv, float Rv,
                                             float extra) {
  const float s = Ru + Rv + extra;
  return d2_pts(mu, mv) < s * s;
}

// Whether the smallest clearance is negative (the mask's COLLIDE decision): the
// exact QP runs only for pairs whose bounding spheres overlap, and the search
// stops at the first negative clearance. Same decision as clearance() < 0 (a
// pair whose spheres do not overlap has a positive clearance).
// Axis-aligned boxes of a capsule's segment grown by `grow` (its radius plus any
// margin): disjoint boxes mean a clearance of at least the margin.
__device__ __forceinline__ bool aabb_meet(const float* a1, const float* b1, float g1,
                                          const float* a2, const float* b2, float g2) {
  bool meet = true;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float lo1 = fminf(a1[q], b1[q]) - g1, hi1 = fmaxf(a1[q], b1[q]) + g1;
    const float lo2 = fminf(a2[q], b2[q]) - g2, hi2 = fmaxf(a2[q], b2[q]) + g2;
    meet = meet && lo1 <= hi2 && lo2 <= hi1;
  }
  return meet;
}

// A capsule segment (box frame) grown by `grow` against the box [-h, h].
__device__ __forceinline__ bool aabb_box_meet(const float* a, const float* b, float grow,
                                              const float* h) {
  bool meet = true;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    meet = meet && fminf(a[q], b[q]) - grow <= h[q] && fmaxf(a[q], b[q]) + grow >= -h[q];
  return meet;
}

__device__ __forceinline__ void to_box(const GeoF& g, int o, const float* x, float* y) {
#pragma unroll
  for (int q = 0; q < 3; ++q)
    y[q] = g.Rt[o][3 * q] * (x[0] - g.p[o][0]) + g.Rt[o][3 * q + 1] * (x[1] - g.p[o][1]) +
           g.Rt[o][3 * q + 2] * (x[2] - g.p[o][2]);
}

__device__ __forceinline__ bool collides(const GeoF& g, const float (*cA)[3], const float (*cB)[3]) {
  for (int k = 0; k < g.n_pairs; ++k) {
    const int u = g.pu[k], v = g.pv[k];
    if (!aabb_meet(cA[u], cB[u], g.r[u] + 1e-5f, cA[v], cB[v], g.r[v] + 1e-5f)) continue;
    if (sqrtf(seg_seg_d2(cA[u], cB[u], cA[v], cB[v])) - g.r[u] - g.r[v] < 0.f) return true;
  }
  // capsule-box: disjoint bounding spheres first (both radii carry 1e-5 m of
  // slack), then the box-frame bounding boxes, then the exact distance
  for (int c = 0; c < g.n_caps; ++c) {
    float m[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) m[q] = 0.5f * (cA[c][q] + cB[c][q]);
    for (int o = 0; o < g.n_boxes; ++o) {
      if (!spheres_meet(m, g.bound[c], g.p[o], g.box_bound[o], 0.f)) continue;
      float a[3], b[3];
      to_box(g, o, cA[c], a);
      to_box(g, o, cB[c], b);
      if (!aabb_box_meet(a, b, g.r[c] + 1e-5f, g.h[o])) continue;
      if (sqrtf(seg_box_d2(a, b, g.h[o])) - g.r[c] < 0.f) return true;
    }
  }
  return false;
}

// Smallest clearance over the listed pairs (segment distance - r_u - r_v) and over
// every capsule and box (segment-box distance - r_c); +inf when both lists are
// empty. A pair's exact distance is computed only when its bounding-sphere lower
// bound is below the running minimum, so the result is the exact minimum.
__device__ __forceinline__ float clearance(const GeoF& g, const float (*cA)[3],
                                           const float (*cB)[3]) {
  float cl = CUDART_INF_F;
  for (int k = 0; k < g.n_pairs; ++k) {
    const int u = g.pu[k], v = g.pv[k];
    float mu[3], mv[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) { mu[q] = 0.5f * (cA[u][q] + cB[u][q]); mv[q] = 0.5f * (cA[v][q] + cB[v][q]); }
    const float lb = sqrtf(d2_pts(mu, mv)) - 0.5f * sqrtf(d2_pts(cA[u], cB[u])) -
                     0.5f * sqrtf(d2_pts(cA[v], cB[v])) - g.r[u] - g.r[v];
    if (lb >= cl) continue;
    cl = fminf(cl, sqrtf(seg_seg_d2(cA[u], cB[u], cA[v], cB[v])) - g.r[u] - g.r[v]);
  }
  for (int o = 0; o < g.n_boxes; ++o) {
    const float hr = sqrtf(g.h[o][0] * g.h[o][0] + g.h[o][1] * g.h[o][1] + g.h[o][2] * g.h[o][2]);
    for (int c = 0; c < g.n_caps; ++c) {
      float a[3], b[3], m[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) m[q] = 0.5f * (cA[c][q] + cB[c][q]);
      const float lb = sqrtf(d2_pts(m, g.p[o])) - 0.5f * sqrtf(d2_pts(cA[c], cB[c])) - hr - g.r[c];
      if (lb >= cl) continue;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        a[q] = g.Rt[o][3 * q] * (cA[c][0] - g.p[o][0]) + g.Rt[o][3 * q + 1] * (cA[c][1] - g.p[o][1]) +
               g.Rt[o][3 * q + 2] * (cA[c][2] - g.p[o][2]);
        b[q] = g.Rt[o][3 * q] * (cB[c][0] - g.p[o][0]) + g.Rt[o][3 * q + 1] * (cB[c][1] - g.p[o][1]) +
               g.Rt[o][3 * q + 2] * (cB[c][2] - g.p[o][2]);
      }
      cl = fminf(cl, sqrtf(seg_box_d2(a, b, g.h[o])) - g.r[c]);
    }
  }
  return cl;
}

}  // namespace cppflow
