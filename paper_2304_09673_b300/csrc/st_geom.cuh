// st_geom.cuh -- FP32 ray generation and ray / volume-of-interest interval
// tests with a fixed operation order: every arithmetic step is one IEEE
// round-to-nearest operation (explicit __f*_rn intrinsics, no contraction),
// so the culling decisions are reproducible bit for bit on any host that
// follows the same order.
#pragma once
#include <cuda_runtime.h>

#include "st_internal.h"

namespace st {

__device__ __forceinline__ float ieee_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ieee_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ieee_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ieee_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ieee_sqrt(float a) { return __fsqrt_rn(a); }
// (a0 b0 + a1 b1) + a2 b2
__device__ __forceinline__ float ieee_dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
  return ieee_add(ieee_add(ieee_mul(a0, b0), ieee_mul(a1, b1)), ieee_mul(a2, b2));
}

// Pixel-centre ray direction of pixel (i, j) (see st_camera in st.h).
__device__ __forceinline__ void pixel_ray(const DevCamera &c, int i, int j, float d[3]) {
  float u = ieee_sub(ieee_div((float)(2 * i + 1), (float)c.W), 1.0f);
  float v = ieee_sub(1.0f, ieee_div((float)(2 * j + 1), (float)c.H));
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = ieee_add(ieee_add(c.F[k], ieee_mul(u, c.R[k])), ieee_mul(v, c.U[k]));
}

// Sphere (centre c, radius r) against ray o + t d: closest-approach form.
// w = c - o, tc = (w.d)/(d.d), q = w - tc d, h2 = q.q; miss if h2 > r^2;
// s = sqrt((r^2 - h2)/(d.d)); [tc - s, tc + s].  `w` is ray independent.
__device__ __forceinline__ bool ray_sphere32(const float w[3], const float d[3], float r,
                                             float &t0, float &t1) {
  float dd = ieee_dot3(d[0], d[1], d[2], d[0], d[1], d[2]);
  float wd = ieee_dot3(w[0], w[1], w[2], d[0], d[1], d[2]);
  float tc = ieee_div(wd, dd);
  float qx = ieee_sub(w[0], ieee_mul(tc, d[0]));
  float qy = ieee_sub(w[1], ieee_mul(tc, d[1]));
  float qz = ieee_sub(w[2], ieee_mul(tc, d[2]));
  float h2 = ieee_dot3(qx, qy, qz, qx, qy, qz);
  float r2 = ieee_mul(r, r);
  if (h2 > r2) return false;
  float s = ieee_sqrt(ieee_div(ieee_sub(r2, h2), dd));
  t0 = ieee_sub(tc, s);
  t1 = ieee_add(tc, s);
  return true;
}

// Oriented box: slabs in the local frame.  lo[i] = M_i . (o - c) (ray
// independent), ld_i = M_i . d, e = half extents.
__device__ __forceinline__ bool ray_obox32(const float lo[3], const float M[9], const float e[3],
                                           const float d[3], float &t0, float &t1) {
  float a_lo = -INFINITY, a_hi = INFINITY;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float ld = ieee_dot3(M[3 * i], M[3 * i + 1], M[3 * i + 2], d[0], d[1], d[2]);
    if (ld == 0.0f) {
      if (lo[i] < -e[i] || lo[i] > e[i]) return false;
      continue;
    }
    float ta = ieee_div(ieee_sub(-e[i], lo[i]), ld);
    float tb = ieee_div(ieee_sub(e[i], lo[i]), ld);
    float a = ta < tb ? ta : tb;
    float b = ta < tb ? tb : ta;
    if (a > a_lo) a_lo = a;
    if (b < a_hi) a_hi = b;
  }
  if (a_lo > a_hi) return false;
  t0 = a_lo;
  t1 = a_hi;
  return true;
}

// Capsule (a, b, r): hull of the intervals of the two end spheres and of the
// cylinder between the end planes.  Ray-independent inputs: wa = a - o,
// wb = b - o (sphere form), w = o - a, ba = b - a, bb = ba.ba, wbv = w.ba,
// fw = wbv / bb, p = w - fw ba.
struct CapsuleConst {
  float wa[3], wb[3], ba[3], p[3];
  float bb, wbv, r;
};

// The cylinder part of the capsule test: radius k.r around [a, b], capped by
// the planes through the ends (also the volume of interest of a torus).
__device__ __forceinline__ bool ray_cylinder32(const CapsuleConst &k, const float d[3], float &t0, float &t1) {
  if (!(k.bb > 0.0f)) return false;
  float db = ieee_dot3(d[0], d[1], d[2], k.ba[0], k.ba[1], k.ba[2]);
  float fd = ieee_div(db, k.bb);
  float ux = ieee_sub(d[0], ieee_mul(fd, k.ba[0]));
  float uy = ieee_sub(d[1], ieee_mul(fd, k.ba[1]));
  float uz = ieee_sub(d[2], ieee_mul(fd, k.ba[2]));
  float A = ieee_dot3(ux, uy, uz, ux, uy, uz);
  float r2 = ieee_mul(k.r, k.r);
  float c0 = -INFINITY, c1 = INFINITY;
  if (A > 0.0f) {
    float pu = ieee_dot3(k.p[0], k.p[1], k.p[2], ux, uy, uz);
    float tc = -ieee_div(pu, A);
    float hx = ieee_add(k.p[0], ieee_mul(tc, ux));
    float hy = ieee_add(k.p[1], ieee_mul(tc, uy));
    float hz = ieee_add(k.p[2], ieee_mul(tc, uz));
    float h2 = ieee_dot3(hx, hy, hz, hx, hy, hz);
    if (h2 > r2) return false;
    float s = ieee_sqrt(ieee_div(ieee_sub(r2, h2), A));
    c0 = ieee_sub(tc, s);
    c1 = ieee_add(tc, s);
  } else {
    float p2 = ieee_dot3(k.p[0], k.p[1], k.p[2], k.p[0], k.p[1], k.p[2]);
    if (p2 > r2) return false;
  }
  if (db == 0.0f) {
    if (k.wbv < 0.0f || k.wbv > k.bb) return false;
  } else {
    float ta = -ieee_div(k.wbv, db);
    float tb = ieee_div(ieee_sub(k.bb, k.wbv), db);
    float sa = ta < tb ? ta : tb;
    float sb = ta < tb ? tb : ta;
    if (sa > c0) c0 = sa;
    if (sb < c1) c1 = sb;
    if (c0 > c1) return false;
  }
  t0 = c0;
  t1 = c1;
  return true;
}

__device__ __forceinline__ bool ray_capsule32(const CapsuleConst &k, const float d[3], float &t0,
                                              float &t1) {
  float lo = INFINITY, hi = -INFINITY, s0, s1;
  if (ray_sphere32(k.wa, d, k.r, s0, s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
  if (ray_sphere32(k.wb, d, k.r, s0, s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
  if (ray_cylinder32(k, d, s0, s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
  if (lo > hi) return false;
  t0 = lo;
  t1 = hi;
  return true;
}

// Volume of interest of primitive j (Sec. 6.1: the primitive's bound offset by
// its range-of-interest bound d_prim), extents in FP32: ((size + d) + pad).
// Families: sphere (sphere); oriented box (rounded box; ellipsoid, the box
// around {f <= d}, half extents r (1 + d / min r); bounded quadric, its
// clipping box grown by d); capsule (capsule; sphere-cone with radius
// max(r_a, r_b) + d); capped cylinder (torus: radius (R + r) + d around the
// axis, half-height r + d); sphere-triangle (rounded triangle: the points
// within (r + d) of the triangle).
enum VoiFamily : int { VOI_SPHERE = 0, VOI_BOX = 1, VOI_CAPSULE = 2, VOI_CYLINDER = 3, VOI_STRI = 4 };
struct Voi {
  int fam;
  float c[3];      // centre (sphere, box), end a (capsule, cylinder), vertex a (triangle)
  float M[9];      // box rotation rows; triangle: unit normal n, edge normals m0, m1
  float e[3];      // box half extents; triangle: vertex c
  float b[3];      // capsule / cylinder end b; triangle: vertex b
  float r;         // sphere / capsule / cylinder / sphere-triangle radius
};

// Ray-independent quantities of a volume of interest seen from the eye.
// Sphere-triangle: w = o, lo3 = (g0, g1, g2), cc.r = so, cc.wa = m2.
struct VoiRay {
  float w[3], lo3[3];
  CapsuleConst cc;
};

// tri_m2: the triangle's third edge normal goes there (the volume of
// interest's ray constants); null when not needed.  kStri = false: a rounded
// triangle only gets its family (no parameters).
template <bool kStri = true>
__device__ __forceinline__ void load_voi(const DevScene &sc, uint32_t j, Voi &v, float *tri_m2 = nullptr) {
  uint32_t a = sc.prim_addr[j];
  uint32_t kind = blob_kind(sc.blob[a]);
  const float4 *w = sc.rec + sc.rec_off[a];
  float dp = sc.d_prim[j], pad = sc.voi_pad;
  float4 w0 = w[0];
  v.c[0] = w0.x; v.c[1] = w0.y; v.c[2] = w0.z;
  if (kind == ST_PRIM_SPHERE) {
    v.fam = VOI_SPHERE;
    v.r = ieee_add(ieee_add(w0.w, dp), pad);
  } else if (kind == ST_PRIM_RBOX) {
    v.fam = VOI_BOX;
    const float rr = w0.w;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float4 m = w[1 + i];
      v.M[3 * i] = m.x; v.M[3 * i + 1] = m.y; v.M[3 * i + 2] = m.z;
      v.e[i] = ieee_add(ieee_add(ieee_add(m.w, rr), dp), pad);
    }
  } else if (kind == ST_PRIM_ELLIPSOID) {
    v.fam = VOI_BOX;
    const float grow = ieee_add(1.0f, ieee_div(dp, w0.w));   // w0.w = min r
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float4 m = w[1 + i];
      v.M[3 * i] = m.x; v.M[3 * i + 1] = m.y; v.M[3 * i + 2] = m.z;
      v.e[i] = ieee_add(ieee_mul(m.w, grow), pad);
    }
  } else if (kind == ST_PRIM_QUADRIC) {
    v.fam = VOI_BOX;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float4 m = w[1 + i];
      v.M[3 * i] = m.x; v.M[3 * i + 1] = m.y; v.M[3 * i + 2] = m.z;
      v.e[i] = ieee_add(ieee_add(m.w, dp), pad);
    }
  } else if (kind == ST_PRIM_RTRI) {
    v.fam = VOI_STRI;
    if (!kStri) return;
    const float4 e0 = w[1], e2 = w[3], w4 = w[4], w5 = w[5], w6 = w[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float a = k == 0 ? w0.x : (k == 1 ? w0.y : w0.z);
      const float ek0 = k == 0 ? e0.x : (k == 1 ? e0.y : e0.z);
      const float ek2 = k == 0 ? e2.x : (k == 1 ? e2.y : e2.z);
      v.b[k] = ieee_add(a, ek0);    // b = a + e0
      v.e[k] = ieee_sub(a, ek2);    // c = a - e2
    }
    v.M[0] = w4.x; v.M[1] = w4.y; v.M[2] = w4.z;
    v.M[3] = w5.x; v.M[4] = w5.y; v.M[5] = w5.z;
    v.M[6] = w6.x; v.M[7] = w6.y; v.M[8] = w6.z;
    if (tri_m2) { tri_m2[0] = w4.w; tri_m2[1] = w5.w; tri_m2[2] = w6.w; }
    v.r = ieee_add(ieee_add(w0.w, dp), pad);
  } else if (kind == ST_PRIM_TORUS) {
    v.fam = VOI_CYLINDER;
    const float4 w1 = w[1];   // unit axis, R
    const float hh = ieee_add(ieee_add(w0.w, dp), pad);
    const float ax[3] = {w1.x, w1.y, w1.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float c = v.c[k];
      v.c[k] = ieee_sub(c, ieee_mul(hh, ax[k]));
      v.b[k] = ieee_add(c, ieee_mul(hh, ax[k]));
    }
    v.r = ieee_add(ieee_add(ieee_add(w1.w, w0.w), dp), pad);
  } else {   // capsule, sphere-cone
    v.fam = VOI_CAPSULE;
    float4 w1 = w[1];
    v.b[0] = w1.x; v.b[1] = w1.y; v.b[2] = w1.z;
    const float rad = kind == ST_PRIM_SCONE ? fmaxf(w0.w, w1.w) : w0.w;
    v.r = ieee_add(ieee_add(rad, dp), pad);
  }
}

// Capsule constants of the segment [p0, p1] with radius r seen from o.
__device__ __forceinline__ void capsule_setup(const float p0[3], const float p1[3], float r, const float o[3],
                                              CapsuleConst &cc) {
  float w[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cc.wa[i] = ieee_sub(p0[i], o[i]);
    cc.wb[i] = ieee_sub(p1[i], o[i]);
    cc.ba[i] = ieee_sub(p1[i], p0[i]);
    w[i] = ieee_sub(o[i], p0[i]);
  }
  cc.bb = ieee_dot3(cc.ba[0], cc.ba[1], cc.ba[2], cc.ba[0], cc.ba[1], cc.ba[2]);
  cc.r = r;
  cc.wbv = 0.0f;
  cc.p[0] = cc.p[1] = cc.p[2] = 0.0f;
  if (cc.bb > 0.0f) {
    cc.wbv = ieee_dot3(w[0], w[1], w[2], cc.ba[0], cc.ba[1], cc.ba[2]);
    float fw = ieee_div(cc.wbv, cc.bb);
#pragma unroll
    for (int i = 0; i < 3; ++i) cc.p[i] = ieee_sub(w[i], ieee_mul(fw, cc.ba[i]));
  }
}

// Sphere-triangle (points within r of the triangle a, b, c): the union of the
// prism over the triangle (|n.(x - a)| <= r and inside the three edge planes
// m_i.(x - v_i) <= 0) and the three edge capsules; being convex, the ray
// meets it in one interval, [least entry, greatest exit] of the pieces.
// Ray-independent inputs: so = n.(o - a), g_i = m_i.(o - v_i), m2.
__device__ __forceinline__ bool ray_stri32(const Voi &v, const float o[3], const float so, const float g[3],
                                           const float m2[3], const float d[3], float &t0, float &t1) {
  float lo = INFINITY, hi = -INFINITY, s0, s1;
  // prism: slab of the plane, then the three edge half-spaces
  {
    float a_lo = -INFINITY, a_hi = INFINITY;
    bool ok = true;
    const float sd = ieee_dot3(v.M[0], v.M[1], v.M[2], d[0], d[1], d[2]);
    if (sd == 0.0f) {
      if (so < -v.r || so > v.r) ok = false;
    } else {
      const float ta = ieee_div(ieee_sub(-v.r, so), sd);
      const float tb = ieee_div(ieee_sub(v.r, so), sd);
      a_lo = ta < tb ? ta : tb;
      a_hi = ta < tb ? tb : ta;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float *m = i == 0 ? v.M + 3 : (i == 1 ? v.M + 6 : m2);
      const float gd = ieee_dot3(m[0], m[1], m[2], d[0], d[1], d[2]);
      if (gd == 0.0f) {
        if (g[i] > 0.0f) ok = false;
      } else {
        const float tl = ieee_div(-g[i], gd);
        if (gd > 0.0f) { if (tl < a_hi) a_hi = tl; }
        else { if (tl > a_lo) a_lo = tl; }
      }
    }
    if (ok && a_lo <= a_hi) { lo = a_lo; hi = a_hi; }
  }
  // edge capsules a-b, b-c, c-a
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float *p0 = i == 0 ? v.c : (i == 1 ? v.b : v.e);
    const float *p1 = i == 0 ? v.b : (i == 1 ? v.e : v.c);
    CapsuleConst cc;
    capsule_setup(p0, p1, v.r, o, cc);
    if (ray_capsule32(cc, d, s0, s1)) { if (s0 < lo) lo = s0; if (s1 > hi) hi = s1; }
  }
  if (lo > hi) return false;
  t0 = lo;
  t1 = hi;
  return true;
}

// q.cc.wa must already hold the triangle's m2 (load_voi's tri_m2) for the
// sphere-triangle family (kStri = false: that family is not set up).
template <bool kStri = true>
__device__ __forceinline__ void voi_ray_setup(const Voi &v, const DevCamera &cam, VoiRay &q) {
  if (kStri && v.fam == VOI_STRI) {
    // w = o (for the per-ray edge capsules), lo3 = (g0, g1, g2), cc.r = so
    float oa[3], ob[3], oc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      q.w[i] = cam.o[i];
      oa[i] = ieee_sub(cam.o[i], v.c[i]);
      ob[i] = ieee_sub(cam.o[i], v.b[i]);
      oc[i] = ieee_sub(cam.o[i], v.e[i]);
    }
    q.cc.r = ieee_dot3(v.M[0], v.M[1], v.M[2], oa[0], oa[1], oa[2]);
    q.lo3[0] = ieee_dot3(v.M[3], v.M[4], v.M[5], oa[0], oa[1], oa[2]);
    q.lo3[1] = ieee_dot3(v.M[6], v.M[7], v.M[8], ob[0], ob[1], ob[2]);
    q.lo3[2] = ieee_dot3(q.cc.wa[0], q.cc.wa[1], q.cc.wa[2], oc[0], oc[1], oc[2]);
  } else if (v.fam == VOI_SPHERE) {
#pragma unroll
    for (int i = 0; i < 3; ++i) q.w[i] = ieee_sub(v.c[i], cam.o[i]);
  } else if (v.fam == VOI_BOX) {
#pragma unroll
    for (int i = 0; i < 3; ++i) q.w[i] = ieee_sub(cam.o[i], v.c[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) q.lo3[i] = ieee_dot3(v.M[3 * i], v.M[3 * i + 1], v.M[3 * i + 2], q.w[0], q.w[1], q.w[2]);
  } else {
    CapsuleConst &cc = q.cc;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cc.wa[i] = ieee_sub(v.c[i], cam.o[i]);
      cc.wb[i] = ieee_sub(v.b[i], cam.o[i]);
      cc.ba[i] = ieee_sub(v.b[i], v.c[i]);
      q.w[i] = ieee_sub(cam.o[i], v.c[i]);
    }
    cc.bb = ieee_dot3(cc.ba[0], cc.ba[1], cc.ba[2], cc.ba[0], cc.ba[1], cc.ba[2]);
    cc.r = v.r;
    if (cc.bb > 0.0f) {
      cc.wbv = ieee_dot3(q.w[0], q.w[1], q.w[2], cc.ba[0], cc.ba[1], cc.ba[2]);
      float fw = ieee_div(cc.wbv, cc.bb);
#pragma unroll
      for (int i = 0; i < 3; ++i) cc.p[i] = ieee_sub(q.w[i], ieee_mul(fw, cc.ba[i]));
    }
  }
}

// Entry and exit of the ray o + t d in the volume of interest, the entry
// clamped to t >= 0 (the eye may be inside); false when the ray misses it.
// kStri = false leaves the sphere-triangle family out (callers that test it
// on a separate path, keeping its registers off the other families' path).
template <bool kStri = true>
__device__ __forceinline__ bool voi_ray_hit(const Voi &v, const VoiRay &q, const float d[3], float &t0,
                                            float &t1) {
  bool h;
  if (v.fam == VOI_SPHERE) h = ray_sphere32(q.w, d, v.r, t0, t1);
  else if (v.fam == VOI_BOX) h = ray_obox32(q.lo3, v.M, v.e, d, t0, t1);
  else if (v.fam == VOI_CAPSULE) h = ray_capsule32(q.cc, d, t0, t1);
  else if (kStri && v.fam == VOI_STRI) h = ray_stri32(v, q.w, q.cc.r, q.lo3, q.cc.wa, d, t0, t1);
  else h = ray_cylinder32(q.cc, d, t0, t1);
  if (!h) return false;
  t0 = t0 > 0.0f ? t0 : 0.0f;
  return t1 >= t0;
}

}  // namespace st
