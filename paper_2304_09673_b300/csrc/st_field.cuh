// st_field.cuh -- field evaluation of a pruned tree view on the GPU.
//
// Node functions are written once over a numeric type T: float for the
// tracing hot loop (approximate MUFU square root / reciprocal), or a
// forward-mode dual number Dual<N> (value and N directional derivatives) for
// the Newton refinement along the ray and the normal.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "st_internal.h"

namespace st {

__device__ __forceinline__ float fsqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float frcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int N>
struct Dual {
  float v;
  float g[N];
  __device__ Dual() {}
  __device__ Dual(float x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) g[i] = 0.f;
  }
};

__device__ __forceinline__ float val(float x) { return x; }
template <int N> __device__ __forceinline__ float val(const Dual<N> &x) { return x.v; }

template <int N> __device__ __forceinline__ Dual<N> operator+(Dual<N> a, const Dual<N> &b) {
  a.v += b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) a.g[i] += b.g[i];
  return a;
}
template <int N> __device__ __forceinline__ Dual<N> operator-(Dual<N> a, const Dual<N> &b) {
  a.v -= b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) a.g[i] -= b.g[i];
  return a;
}
template <int N> __device__ __forceinline__ Dual<N> operator-(Dual<N> a) {
  a.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) a.g[i] = -a.g[i];
  return a;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
  return r;
}
template <int N> __device__ __forceinline__ Dual<N> operator+(Dual<N> a, float b) { a.v += b; return a; }
template <int N> __device__ __forceinline__ Dual<N> operator+(float b, Dual<N> a) { a.v += b; return a; }
template <int N> __device__ __forceinline__ Dual<N> operator-(Dual<N> a, float b) { a.v -= b; return a; }
template <int N> __device__ __forceinline__ Dual<N> operator-(float b, Dual<N> a) { return Dual<N>(b) - a; }
template <int N> __device__ __forceinline__ Dual<N> operator*(Dual<N> a, float b) {
  a.v *= b;
#pragma unroll
  for (int i = 0; i < N; ++i) a.g[i] *= b;
  return a;
}
template <int N> __device__ __forceinline__ Dual<N> operator*(float b, Dual<N> a) { return a * b; }

__device__ __forceinline__ float sqrt_(float x) { return fsqrt(x); }
template <int N> __device__ __forceinline__ Dual<N> sqrt_(const Dual<N> &x) {
  Dual<N> r;
  r.v = sqrtf(fmaxf(x.v, 0.f));
  float s = r.v > 0.f ? 0.5f / r.v : 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) r.g[i] = x.g[i] * s;
  return r;
}
__device__ __forceinline__ float rcp_(float x) { return frcp(x); }
template <int N> __device__ __forceinline__ Dual<N> rcp_(const Dual<N> &x) {
  Dual<N> r;
  r.v = 1.0f / x.v;
  float s = -r.v * r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.g[i] = x.g[i] * s;
  return r;
}
__device__ __forceinline__ float abs_(float x) { return fabsf(x); }
template <int N> __device__ __forceinline__ Dual<N> abs_(const Dual<N> &x) { return x.v < 0.f ? -x : x; }
__device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
template <int N> __device__ __forceinline__ Dual<N> min_(const Dual<N> &a, const Dual<N> &b) { return b.v < a.v ? b : a; }
template <int N> __device__ __forceinline__ Dual<N> max_(const Dual<N> &a, const Dual<N> &b) { return b.v > a.v ? b : a; }
template <int N> __device__ __forceinline__ Dual<N> max_(const Dual<N> &a, float b) { return b > a.v ? Dual<N>(b) : a; }
template <int N> __device__ __forceinline__ Dual<N> min_(const Dual<N> &a, float b) { return b < a.v ? Dual<N>(b) : a; }

// Explicitly rounded FP32 arithmetic.  The field is evaluated by several code
// paths (lockstep over two rays per lane, the warp-wide tail evaluation) and
// a ray's trajectory must not depend on which one steps it, so the fusion of
// products and sums into FMA is written out instead of left to the compiler.
// Dual numbers (single code path, refinement only) use their operators.
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <class A, class B> __device__ __forceinline__ auto add_(const A &a, const B &b) { return a + b; }
template <class A, class B> __device__ __forceinline__ auto sub_(const A &a, const B &b) { return a - b; }
template <class A, class B> __device__ __forceinline__ auto mul_(const A &a, const B &b) { return a * b; }
template <class A, class B, class C> __device__ __forceinline__ auto fma_(const A &a, const B &b, const C &c) {
  return a * b + c;
}

// ---- paired FP32 (Blackwell FFMA2 / FADD2 / FMUL2) -------------------------------
// Two evaluation points per thread as one float2: every arithmetic step is one
// paired instruction whose components round exactly as the scalar __fmaf_rn /
// __fadd_rn / __fmul_rn (so a ray's values do not depend on whether it is
// evaluated alone or in a pair); min / max / abs, the MUFU square root and
// reciprocal and the branches are taken per component.
struct F2 {
  float2 v;
  __device__ F2() {}
  __device__ explicit F2(float s) : v(make_float2(s, s)) {}
  __device__ F2(float2 x) : v(x) {}
};
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ F2 add_(const F2 &a, const F2 &b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 add_(const F2 &a, float b) { return F2(__fadd2_rn(a.v, bc2(b))); }
__device__ __forceinline__ F2 add_(float a, const F2 &b) { return F2(__fadd2_rn(bc2(a), b.v)); }
// a - b as a + (-1) b: the product is exact, so the fused form rounds once,
// as __fsub_rn does
__device__ __forceinline__ F2 sub_(const F2 &a, const F2 &b) { return F2(__ffma2_rn(b.v, bc2(-1.f), a.v)); }
__device__ __forceinline__ F2 sub_(const F2 &a, float b) { return F2(__fadd2_rn(a.v, bc2(-b))); }
__device__ __forceinline__ F2 sub_(float a, const F2 &b) { return F2(__ffma2_rn(b.v, bc2(-1.f), bc2(a))); }
__device__ __forceinline__ F2 mul_(const F2 &a, const F2 &b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 mul_(const F2 &a, float b) { return F2(__fmul2_rn(a.v, bc2(b))); }
__device__ __forceinline__ F2 fma_(const F2 &a, const F2 &b, const F2 &c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 fma_(const F2 &a, float b, const F2 &c) { return F2(__ffma2_rn(a.v, bc2(b), c.v)); }
__device__ __forceinline__ F2 fma_(const F2 &a, const F2 &b, float c) { return F2(__ffma2_rn(a.v, b.v, bc2(c))); }
__device__ __forceinline__ F2 fma_(const F2 &a, float b, float c) { return F2(__ffma2_rn(a.v, bc2(b), bc2(c))); }
__device__ __forceinline__ F2 operator-(const F2 &a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 min_(const F2 &a, const F2 &b) { return F2(make_float2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y))); }
__device__ __forceinline__ F2 max_(const F2 &a, const F2 &b) { return F2(make_float2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y))); }
__device__ __forceinline__ F2 min_(const F2 &a, float b) { return F2(make_float2(fminf(a.v.x, b), fminf(a.v.y, b))); }
__device__ __forceinline__ F2 max_(const F2 &a, float b) { return F2(make_float2(fmaxf(a.v.x, b), fmaxf(a.v.y, b))); }
__device__ __forceinline__ F2 abs_(const F2 &a) { return F2(make_float2(fabsf(a.v.x), fabsf(a.v.y))); }
__device__ __forceinline__ F2 sqrt_(const F2 &a) { return F2(make_float2(fsqrt(a.v.x), fsqrt(a.v.y))); }
__device__ __forceinline__ F2 rcp_(const F2 &a) { return F2(make_float2(frcp(a.v.x), frcp(a.v.y))); }

// Comparisons and selects: a bool for one point (float, dual number), a pair
// of bools for F2.
struct M2 { bool x, y; };
__device__ __forceinline__ bool le_(float a, float b) { return a <= b; }
__device__ __forceinline__ bool gt_(float a, float b) { return a > b; }
template <int N> __device__ __forceinline__ bool le_(const Dual<N> &a, float b) { return a.v <= b; }
template <int N> __device__ __forceinline__ bool gt_(const Dual<N> &a, float b) { return a.v > b; }
__device__ __forceinline__ M2 le_(const F2 &a, float b) { return M2{a.v.x <= b, a.v.y <= b}; }
__device__ __forceinline__ M2 gt_(const F2 &a, float b) { return M2{a.v.x > b, a.v.y > b}; }
__device__ __forceinline__ bool and_(bool a, bool b) { return a && b; }
__device__ __forceinline__ M2 and_(M2 a, M2 b) { return M2{a.x && b.x, a.y && b.y}; }
template <class T> __device__ __forceinline__ T sel_(bool m, const T &a, const T &b) { return m ? a : b; }
__device__ __forceinline__ F2 sel_(M2 m, const F2 &a, const F2 &b) {
  return F2(make_float2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y));
}

// Record word k of a view node: from the view's shared parameter cache or,
// for nodes that did not fit, from the scene's global record array.
struct RecSrc {
  const float4 *rec;  // global records
  const float4 *dc;   // shared parameter cache of the view (may be null)
};
__device__ __forceinline__ const float4 *rec_ptr(const RecSrc &S, uint32_t w) {
  const uint32_t off = w & kViewOffMask;
  return (w & kViewGlobal) ? S.rec + off : S.dc + off;
}
__device__ __forceinline__ float4 ldrec(const float4 *q) { return *q; }

// ---- primitives (exact SDFs, Lipschitz 1); records preloaded ----------------------
template <class T>
__device__ __forceinline__ T sd_sphere(const float4 a, const T p[3]) {
  const T dx = sub_(p[0], a.x), dy = sub_(p[1], a.y), dz = sub_(p[2], a.z);
  return sub_(sqrt_(fma_(dx, dx, fma_(dy, dy, mul_(dz, dz)))), a.w);
}

// q = |M (p - c)| - b ; |max(q, 0)| + min(max_i q_i, 0) - r_round
template <class T>
__device__ __forceinline__ T sd_rbox(const float4 a0, const float4 a1, const float4 a2, const float4 a3,
                                     const T p[3]) {
  const T wx = sub_(p[0], a0.x), wy = sub_(p[1], a0.y), wz = sub_(p[2], a0.z);
  const T q0 = sub_(abs_(fma_(wx, a1.x, fma_(wy, a1.y, mul_(wz, a1.z)))), a1.w);
  const T q1 = sub_(abs_(fma_(wx, a2.x, fma_(wy, a2.y, mul_(wz, a2.z)))), a2.w);
  const T q2 = sub_(abs_(fma_(wx, a3.x, fma_(wy, a3.y, mul_(wz, a3.z)))), a3.w);
  const T m0 = max_(q0, 0.f), m1 = max_(q1, 0.f), m2 = max_(q2, 0.f);
  const T inner = min_(max_(q0, max_(q1, q2)), 0.f);
  return sub_(add_(sqrt_(fma_(m0, m0, fma_(m1, m1, mul_(m2, m2)))), inner), a0.w);
}

// distance to segment [a, b] minus r; records [a, r] and [b - a, 1/|b-a|^2]
template <class T>
__device__ __forceinline__ T sd_capsule(const float4 a0, const float4 a2, const T p[3]) {
  const T px = sub_(p[0], a0.x), py = sub_(p[1], a0.y), pz = sub_(p[2], a0.z);
  T h = mul_(fma_(px, a2.x, fma_(py, a2.y, mul_(pz, a2.z))), a2.w);
  h = min_(max_(h, 0.f), 1.f);
  const T dx = fma_(h, -a2.x, px), dy = fma_(h, -a2.y, py), dz = fma_(h, -a2.z, pz);
  return sub_(sqrt_(fma_(dx, dx, fma_(dy, dy, mul_(dz, dz)))), a0.w);
}

// Torus around the unit axis u through c: distance to the circle of radius R
// minus r; records [c, r] [u, R].  (The radial square root takes a tiny floor
// so that derivatives stay finite on the axis.)
template <class T>
__device__ __forceinline__ T sd_torus(const float4 a0, const float4 a1, const T p[3]) {
  const T vx = sub_(p[0], a0.x), vy = sub_(p[1], a0.y), vz = sub_(p[2], a0.z);
  const T h = fma_(vx, a1.x, fma_(vy, a1.y, mul_(vz, a1.z)));
  const T vv = fma_(vx, vx, fma_(vy, vy, mul_(vz, vz)));
  const T q = sub_(sqrt_(max_(fma_(h, -h, vv), 1e-30f)), a1.w);
  return sub_(sqrt_(fma_(q, q, mul_(h, h))), a0.w);
}

// Sphere-cone (convex hull of the balls (a, r_a), (b, r_b)): in the axial
// plane (y along u = (b - a)/h from a, x the distance to the axis) the side
// has outward normal (cos, sin) and spans lam = cos y - sin x in [0, cos h];
// nearest feature ball a, side or ball b.  Records [a, r_a] [b, r_b] [u, h]
// [sin, cos, cos h, 0].
template <class T>
__device__ __forceinline__ T sd_scone(const float4 a0, const float4 a1, const float4 a2, const float4 a3,
                                      const T p[3]) {
  const T vx = sub_(p[0], a0.x), vy = sub_(p[1], a0.y), vz = sub_(p[2], a0.z);
  const T y = fma_(vx, a2.x, fma_(vy, a2.y, mul_(vz, a2.z)));
  const T vv = fma_(vx, vx, fma_(vy, vy, mul_(vz, vz)));
  const T x2 = max_(fma_(y, -y, vv), 1e-30f);
  const T x = sqrt_(x2);
  const T lam = fma_(y, a3.y, mul_(x, -a3.x));
  const T fa = sub_(sqrt_(max_(vv, 1e-30f)), a0.w);
  const T yb = sub_(y, a2.w);
  const T fb = sub_(sqrt_(fma_(yb, yb, x2)), a1.w);
  const T fs = sub_(fma_(x, a3.y, mul_(y, a3.x)), a0.w);
  return val(lam) < 0.f ? fa : (val(lam) > a3.z ? fb : fs);
}

// Ellipsoid bound min(r) (|M (p - c) / r| - 1); records [c, min r]
// [M row i, r_i] x 3 [1/r0, 1/r1, 1/r2, 0].
template <class T>
__device__ __forceinline__ T sd_ellipsoid(const float4 a0, const float4 a1, const float4 a2, const float4 a3,
                                          const float4 a4, const T p[3]) {
  const T wx = sub_(p[0], a0.x), wy = sub_(p[1], a0.y), wz = sub_(p[2], a0.z);
  const T z0 = mul_(fma_(wx, a1.x, fma_(wy, a1.y, mul_(wz, a1.z))), a4.x);
  const T z1 = mul_(fma_(wx, a2.x, fma_(wy, a2.y, mul_(wz, a2.z))), a4.y);
  const T z2 = mul_(fma_(wx, a3.x, fma_(wy, a3.y, mul_(wz, a3.z))), a4.z);
  const T s = sqrt_(fma_(z0, z0, fma_(z1, z1, mul_(z2, z2))));
  return fma_(s, a0.w, -a0.w);
}

// Rounded triangle: distance to the triangle (a, b, c) minus r.  With w =
// p - a, the point projects inside the triangle when it lies on the inner
// side of the three edge planes m_i . (p - v_i) <= 0 (m_i = e_i x n, the
// outward in-plane edge normals; tested on FP32 values, so the float and
// dual-number evaluations take the same branch); the distance is then
// |n . w|, else the least distance to the three edge segments.  Records [a, r] [e0, 1/|e0|^2]
// [e1, 1/|e1|^2] [e2, 1/|e2|^2] [n, m2.x] [m0, m2.y] [m1, m2.z].
template <class T>
__device__ __forceinline__ T seg_dist2(const T &wx, const T &wy, const T &wz, const float4 e) {
  T h = mul_(fma_(wx, e.x, fma_(wy, e.y, mul_(wz, e.z))), e.w);
  h = min_(max_(h, 0.f), 1.f);
  const T qx = fma_(h, -e.x, wx), qy = fma_(h, -e.y, wy), qz = fma_(h, -e.z, wz);
  return fma_(qx, qx, fma_(qy, qy, mul_(qz, qz)));
}
template <class T>
__device__ __forceinline__ T sd_rtri(const float4 *q, const T p[3]) {
  // Few values live at a time (this body is part of the out-of-line
  // sd_further, whose registers count for the tracing kernel): the inside
  // tests first, then the plane distance or the three edge distances.
  const float4 a0 = ldrec(q);
  const T wx = sub_(p[0], a0.x), wy = sub_(p[1], a0.y), wz = sub_(p[2], a0.z);   // p - a
  bool inside;
  {
    const float4 a5 = ldrec(q + 5);
    inside = fma_(val(wx), a5.x, fma_(val(wy), a5.y, mul_(val(wz), a5.z))) <= 0.f;
  }
  {
    const float4 a1 = ldrec(q + 1), a6 = ldrec(q + 6);
    const float ux = sub_(val(wx), a1.x), uy = sub_(val(wy), a1.y), uz = sub_(val(wz), a1.z);   // p - b
    inside = inside && fma_(ux, a6.x, fma_(uy, a6.y, mul_(uz, a6.z))) <= 0.f;
  }
  {
    const float4 a3 = ldrec(q + 3);
    const float m2x = ldrec(q + 4).w, m2y = ldrec(q + 5).w, m2z = ldrec(q + 6).w;
    const float vx = add_(val(wx), a3.x), vy = add_(val(wy), a3.y), vz = add_(val(wz), a3.z);   // p - c
    inside = inside && fma_(vx, m2x, fma_(vy, m2y, mul_(vz, m2z))) <= 0.f;
  }
  T d2;
  if (inside) {
    const float4 a4 = ldrec(q + 4);
    const T pd = fma_(wx, a4.x, fma_(wy, a4.y, mul_(wz, a4.z)));
    d2 = mul_(pd, pd);
  } else {
    const float4 a1 = ldrec(q + 1);
    d2 = seg_dist2<T>(wx, wy, wz, a1);
    d2 = min_(d2, seg_dist2<T>(sub_(wx, a1.x), sub_(wy, a1.y), sub_(wz, a1.z), ldrec(q + 2)));
    const float4 a3 = ldrec(q + 3);
    d2 = min_(d2, seg_dist2<T>(add_(wx, a3.x), add_(wy, a3.y), add_(wz, a3.z), a3));
  }
  return sub_(sqrt_(d2), a0.w);
}

// Bounded quadric: max(q'(clamp_e(u)), box distance(u)) in local
// coordinates u = M (p - c), q' = q / G (coefficients pre-divided by the
// gradient bound), accumulated axis by axis.  Records [c, kappa'] [M row i,
// e_i] x 3 [alpha', beta', gamma', delta'].
template <class T>
__device__ __forceinline__ T sd_quadric(const float4 *q, const T p[3]) {
  const float4 a0 = ldrec(q);
  const T wx = sub_(p[0], a0.x), wy = sub_(p[1], a0.y), wz = sub_(p[2], a0.z);
  const float4 cf = ldrec(q + 4);
  T qv = T(a0.w), out2 = T(0.f), inner = T(-INFINITY);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float4 m = ldrec(q + 1 + i);
    const T u = fma_(wx, m.x, fma_(wy, m.y, mul_(wz, m.z)));
    const T c = min_(max_(u, -m.w), m.w);
    qv = i == 2 ? fma_(c, fma_(c, cf.z, cf.w), qv) : fma_(mul_(c, c), i == 0 ? cf.x : cf.y, qv);
    const T b = sub_(abs_(u), m.w);
    const T bp = max_(b, 0.f);
    out2 = fma_(bp, bp, out2);
    inner = max_(inner, b);
  }
  const T box = add_(sqrt_(out2), min_(inner, 0.f));
  return max_(qv, box);
}

// The further families out of line: one copy per value type instead of one
// per interpreter instantiation and call site, so scenes without them keep
// the interpreter's code (and instruction-fetch footprint) of the three
// basic families.  kAll = false: the copy without the rounded triangle and
// the bounded quadric, for scenes whose further primitives are tori,
// sphere-cones and ellipsoids only (the larger body costs such scenes ~10 %
// of tracing time through the calling kernel's registers).
template <class T, bool kAll = true>
__device__ __noinline__ T sd_further(uint32_t code, const float4 *q, T px, T py, T pz) {
  const T p[3] = {px, py, pz};
  if (code == V_TORUS) return sd_torus<T>(ldrec(q), ldrec(q + 1), p);
  if (code == V_SCONE) return sd_scone<T>(ldrec(q), ldrec(q + 1), ldrec(q + 2), ldrec(q + 3), p);
  if (kAll) {
    if (code == V_RTRI) return sd_rtri<T>(q, p);
    if (code == V_QUADRIC) return sd_quadric<T>(q, p);
  }
  return sd_ellipsoid<T>(ldrec(q), ldrec(q + 1), ldrec(q + 2), ldrec(q + 3), ldrec(q + 4), p);
}

// The further families for a pair of points: the scalar function per
// component (out of line, as for one point).
template <bool kAll>
__device__ __forceinline__ F2 further_pair(uint32_t code, const float4 *q, const F2 p[3]) {
  return F2(make_float2(sd_further<float, kAll>(code, q, p[0].v.x, p[1].v.x, p[2].v.x),
                        sd_further<float, kAll>(code, q, p[0].v.y, p[1].v.y, p[2].v.y)));
}
template <class T, bool kAll>
__device__ __forceinline__ T further_eval(uint32_t code, const float4 *q, const T p[3]) {
  if constexpr (std::is_same<T, F2>::value)
    return further_pair<kAll>(code, q, p);
  else
    return sd_further<T, kAll>(code, q, p[0], p[1], p[2]);
}

// ---- compact smooth operators G_op (Sec. 5) -------------------------------------
// Record [k, d_o, c1 = 6 / (6 d_o - k), 1/k].  Smooth displacement of Eq. 5:
// d(f0, f1, k) = k/6 max(1 - a/k, 0)^3 with a = |f0 - f1|; transition
// b_r(x) = k max(1 - c1 x, 0); a non-positive blend range gives no blend.
template <class T>
__device__ __forceinline__ T cube_(const T &x) { return mul_(x, mul_(x, x)); }

// Displacement with blend range kr, as (kr / 6) and max(1 - a/kr, 0)^3 for a
// fused m -/+ (kr/6) x^3; a non-positive range gives no displacement.
template <class T>
__device__ __forceinline__ void disp_terms(const T &kr, const T &a, T &kr6, T &x3) {
  const auto pos = gt_(kr, 1e-30f);
  const T x = mul_(max_(sub_(kr, a), 0.f), rcp_(sel_(pos, kr, T(1.f))));
  kr6 = sel_(pos, mul_(kr, 1.f / 6.f), T(0.f));
  x3 = cube_(x);
}

// The three compact operators G_op (union, intersection, difference) as one
// branch-free body: the (warp-uniform) operator code selects min / max, the
// sign of the displacement and the clamp of the blend range (k' <= k for the
// intersection and the difference, |k'| for the difference), so the
// interpreter has one case for all three.  The blended value is always
// computed and selected by the range test f0 <= d_o and f1 <= d_o.
template <class T>
__device__ __forceinline__ T op_compact_any(uint32_t code, float4 c, const T &f0, const T &f1) {
  const bool uni = code == V_UNION, dif = code == V_DIFF;
  const auto inside = and_(le_(f0, c.y), le_(f1, c.y));
  const float k6 = mul_(c.x, 1.f / 6.f);
  const T g1 = dif ? -f1 : f1;
  const T m = uni ? min_(f0, g1) : max_(f0, g1);
  const T a = abs_(sub_(f0, g1));
  const T x = mul_(max_(sub_(c.x, a), 0.f), c.w);
  const T g = fma_(cube_(x), uni ? -k6 : k6, m);
  const T kb = mul_(max_(fma_(g, -c.z, 1.f), 0.f), c.x);
  const T kr = uni ? kb : min_(dif ? abs_(kb) : kb, c.x);
  T kr6, x3;
  disp_terms(kr, a, kr6, x3);
  const T res = fma_(uni ? -kr6 : kr6, x3, m);
  return sel_(inside, res, m);
}

template <class T>
__device__ __forceinline__ T op_sharp_any(uint32_t code, const T &f0, const T &f1) {
  const T g1 = code == V_SDIFF ? -f1 : f1;
  return code == V_SUNION ? min_(f0, g1) : max_(f0, g1);
}

__device__ __forceinline__ uint32_t node_flops(uint32_t code) {
  switch (code) {
    case V_SPHERE: return kFlopsSphere;
    case V_RBOX: return kFlopsRbox;
    case V_CAPSULE: return kFlopsCapsule;
    case V_TORUS: return kFlopsTorus;
    case V_SCONE: return kFlopsScone;
    case V_ELLIPSOID: return kFlopsEllipsoid;
    case V_RTRI: return kFlopsRtri;
    case V_QUADRIC: return kFlopsQuadric;
    case V_UNION: case V_INTER: case V_DIFF: return kFlopsCompactOp;
    case V_SUNION: case V_SINTER: case V_SDIFF: return kFlopsSharpOp;
    default: return 0;
  }
}

// Stacks that carry the output slots of the CTA-split evaluation.
template <class S, class = void> struct StkCta { static constexpr bool value = false; };
template <class S> struct StkCta<S, std::void_t<decltype(S::kCta)>> { static constexpr bool value = S::kCta; };

// One node of Algorithm 3 for R points: a primitive pushes the running value
// and evaluates itself, an operator pops its left operand and combines; q is
// the node's record (unused by nodes without one).
template <int R, class T, class Stk, int kFam>
__device__ __forceinline__ void eval_node(uint32_t code, const float4 *q, const T (&p)[R][3], T (&acc)[R], Stk &stk,
                                          int &sp) {
  // Nested warp-uniform branches in order of frequency (compact operators,
  // then the three basic primitives) rather than a switch: the switch's
  // indexed jump costs every node a branch-target resolution (measured on
  // B300: 9-12 % of the 1080p trace).
  if (code <= V_DIFF) {
    if (code >= V_UNION) {
      const float4 c = ldrec(q);
      T l[R];
      stk.pop(--sp, l);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = op_compact_any<T>(code, c, l[r], acc[r]);
    } else {
      stk.push(sp++, acc);
      if (code == V_SPHERE) {
        const float4 a = ldrec(q);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = sd_sphere<T>(a, p[r]);
      } else if (code == V_RBOX) {
        const float4 a0 = ldrec(q), a1 = ldrec(q + 1), a2 = ldrec(q + 2), a3 = ldrec(q + 3);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = sd_rbox<T>(a0, a1, a2, a3, p[r]);
      } else {
        const float4 a0 = ldrec(q), a2 = ldrec(q + 2);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = sd_capsule<T>(a0, a2, p[r]);
      }
    }
  } else if (code <= V_SDIFF) {
    T l[R];
    stk.pop(--sp, l);
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = op_sharp_any<T>(code, l[r], acc[r]);
  } else if (code == V_LEFT) {
    stk.pop(--sp, acc);
  } else if (code == V_RIGHT) {
    --sp;
  } else if (code == V_INF) {
    --sp;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = T(INFINITY);
  } else if (StkCta<Stk>::value && code >= V_STORE) {
    // CTA-split evaluation (pairs of points only; see st_trace.cu): STORE
    // writes the running value to the stack's next output slot and pops,
    // LOAD pushes and takes the lane's value from the node's staged record.
    if constexpr (StkCta<Stk>::value) {
      const int lane = threadIdx.x & 31;
      if (code == V_STORE) {
        __stcg(stk.xout + (size_t)stk.xn * 32 + lane, acc[0].v);
        ++stk.xn;
        stk.pop(--sp, acc);
      } else {
        stk.push(sp++, acc);
        acc[0] = F2(reinterpret_cast<const float2 *>(q)[lane]);
      }
    }
  } else {   // the further primitive families (codes 12..16)
    stk.push(sp++, acc);
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = kFam ? further_eval<T, kFam == 2>(code, q, p[r]) : T(INFINITY);
  }
}

// Algorithm 3 for R independent evaluation points per thread, sharing one
// decode and one record load per node.  The top of each stack lives in
// acc[r]; deeper entries in `stk` (one slot holds the R values).  The first
// primitive pushes an unused value, so `stk` needs one slot more than the
// live depth.  T is float (tracing) or a dual number (refinement).
// kFam, the primitive families the instance evaluates: 0 a lean instance for
// views of spheres, rounded boxes and capsules only (the further families are
// never evaluated; a view holding one gets +inf there -- the host picks the
// lean instance only for scenes without them), 1 also tori, sphere-cones and
// ellipsoids, 2 all eight families.
template <int R, class T, class Stk, int kFam = 2>
__device__ __forceinline__ void eval_view_r(const uint32_t *view, int n_view, const RecSrc &src,
                                            const T (&p)[R][3], T (&acc)[R], Stk &stk) {
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = T(0.f);
  int sp = 0;
  uint32_t w = n_view > 0 ? view[0] : 0u;
  for (int i = 0; i < n_view; ++i) {
    const uint32_t code = w >> kViewCodeShift;
    const float4 *q = rec_ptr(src, w);
    if (i + 1 < n_view) w = view[i + 1];
    eval_node<R, T, Stk, kFam>(code, q, p, acc, stk, sp);
  }
}

// Single-point convenience form.
template <class T, class Stk>
__device__ __forceinline__ T eval_view(const uint32_t *view, int n_view, const RecSrc &src, const T p[3],
                                       Stk &stk) {
  T pp[1][3] = {{p[0], p[1], p[2]}};
  T acc[1];
  eval_view_r<1, T>(view, n_view, src, pp, acc, stk);
  return acc[0];
}

// Shared-memory stacks: slot s of lane l at base[s * 32 + l], 8 bytes per
// slot (two float values, or one value + derivative).
struct SmemStack2 {   // R = 2 float points
  float2 *base;
  __device__ __forceinline__ void push(int s, const float (&a)[2]) { base[s * 32] = make_float2(a[0], a[1]); }
  __device__ __forceinline__ void pop(int s, float (&a)[2]) const {
    const float2 v = base[s * 32];
    a[0] = v.x;
    a[1] = v.y;
  }
};
struct SmemStackF2 {  // R = 1 pair of float points (F2), the same slots as SmemStack2
  float2 *base;
  __device__ __forceinline__ void push(int s, const F2 (&a)[1]) { base[s * 32] = a[0].v; }
  __device__ __forceinline__ void pop(int s, F2 (&a)[1]) const { a[0] = F2(base[s * 32]); }
};
// The same with the output slots of the CTA-split evaluation (the only stack
// whose interpreter instance handles its STORE and LOAD codes).
struct SmemStackF2Cta {
  float2 *base;
  float2 *xout;   // the warp's output slots (slot s of lane l at xout[s * 32 + l])
  int xn;         // ... and the next slot to write
  static constexpr bool kCta = true;
  __device__ __forceinline__ void push(int s, const F2 (&a)[1]) { base[s * 32] = a[0].v; }
  __device__ __forceinline__ void pop(int s, F2 (&a)[1]) const { a[0] = F2(base[s * 32]); }
};
struct SmemStack1 {   // R = 1 float point (the .x half of SmemStack2's slots)
  float2 *base;
  __device__ __forceinline__ void push(int s, const float (&a)[1]) { reinterpret_cast<float *>(base + s * 32)[0] = a[0]; }
  __device__ __forceinline__ void pop(int s, float (&a)[1]) const { a[0] = reinterpret_cast<const float *>(base + s * 32)[0]; }
};
struct SmemStackD1 {  // R = 1 dual number (value, derivative)
  float2 *base;
  __device__ __forceinline__ void push(int s, const Dual<1> (&a)[1]) { base[s * 32] = make_float2(a[0].v, a[0].g[0]); }
  __device__ __forceinline__ void pop(int s, Dual<1> (&a)[1]) const {
    const float2 v = base[s * 32];
    a[0].v = v.x;
    a[0].g[0] = v.y;
  }
};

// Thread-local stack (inspection kernels).
template <class T>
struct LocalStack {
  T s[ST_MAX_STACK + 2];
  __device__ __forceinline__ void push(int i, const T (&a)[1]) { s[i] = a[0]; }
  __device__ __forceinline__ void pop(int i, T (&a)[1]) const { a[0] = s[i]; }
};

}  // namespace st
