// st_field.cuh -- field evaluation of a pruned tree view on the GPU.
//
// Node functions are written once over a numeric type T: float for the
// tracing hot loop (approximate MUFU square root / reciprocal), or a
// forward-mode dual number Dual<N> for the Newton refinement (N = 1,
// derivative along the ray) and the normal (N = 3, gradient).
#pragma once
#include <cuda_runtime.h>

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

__device__ __forceinline__ float4 ldrec(const float4 *q) { return __ldg(q); }

// ---- primitives (exact SDFs, Lipschitz 1) --------------------------------------
template <class T>
__device__ __forceinline__ T sd_sphere(const float4 *q, const T p[3]) {
  float4 a = ldrec(q);
  T dx = p[0] - a.x, dy = p[1] - a.y, dz = p[2] - a.z;
  return sqrt_(dx * dx + dy * dy + dz * dz) - a.w;
}

// q = |M (p - c)| - b ; |max(q, 0)| + min(max_i q_i, 0) - r_round
template <class T>
__device__ __forceinline__ T sd_rbox(const float4 *q, const T p[3]) {
  float4 a0 = ldrec(q), a1 = ldrec(q + 1), a2 = ldrec(q + 2), a3 = ldrec(q + 3);
  T wx = p[0] - a0.x, wy = p[1] - a0.y, wz = p[2] - a0.z;
  T q0 = abs_(wx * a1.x + wy * a1.y + wz * a1.z) - a1.w;
  T q1 = abs_(wx * a2.x + wy * a2.y + wz * a2.z) - a2.w;
  T q2 = abs_(wx * a3.x + wy * a3.y + wz * a3.z) - a3.w;
  T m0 = max_(q0, 0.f), m1 = max_(q1, 0.f), m2 = max_(q2, 0.f);
  T inner = min_(max_(q0, max_(q1, q2)), 0.f);
  return sqrt_(m0 * m0 + m1 * m1 + m2 * m2) + inner - a0.w;
}

// distance to segment [a, b] minus r; record [a, r] [b, 0] [b - a, 1/|b-a|^2]
template <class T>
__device__ __forceinline__ T sd_capsule(const float4 *q, const T p[3]) {
  float4 a0 = ldrec(q), a2 = ldrec(q + 2);
  T px = p[0] - a0.x, py = p[1] - a0.y, pz = p[2] - a0.z;
  T h = (px * a2.x + py * a2.y + pz * a2.z) * a2.w;
  h = min_(max_(h, 0.f), 1.f);
  T dx = px - h * a2.x, dy = py - h * a2.y, dz = pz - h * a2.z;
  return sqrt_(dx * dx + dy * dy + dz * dz) - a0.w;
}

// ---- compact smooth operators G_op (Sec. 5) -------------------------------------
// Record [k, d_o, c1 = 6 / (6 d_o - k), 1/k].  Smooth displacement of Eq. 5:
// d(f0, f1, k) = k/6 max(1 - a/k, 0)^3 with a = |f0 - f1|; transition
// b_r(x) = k max(1 - c1 x, 0); a non-positive blend range gives no blend.
template <class T>
__device__ __forceinline__ T disp_range(const T &kr, const T &a) {
  if (!(val(kr) > 1e-30f)) return T(0.f);
  T x = max_(kr - a, 0.f) * rcp_(kr);
  return (kr * (1.f / 6.f)) * (x * x * x);
}

template <class T>
__device__ __forceinline__ T op_compact(uint32_t code, float4 c, const T &f0, const T &f1) {
  const bool inside = val(f0) <= c.y && val(f1) <= c.y;
  if (code == V_UNION) {
    T m = min_(f0, f1);
    if (!inside) return m;
    T a = abs_(f0 - f1);
    T x = max_(c.x - a, 0.f) * c.w;
    T g = m - (c.x * (1.f / 6.f)) * (x * x * x);
    T kr = c.x * max_(1.f - g * c.z, 0.f);
    return m - disp_range(kr, a);
  }
  if (code == V_INTER) {
    T m = max_(f0, f1);
    if (!inside) return m;
    T a = abs_(f0 - f1);
    T x = max_(c.x - a, 0.f) * c.w;
    T g = m + (c.x * (1.f / 6.f)) * (x * x * x);
    T kr = min_(c.x * max_(1.f - g * c.z, 0.f), c.x);
    return m + disp_range(kr, a);
  }
  // difference: csg max(f0, -f1), displacement d(f0, -f1, .)
  T nf1 = -f1;
  T m = max_(f0, nf1);
  if (!inside) return m;
  T a = abs_(f0 - nf1);
  T x = max_(c.x - a, 0.f) * c.w;
  T g = m + (c.x * (1.f / 6.f)) * (x * x * x);
  T kr = min_(abs_(c.x * max_(1.f - g * c.z, 0.f)), c.x);
  return m + disp_range(kr, a);
}

template <class T>
__device__ __forceinline__ T op_sharp(uint32_t code, const T &f0, const T &f1) {
  if (code == V_SUNION) return min_(f0, f1);
  if (code == V_SINTER) return max_(f0, f1);
  return max_(f0, -f1);
}

__device__ __forceinline__ uint32_t node_flops(uint32_t code) {
  switch (code) {
    case V_SPHERE: return kFlopsSphere;
    case V_RBOX: return kFlopsRbox;
    case V_CAPSULE: return kFlopsCapsule;
    case V_UNION: case V_INTER: case V_DIFF: return kFlopsCompactOp;
    case V_SUNION: case V_SINTER: case V_SDIFF: return kFlopsSharpOp;
    default: return 0;
  }
}

// Algorithm 3: post-order stack evaluation of the pruned view.  The top of
// the stack lives in `acc`; deeper entries in `stk` (stride `ss` floats).
// The first primitive pushes an unused value, so `stk` needs one slot more
// than the live depth.
template <class T, class Stk>
__device__ __forceinline__ T eval_view(const uint32_t *view, int n_view, const float4 *rec, const T p[3],
                                       Stk &stk) {
  T acc(0.f);
  int sp = 0;
  uint32_t w = n_view > 0 ? view[0] : 0u;
  for (int i = 0; i < n_view; ++i) {
    const uint32_t code = w >> kViewOffBits;
    const float4 *q = rec + (w & kViewOffMask);
    if (i + 1 < n_view) w = view[i + 1];
    switch (code) {
      case V_SPHERE: stk.set(sp++, acc); acc = sd_sphere<T>(q, p); break;
      case V_RBOX: stk.set(sp++, acc); acc = sd_rbox<T>(q, p); break;
      case V_CAPSULE: stk.set(sp++, acc); acc = sd_capsule<T>(q, p); break;
      case V_UNION: case V_INTER: case V_DIFF: {
        T l = stk.get(--sp);
        acc = op_compact<T>(code, ldrec(q), l, acc);
        break;
      }
      case V_SUNION: case V_SINTER: case V_SDIFF: {
        T l = stk.get(--sp);
        acc = op_sharp<T>(code, l, acc);
        break;
      }
      case V_INF: --sp; acc = T(INFINITY); break;
      case V_RIGHT: --sp; break;
      default: acc = stk.get(--sp); break;  // V_LEFT
    }
  }
  return acc;
}

// Shared-memory stack: slot s of lane l at base[s * 32 + l].
struct SmemStack {
  float *base;
  __device__ __forceinline__ void set(int s, float v) { base[s * 32] = v; }
  __device__ __forceinline__ float get(int s) const { return base[s * 32]; }
};

// Thread-local stack for the dual-number passes.
template <class T>
struct LocalStack {
  T s[ST_MAX_STACK + 2];
  __device__ __forceinline__ void set(int i, const T &v) { s[i] = v; }
  __device__ __forceinline__ T get(int i) const { return s[i]; }
};

}  // namespace st
