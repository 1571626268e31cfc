// st_field.cuh -- field evaluation of a pruned tree view on the GPU.
//
// Node functions are written once over a numeric type T: float for the
// tracing hot loop (approximate MUFU square root / reciprocal), or a
// forward-mode dual number Dual<N> (value and N directional derivatives) for
// the Newton refinement along the ray and the normal.
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
  T dx = p[0] - a.x, dy = p[1] - a.y, dz = p[2] - a.z;
  return sqrt_(dx * dx + dy * dy + dz * dz) - a.w;
}

// q = |M (p - c)| - b ; |max(q, 0)| + min(max_i q_i, 0) - r_round
template <class T>
__device__ __forceinline__ T sd_rbox(const float4 a0, const float4 a1, const float4 a2, const float4 a3,
                                     const T p[3]) {
  T wx = p[0] - a0.x, wy = p[1] - a0.y, wz = p[2] - a0.z;
  T q0 = abs_(wx * a1.x + wy * a1.y + wz * a1.z) - a1.w;
  T q1 = abs_(wx * a2.x + wy * a2.y + wz * a2.z) - a2.w;
  T q2 = abs_(wx * a3.x + wy * a3.y + wz * a3.z) - a3.w;
  T m0 = max_(q0, 0.f), m1 = max_(q1, 0.f), m2 = max_(q2, 0.f);
  T inner = min_(max_(q0, max_(q1, q2)), 0.f);
  return sqrt_(m0 * m0 + m1 * m1 + m2 * m2) + inner - a0.w;
}

// distance to segment [a, b] minus r; records [a, r] and [b - a, 1/|b-a|^2]
template <class T>
__device__ __forceinline__ T sd_capsule(const float4 a0, const float4 a2, const T p[3]) {
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
  const bool pos = val(kr) > 1e-30f;
  T x = max_(kr - a, 0.f) * rcp_(pos ? kr : T(1.f));
  T d = (kr * (1.f / 6.f)) * (x * x * x);
  return pos ? d : T(0.f);
}

// Branch-free: the blended value is always computed and selected by the
// range test (no divergence inside a warp that evaluates the same node).
template <uint32_t CODE, class T>
__device__ __forceinline__ T op_compact(float4 c, const T &f0, const T &f1) {
  const bool inside = val(f0) <= c.y && val(f1) <= c.y;
  if (CODE == V_UNION) {
    T m = min_(f0, f1);
    T a = abs_(f0 - f1);
    T x = max_(c.x - a, 0.f) * c.w;
    T g = m - (c.x * (1.f / 6.f)) * (x * x * x);
    T kr = c.x * max_(1.f - g * c.z, 0.f);
    T res = m - disp_range(kr, a);
    return inside ? res : m;
  } else if (CODE == V_INTER) {
    T m = max_(f0, f1);
    T a = abs_(f0 - f1);
    T x = max_(c.x - a, 0.f) * c.w;
    T g = m + (c.x * (1.f / 6.f)) * (x * x * x);
    T kr = min_(c.x * max_(1.f - g * c.z, 0.f), c.x);
    T res = m + disp_range(kr, a);
    return inside ? res : m;
  } else {
    // difference: csg max(f0, -f1), displacement d(f0, -f1, .)
    T nf1 = -f1;
    T m = max_(f0, nf1);
    T a = abs_(f0 - nf1);
    T x = max_(c.x - a, 0.f) * c.w;
    T g = m + (c.x * (1.f / 6.f)) * (x * x * x);
    T kr = min_(abs_(c.x * max_(1.f - g * c.z, 0.f)), c.x);
    T res = m + disp_range(kr, a);
    return inside ? res : m;
  }
}

template <uint32_t CODE, class T>
__device__ __forceinline__ T op_sharp(const T &f0, const T &f1) {
  if (CODE == V_SUNION) return min_(f0, f1);
  if (CODE == V_SINTER) return max_(f0, f1);
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

// Algorithm 3 for R independent evaluation points per thread, sharing one
// decode and one record load per node.  The top of each stack lives in
// acc[r]; deeper entries in `stk` (one slot holds the R values).  The first
// primitive pushes an unused value, so `stk` needs one slot more than the
// live depth.  T is float (tracing) or a dual number (refinement).
template <int R, class T, class Stk>
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
    switch (code) {
      case V_SPHERE: {
        const float4 a = ldrec(q);
        stk.push(sp++, acc);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = sd_sphere<T>(a, p[r]);
        break;
      }
      case V_RBOX: {
        const float4 a0 = ldrec(q), a1 = ldrec(q + 1), a2 = ldrec(q + 2), a3 = ldrec(q + 3);
        stk.push(sp++, acc);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = sd_rbox<T>(a0, a1, a2, a3, p[r]);
        break;
      }
      case V_CAPSULE: {
        const float4 a0 = ldrec(q), a2 = ldrec(q + 2);
        stk.push(sp++, acc);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = sd_capsule<T>(a0, a2, p[r]);
        break;
      }
      case V_UNION: {
        const float4 c = ldrec(q);
        T l[R];
        stk.pop(--sp, l);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = op_compact<V_UNION, T>(c, l[r], acc[r]);
        break;
      }
      case V_INTER: {
        const float4 c = ldrec(q);
        T l[R];
        stk.pop(--sp, l);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = op_compact<V_INTER, T>(c, l[r], acc[r]);
        break;
      }
      case V_DIFF: {
        const float4 c = ldrec(q);
        T l[R];
        stk.pop(--sp, l);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = op_compact<V_DIFF, T>(c, l[r], acc[r]);
        break;
      }
      case V_SUNION: {
        T l[R];
        stk.pop(--sp, l);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = op_sharp<V_SUNION, T>(l[r], acc[r]);
        break;
      }
      case V_SINTER: {
        T l[R];
        stk.pop(--sp, l);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = op_sharp<V_SINTER, T>(l[r], acc[r]);
        break;
      }
      case V_SDIFF: {
        T l[R];
        stk.pop(--sp, l);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = op_sharp<V_SDIFF, T>(l[r], acc[r]);
        break;
      }
      case V_INF: {
        --sp;
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = T(INFINITY);
        break;
      }
      case V_RIGHT: --sp; break;
      default: {  // V_LEFT
        stk.pop(--sp, acc);
        break;
      }
    }
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
