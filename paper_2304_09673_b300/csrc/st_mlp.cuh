// st_mlp.cuh -- the learned relaxation factor: step features and the warp-level
// BF16 tensor-core inference of the MLP 6 -> 32 -> 32 -> 1 (ReLU, output
// omega = 1 + sigmoid(o)) used inside the tracer.
//
// Parameter vector (FP32, ST_MLP_PARAMS floats, training layout):
//   W1[32][6] (out, in), b1[32], W2[32][32], b2[32], w3[32], b3
// Packed inference layout (st_mlp_pack, kMlpPackBytes):
//   W1 as bf16 [32][16] (out, in zero-padded), W2 bf16 [32][32],
//   w3 bf16 [8][32] (row 0 = w3, rows 1..7 zero), b1 f32[32], b2 f32[32], b3 f32.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace st {

constexpr int kMlpIn = 6, kMlpH = 32;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 1313
constexpr size_t kMlpPackBytes = 4096;
constexpr size_t kMlpW1Off = 0, kMlpW2Off = 1024, kMlpW3Off = 3072, kMlpB1Off = 3584, kMlpB2Off = 3712,
                 kMlpB3Off = 3840;

// Step features (fixed scaling, identical in recording and inference):
//   x0 = 8 f / L, x1 = 8 f_prev / L (f when there is no previous point),
//   x2 = 8 x previous step length in distance units (0 when none),
//   x3 = steps / 64, x4 = log2(1 + primitives in the view) / 8,
//   x5 = log2(1 + A-buffer list length) / 8.
__host__ __device__ inline void step_features(float f, float f_prev, float dz_prev_dist, bool have_prev,
                                              uint32_t steps, int n_prim, uint32_t list_len, float inv_l,
                                              float x[6]) {
  x[0] = 8.f * f * inv_l;
  x[1] = 8.f * (have_prev ? f_prev : f) * inv_l;
  x[2] = have_prev ? 8.f * dz_prev_dist : 0.f;
  x[3] = (float)steps * (1.f / 64.f);
  x[4] = log2f(1.f + (float)n_prim) * 0.125f;
  x[5] = log2f(1.f + (float)list_len) * 0.125f;
}

// Training label of one recorded plain step (learned-step reading of the
// paper's over-relaxation, Sec. 10): with consecutive plain-step values
// f_i, f_{i+1}, the field drops at rate k = 1 - f_{i+1} / f_i per plain step
// and a relaxed step omega passes the sphere-overlap test while
// omega <= 2 / (1 + k).  Label = 0.97 x that bound, clamped to [1, 2].
__host__ __device__ inline float step_label(float f_i, float f_next) {
  float k = 1.f - f_next / f_i;
  k = fminf(fmaxf(k, 0.f), 1.f);
  const float w = 0.97f * 2.f / (1.f + k);
  return fminf(fmaxf(w, 1.f), 2.f);
}

// Packed weights staged in shared memory (16-byte aligned), held as one base
// pointer with the parts at their fixed offsets: the tracer keeps this across
// its whole loop, and one pointer instead of six values leaves registers to
// the marching state (learned step, B300: 1080p -2 %, 10k clustered -12 %).
struct MlpSmem {
  const unsigned char *base;
  __device__ __forceinline__ const uint32_t *w1() const { return reinterpret_cast<const uint32_t *>(base + kMlpW1Off); }
  __device__ __forceinline__ const uint32_t *w2() const { return reinterpret_cast<const uint32_t *>(base + kMlpW2Off); }
  __device__ __forceinline__ const uint32_t *w3() const { return reinterpret_cast<const uint32_t *>(base + kMlpW3Off); }
  __device__ __forceinline__ const float *b1() const { return reinterpret_cast<const float *>(base + kMlpB1Off); }
  __device__ __forceinline__ const float *b2() const { return reinterpret_cast<const float *>(base + kMlpB2Off); }
  __device__ __forceinline__ float b3() const { return *reinterpret_cast<const float *>(base + kMlpB3Off); }
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// m16n8k8: layer 1 has 6 inputs, so K = 8 covers them (columns 6, 7 zero).
__device__ __forceinline__ void mma_bf16_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// One 16-row tile of the network: layer-1 A fragments (rows g and g + 8,
// input columns 2t, 2t + 1) in, output column 0 of rows g and g + 8 out
// (valid in lanes with t == 0).
__device__ __forceinline__ void mlp_tile(const MlpSmem &W, uint32_t a0, uint32_t a1, int g, int t, float &o_lo,
                                         float &o_hi) {
  const float2 *b1 = reinterpret_cast<const float2 *>(W.b1());
  const float2 *b2 = reinterpret_cast<const float2 *>(W.b2());
  float h1[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 b = b1[4 * q + t];
    h1[q][0] = b.x; h1[q][1] = b.y; h1[q][2] = b.x; h1[q][3] = b.y;
    mma_bf16_k8(h1[q], a0, a1, W.w1()[(8 * q + g) * 8 + t]);
  }
  uint32_t a2[2][4];
#pragma unroll
  for (int kt = 0; kt < 2; ++kt) {
    a2[kt][0] = pack_bf16(fmaxf(h1[2 * kt][0], 0.f), fmaxf(h1[2 * kt][1], 0.f));
    a2[kt][1] = pack_bf16(fmaxf(h1[2 * kt][2], 0.f), fmaxf(h1[2 * kt][3], 0.f));
    a2[kt][2] = pack_bf16(fmaxf(h1[2 * kt + 1][0], 0.f), fmaxf(h1[2 * kt + 1][1], 0.f));
    a2[kt][3] = pack_bf16(fmaxf(h1[2 * kt + 1][2], 0.f), fmaxf(h1[2 * kt + 1][3], 0.f));
  }
  float h2[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 b = b2[4 * q + t];
    h2[q][0] = b.x; h2[q][1] = b.y; h2[q][2] = b.x; h2[q][3] = b.y;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt)
      mma_bf16(h2[q], a2[kt], W.w2()[(8 * q + g) * 16 + 8 * kt + t], W.w2()[(8 * q + g) * 16 + 8 * kt + t + 4]);
  }
  uint32_t a3[2][4];
#pragma unroll
  for (int kt = 0; kt < 2; ++kt) {
    a3[kt][0] = pack_bf16(fmaxf(h2[2 * kt][0], 0.f), fmaxf(h2[2 * kt][1], 0.f));
    a3[kt][1] = pack_bf16(fmaxf(h2[2 * kt][2], 0.f), fmaxf(h2[2 * kt][3], 0.f));
    a3[kt][2] = pack_bf16(fmaxf(h2[2 * kt + 1][0], 0.f), fmaxf(h2[2 * kt + 1][1], 0.f));
    a3[kt][3] = pack_bf16(fmaxf(h2[2 * kt + 1][2], 0.f), fmaxf(h2[2 * kt + 1][3], 0.f));
  }
  float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int kt = 0; kt < 2; ++kt) mma_bf16(o, a3[kt], W.w3()[g * 16 + 8 * kt + t], W.w3()[g * 16 + 8 * kt + t + 4]);
  const float b3 = W.b3();
  o_lo = o[0] + b3;
  o_hi = o[2] + b3;
}

// 1 + sigmoid(v) = 1.5 + tanh(v / 2) / 2 (one MUFU tanh).
__device__ __forceinline__ float omega_of(float v) {
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(0.5f * v));
  return 1.5f + 0.5f * th;
}

// Warp-collective: evaluates the MLP on the feature vectors of live slots
// (slot s of a lane is live when bit s of `live` is set) and returns omega
// per slot (1 for dead slots).  Live slots are packed into consecutive rows
// (slot 0 of the lanes in order, then slot 1), so only ceil(live / 16)
// 16-row tiles run; a row's result does not depend on its position.
// xs: per-warp shared scratch of 64 rows x 4 words (1 KB; words 0..2 hold
// the six BF16 features), os: 64 floats.
__device__ __forceinline__ void mlp_omega_warp(const MlpSmem &W, const float (&x)[2][6], float (&omega)[2],
                                               __nv_bfloat16 *xs, float *os, uint32_t live = 3u) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  uint32_t *xu = reinterpret_cast<uint32_t *>(xs);
  uint32_t lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  const uint32_t m0 = __ballot_sync(0xFFFFFFFFu, live & 1u);
  const uint32_t m1 = __ballot_sync(0xFFFFFFFFu, (live >> 1) & 1u);
  const int row[2] = {__popc(m0 & lt), __popc(m0) + __popc(m1 & lt)};
  const int n_rows = __popc(m0) + __popc(m1);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if ((live >> s) & 1u) {
      uint32_t *r = xu + row[s] * 4;
      r[0] = pack_bf16(x[s][0], x[s][1]);
      r[1] = pack_bf16(x[s][2], x[s][3]);
      r[2] = pack_bf16(x[s][4], x[s][5]);
    }
  }
  __syncwarp();
#pragma unroll 1
  for (int m0r = 0; m0r < n_rows; m0r += 16) {
    // Rows past n_rows hold stale words; their outputs are never used.
    const uint32_t a0 = t < 3 ? xu[(m0r + g) * 4 + t] : 0u;
    const uint32_t a1 = t < 3 ? xu[(m0r + g + 8) * 4 + t] : 0u;
    float lo, hi;
    mlp_tile(W, a0, a1, g, t, lo, hi);
    if (t == 0) {
      os[m0r + g] = lo;
      os[m0r + g + 8] = hi;
    }
  }
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 2; ++s) omega[s] = ((live >> s) & 1u) ? omega_of(os[row[s]]) : 1.f;
  __syncwarp();
}

// Stages the packed weights into shared memory (CTA-collective).
__device__ __forceinline__ MlpSmem load_mlp(const void *packed, unsigned char *sm) {
  const uint4 *src = reinterpret_cast<const uint4 *>(packed);
  uint4 *dst = reinterpret_cast<uint4 *>(sm);
  for (int i = threadIdx.x; i < (int)(kMlpPackBytes / 16); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  MlpSmem w;
  w.base = sm;
  return w;
}

}  // namespace st
