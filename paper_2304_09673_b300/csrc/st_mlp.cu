// st_mlp.cu -- training and inspection kernels of the learned relaxation
// factor (MLP 6 -> 32 -> 32 -> 1, ReLU, omega = 1 + sigmoid(o)).
//
//   k_mlp_grad   FP32 forward + backward over a batch of step records; the
//                loss is the asymmetric squared error sum_i w_i (omega_i - y_i)^2
//                with w_i = 4 when omega_i > y_i (an overshooting factor costs
//                a rejected step) and 1 otherwise; gradients of that sum.
//   k_mlp_grad_tc  the same gradient with BF16 tensor-core products (mma.sync,
//                FP32 accumulation, FP32 master weights): the training default.
//   k_mlp_adam   Adam update of the FP32 parameters.
//   k_mlp_infer  the tracer's BF16 tensor-core inference (mlp_omega_warp) on
//                arbitrary feature rows, for checking.
#include <cmath>
#include <cstring>
#include <string>

#include "st_kernels.h"
#include "st_mlp.cuh"

namespace st {

namespace {

constexpr int kTB = 64;        // records per CTA round
constexpr int kGradThreads = 128;

// Parameter offsets in the training vector.
constexpr int oW1 = 0, oB1 = 192, oW2 = 224, oB2 = 1248, oW3 = 1280, oB3 = 1312;

__global__ void __launch_bounds__(kGradThreads)
k_mlp_grad(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ Y, int n,
           float *__restrict__ G, float *__restrict__ loss_sum) {
  __shared__ float sP[kMlpParams];
  __shared__ float sG[kMlpParams];
  __shared__ float sX[kTB][kMlpIn];
  __shared__ float sH1[kTB][kMlpH + 1], sH2[kTB][kMlpH + 1];
  __shared__ float sD1[kTB][kMlpH + 1], sD2[kTB][kMlpH + 1];
  __shared__ float sDo[kTB];
  __shared__ float sLoss;
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    sP[i] = P[i];
    sG[i] = 0.f;
  }
  if (threadIdx.x == 0) sLoss = 0.f;
  __syncthreads();
  for (int base = blockIdx.x * kTB; base < n; base += gridDim.x * kTB) {
    const int i = threadIdx.x;
    if (i < kTB) {
      const int r = base + i;
      const bool valid = r < n;
      float x[kMlpIn];
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) x[k] = valid ? X[(size_t)r * kMlpIn + k] : 0.f;
      float a1[kMlpH], h1[kMlpH], a2[kMlpH], h2[kMlpH];
#pragma unroll 4
      for (int j = 0; j < kMlpH; ++j) {
        float s = sP[oB1 + j];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) s += sP[oW1 + j * kMlpIn + k] * x[k];
        a1[j] = s;
        h1[j] = fmaxf(s, 0.f);
      }
#pragma unroll 4
      for (int j = 0; j < kMlpH; ++j) {
        float s = sP[oB2 + j];
#pragma unroll 8
        for (int k = 0; k < kMlpH; ++k) s += sP[oW2 + j * kMlpH + k] * h1[k];
        a2[j] = s;
        h2[j] = fmaxf(s, 0.f);
      }
      float o = sP[oB3];
#pragma unroll 8
      for (int k = 0; k < kMlpH; ++k) o += sP[oW3 + k] * h2[k];
      const float sg = 1.f / (1.f + expf(-o));
      const float w = 1.f + sg;
      const float y = valid ? Y[r] : 0.f;
      const float err = w - y;
      const float wt = err > 0.f ? 4.f : 1.f;
      const float dw = valid ? 2.f * wt * err : 0.f;
      const float dout = dw * sg * (1.f - sg);
      if (valid) atomicAdd(&sLoss, wt * err * err);
      float d2[kMlpH];
#pragma unroll 8
      for (int j = 0; j < kMlpH; ++j) d2[j] = a2[j] > 0.f ? dout * sP[oW3 + j] : 0.f;
#pragma unroll 4
      for (int k = 0; k < kMlpH; ++k) {
        float s = 0.f;
#pragma unroll 8
        for (int j = 0; j < kMlpH; ++j) s += sP[oW2 + j * kMlpH + k] * d2[j];
        sD1[i][k] = a1[k] > 0.f ? s : 0.f;
      }
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) sX[i][k] = x[k];
#pragma unroll 8
      for (int j = 0; j < kMlpH; ++j) {
        sH1[i][j] = h1[j];
        sH2[i][j] = h2[j];
        sD2[i][j] = d2[j];
      }
      sDo[i] = dout;
    }
    __syncthreads();
    // Per-parameter sums over the round's records.
    for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) {
      float s = 0.f;
      if (p < oB1) {
        const int j = p / kMlpIn, k = p % kMlpIn;
        for (int r = 0; r < kTB; ++r) s += sD1[r][j] * sX[r][k];
      } else if (p < oW2) {
        const int j = p - oB1;
        for (int r = 0; r < kTB; ++r) s += sD1[r][j];
      } else if (p < oB2) {
        const int j = (p - oW2) / kMlpH, k = (p - oW2) % kMlpH;
        for (int r = 0; r < kTB; ++r) s += sD2[r][j] * sH1[r][k];
      } else if (p < oW3) {
        const int j = p - oB2;
        for (int r = 0; r < kTB; ++r) s += sD2[r][j];
      } else if (p < oB3) {
        const int k = p - oW3;
        for (int r = 0; r < kTB; ++r) s += sDo[r] * sH2[r][k];
      } else {
        for (int r = 0; r < kTB; ++r) s += sDo[r];
      }
      sG[p] += s;
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) atomicAdd(&G[p], sG[p]);
  if (threadIdx.x == 0) atomicAdd(loss_sum, sLoss);
}

// ---- tensor-core gradient (BF16 operands, FP32 accumulation) ----------------
// Each warp takes 16 records at a time.  Forward: the inference's three
// mma.sync layers, keeping the ReLU masks and the rounded activations.
// Backward: d2 = dout w3 (masked) and d1 = bf16(d2) W2 (mma with W2^T), then
// the weight gradients as products over the 16 records (M = output unit,
// N = input unit, K = record): the records' signals and activations go
// through shared memory transposed ([unit][record], BF16), so both operands
// load as 32-bit pairs.  Bias gradients and w3's gradient are FP32 sums in
// registers.  The per-lane sums go to a CTA copy of the gradient in shared
// memory, then to the caller's vector.
constexpr int kTcWarps = 4;
constexpr int kTcStride = 12;   // words per row of a transposed [unit][16 records] tile (conflict-free)

struct TcOperands {            // BF16 pairs (low half = lower index) and FP32 vectors
  uint32_t w1[kMlpH * 8];      // W1 [out j][in k], k padded to 16 (6 used)
  uint32_t w2[kMlpH * 16];     // W2 [out j][in i]
  uint32_t w2t[kMlpH * 16];    // W2^T [in i][out j]
  uint32_t w3[8 * 16];         // w3 as row 0 of an [8][32] block
  float b1[kMlpH], b2[kMlpH], w3f[kMlpH];   // w3f: w3 rounded to BF16
  float b3;
};

struct TcTiles {               // one warp's transposed tiles
  uint32_t h1t[kMlpH * kTcStride];
  uint32_t d2t[kMlpH * kTcStride];
  uint32_t d1t[kMlpH * kTcStride];
  uint32_t xt[8 * kTcStride];
};

__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ void put_bf16(uint32_t *tile, int unit, int rec, float v) {
  reinterpret_cast<__nv_bfloat16 *>(tile)[unit * 2 * kTcStride + rec] = __float2bfloat16_rn(v);
}

__device__ void load_tc_operands(const float *__restrict__ P, TcOperands &S) {
  for (int w = threadIdx.x; w < kMlpH * 16; w += blockDim.x) {
    const int r = w >> 4, c = 2 * (w & 15);
    S.w2[w] = pack_bf16(P[oW2 + r * kMlpH + c], P[oW2 + r * kMlpH + c + 1]);
    S.w2t[w] = pack_bf16(P[oW2 + c * kMlpH + r], P[oW2 + (c + 1) * kMlpH + r]);
  }
  for (int w = threadIdx.x; w < kMlpH * 8; w += blockDim.x) {
    const int j = w >> 3, k = 2 * (w & 7);
    S.w1[w] = pack_bf16(k < kMlpIn ? P[oW1 + j * kMlpIn + k] : 0.f, k + 1 < kMlpIn ? P[oW1 + j * kMlpIn + k + 1] : 0.f);
  }
  for (int w = threadIdx.x; w < 8 * 16; w += blockDim.x)
    S.w3[w] = w < 16 ? pack_bf16(P[oW3 + 2 * w], P[oW3 + 2 * w + 1]) : 0u;
  for (int j = threadIdx.x; j < kMlpH; j += blockDim.x) {
    S.b1[j] = P[oB1 + j];
    S.b2[j] = P[oB2 + j];
    S.w3f[j] = round_bf16(P[oW3 + j]);
  }
  if (threadIdx.x == 0) S.b3 = P[oB3];
}

__global__ void __launch_bounds__(kTcWarps * 32)
k_mlp_grad_tc(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ Y, int n,
              float *__restrict__ G, float *__restrict__ loss_sum) {
  __shared__ __align__(16) TcOperands S;
  __shared__ __align__(16) TcTiles T[kTcWarps];
  __shared__ float sG[kMlpParams];
  __shared__ float sLoss;
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sG[i] = 0.f;
  if (threadIdx.x == 0) sLoss = 0.f;
  load_tc_operands(P, S);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  TcTiles &Tw = T[warp];
  // Per-lane sums: weight gradients as mma accumulators (gW2: 2 x 4 tiles,
  // gW1: 2 tiles), FP32 column sums for columns 8q + 2t + e.
  float gw2[2][4][4], gw1[2][4];
  float gb1[4][2], gb2[4][2], gw3[4][2];
  float gb3 = 0.f, lsum = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      gw1[a][e] = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) gw2[a][b][e] = 0.f;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int e = 0; e < 2; ++e) gb1[q][e] = gb2[q][e] = gw3[q][e] = 0.f;

  for (int base = (blockIdx.x * kTcWarps + warp) * 16; base < n; base += gridDim.x * kTcWarps * 16) {
    // Fragment rows: record g ("lo") and g + 8 ("hi"); columns 8q + 2t + e.
    const int r_lo = base + g, r_hi = base + g + 8;
    const bool v_lo = r_lo < n, v_hi = r_hi < n;
    float x_lo[2], x_hi[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = 2 * t + e;
      x_lo[e] = (t < 3 && v_lo) ? X[(size_t)r_lo * kMlpIn + k] : 0.f;
      x_hi[e] = (t < 3 && v_hi) ? X[(size_t)r_hi * kMlpIn + k] : 0.f;
    }
    const uint32_t xa0 = pack_bf16(x_lo[0], x_lo[1]), xa1 = pack_bf16(x_hi[0], x_hi[1]);
    // forward, as the tracer's inference: pre-activations a, rounded ReLU outputs h
    float a1[4][4], h1[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 b = reinterpret_cast<const float2 *>(S.b1)[4 * q + t];
      a1[q][0] = b.x; a1[q][1] = b.y; a1[q][2] = b.x; a1[q][3] = b.y;
      mma_bf16_k8(a1[q], xa0, xa1, S.w1[(8 * q + g) * 8 + t]);
#pragma unroll
      for (int e = 0; e < 4; ++e) h1[q][e] = round_bf16(fmaxf(a1[q][e], 0.f));
    }
    uint32_t af[2][4];
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
      af[kt][0] = pack_bf16(h1[2 * kt][0], h1[2 * kt][1]);
      af[kt][1] = pack_bf16(h1[2 * kt][2], h1[2 * kt][3]);
      af[kt][2] = pack_bf16(h1[2 * kt + 1][0], h1[2 * kt + 1][1]);
      af[kt][3] = pack_bf16(h1[2 * kt + 1][2], h1[2 * kt + 1][3]);
    }
    float a2[4][4], h2[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 b = reinterpret_cast<const float2 *>(S.b2)[4 * q + t];
      a2[q][0] = b.x; a2[q][1] = b.y; a2[q][2] = b.x; a2[q][3] = b.y;
#pragma unroll
      for (int kt = 0; kt < 2; ++kt)
        mma_bf16(a2[q], af[kt], S.w2[(8 * q + g) * 16 + 8 * kt + t], S.w2[(8 * q + g) * 16 + 8 * kt + t + 4]);
#pragma unroll
      for (int e = 0; e < 4; ++e) h2[q][e] = round_bf16(fmaxf(a2[q][e], 0.f));
    }
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
      af[kt][0] = pack_bf16(h2[2 * kt][0], h2[2 * kt][1]);
      af[kt][1] = pack_bf16(h2[2 * kt][2], h2[2 * kt][3]);
      af[kt][2] = pack_bf16(h2[2 * kt + 1][0], h2[2 * kt + 1][1]);
      af[kt][3] = pack_bf16(h2[2 * kt + 1][2], h2[2 * kt + 1][3]);
    }
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) mma_bf16(o, af[kt], S.w3[g * 16 + 8 * kt + t], S.w3[g * 16 + 8 * kt + t + 4]);
    // output column 0 sits in the lanes with t == 0
    const float o_rows[2] = {__shfl_sync(0xFFFFFFFFu, o[0], lane & ~3) + S.b3,
                             __shfl_sync(0xFFFFFFFFu, o[2], lane & ~3) + S.b3};
    float dout[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool valid = h ? v_hi : v_lo;
      const float sg = 1.f / (1.f + expf(-o_rows[h]));
      const float err = 1.f + sg - (valid ? Y[h ? r_hi : r_lo] : 0.f);
      const float wt = err > 0.f ? 4.f : 1.f;
      dout[h] = valid ? 2.f * wt * err * sg * (1.f - sg) : 0.f;
      if (t == 0 && valid) lsum += wt * err * err;
    }
    if (t == 0) gb3 += dout[0] + dout[1];
    // backward: d2 = dout w3 where a2 > 0; d1 = bf16(d2) W2 where a1 > 0
    float d2[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        d2[q][e] = a2[q][e] > 0.f ? dout[e >> 1] * S.w3f[8 * q + 2 * t + (e & 1)] : 0.f;
        gb2[q][e & 1] += d2[q][e];
        gw3[q][e & 1] += dout[e >> 1] * h2[q][e];
        d2[q][e] = round_bf16(d2[q][e]);
      }
    }
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
      af[kt][0] = pack_bf16(d2[2 * kt][0], d2[2 * kt][1]);
      af[kt][1] = pack_bf16(d2[2 * kt][2], d2[2 * kt][3]);
      af[kt][2] = pack_bf16(d2[2 * kt + 1][0], d2[2 * kt + 1][1]);
      af[kt][3] = pack_bf16(d2[2 * kt + 1][2], d2[2 * kt + 1][3]);
    }
    float d1[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d1[q][0] = d1[q][1] = d1[q][2] = d1[q][3] = 0.f;
#pragma unroll
      for (int kt = 0; kt < 2; ++kt)
        mma_bf16(d1[q], af[kt], S.w2t[(8 * q + g) * 16 + 8 * kt + t], S.w2t[(8 * q + g) * 16 + 8 * kt + t + 4]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        d1[q][e] = a1[q][e] > 0.f ? d1[q][e] : 0.f;
        gb1[q][e & 1] += d1[q][e];
      }
    }
    // the records' activations and signals, transposed to [unit][record]
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int unit = 8 * q + 2 * t + (e & 1), rec = (e >> 1) * 8 + g;
        put_bf16(Tw.h1t, unit, rec, h1[q][e]);
        put_bf16(Tw.d2t, unit, rec, d2[q][e]);
        put_bf16(Tw.d1t, unit, rec, d1[q][e]);
      }
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {   // input units 6 and 7 (lanes t == 3) are zero
      put_bf16(Tw.xt, 2 * t + e, g, x_lo[e]);
      put_bf16(Tw.xt, 2 * t + e, g + 8, x_hi[e]);
    }
    __syncwarp();
    // weight gradients over the 16 records: gW2 = d2^T h1, gW1 = d1^T x
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const uint32_t *ar = Tw.d2t + (16 * mt + g) * kTcStride + t;
      const uint32_t a_d2[4] = {ar[0], ar[8 * kTcStride], ar[4], ar[8 * kTcStride + 4]};
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const uint32_t *br = Tw.h1t + (8 * nt + g) * kTcStride + t;
        mma_bf16(gw2[mt][nt], a_d2, br[0], br[4]);
      }
      const uint32_t *ar1 = Tw.d1t + (16 * mt + g) * kTcStride + t;
      const uint32_t a_d1[4] = {ar1[0], ar1[8 * kTcStride], ar1[4], ar1[8 * kTcStride + 4]};
      const uint32_t *bx = Tw.xt + g * kTcStride + t;
      mma_bf16(gw1[mt], a_d1, bx[0], bx[4]);
    }
  }

  // Lane sums -> the CTA's gradient.  Accumulator element e of a tile sits at
  // row 16 mt + g + 8 (e >> 1), column 8 nt + 2t + (e & 1).
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 16 * mt + g + 8 * (e >> 1), c = 2 * t + (e & 1);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) atomicAdd(&sG[oW2 + j * kMlpH + 8 * nt + c], gw2[mt][nt][e]);
      if (c < kMlpIn) atomicAdd(&sG[oW1 + j * kMlpIn + c], gw1[mt][e]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float s1 = gb1[q][e], s2 = gb2[q][e], s3 = gw3[q][e];
#pragma unroll
      for (int m = 4; m < 32; m <<= 1) {   // over the 8 lanes of one column pair (g)
        s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, m);
        s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, m);
        s3 += __shfl_xor_sync(0xFFFFFFFFu, s3, m);
      }
      if (g == 0) {
        const int c = 8 * q + 2 * t + e;
        atomicAdd(&sG[oB1 + c], s1);
        atomicAdd(&sG[oB2 + c], s2);
        atomicAdd(&sG[oW3 + c], s3);
      }
    }
  }
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) {
    gb3 += __shfl_xor_sync(0xFFFFFFFFu, gb3, m);
    lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, m);
  }
  if (lane == 0) {
    atomicAdd(&sG[oB3], gb3);
    atomicAdd(&sLoss, lsum);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) atomicAdd(&G[p], sG[p]);
  if (threadIdx.x == 0) atomicAdd(loss_sum, sLoss);
}


__global__ void k_mlp_adam(float *P, const float *G, float *M, float *V, float lr, float b1, float b2, float eps,
                           float scale, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float g = G[p] * scale;
  const float m = b1 * M[p] + (1.f - b1) * g;
  const float v = b2 * V[p] + (1.f - b2) * g * g;
  M[p] = m;
  V[p] = v;
  P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void __launch_bounds__(128) k_mlp_infer(const void *packed, const float *X, int n, float *omega) {
  __shared__ __align__(16) unsigned char s_w[kMlpPackBytes];
  __shared__ __align__(16) __nv_bfloat16 s_x[4][64 * 16];
  __shared__ float s_o[4][64];
  const MlpSmem W = load_mlp(packed, s_w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int base = (blockIdx.x * 4 + warp) * 64; base < n; base += gridDim.x * 4 * 64) {
    float x[2][6], om[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int r = base + s * 32 + lane;
#pragma unroll
      for (int k = 0; k < 6; ++k) x[s][k] = r < n ? X[(size_t)r * 6 + k] : 0.f;
    }
    mlp_omega_warp(W, x, om, s_x[warp], s_o[warp]);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int r = base + s * 32 + lane;
      if (r < n) omega[r] = om[s];
    }
  }
}

uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t bias = 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even
  return (uint16_t)((u + bias) >> 16);
}

}  // namespace

}  // namespace st

using namespace st;

#define MLP_CK(call)                                                      \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) {                                              \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));      \
      return ST_ERR_CUDA;                                                 \
    }                                                                     \
  } while (0)

extern "C" {

size_t st_mlp_pack_size(void) { return kMlpPackBytes; }
int st_mlp_param_count(void) { return kMlpParams; }

int st_mlp_pack(const float *params, void *packed) {
  if (!params || !packed) { set_error("st_mlp_pack: null argument"); return ST_ERR_INVALID; }
  unsigned char *out = static_cast<unsigned char *>(packed);
  std::memset(out, 0, kMlpPackBytes);
  uint16_t *w1 = reinterpret_cast<uint16_t *>(out + kMlpW1Off);
  uint16_t *w2 = reinterpret_cast<uint16_t *>(out + kMlpW2Off);
  uint16_t *w3 = reinterpret_cast<uint16_t *>(out + kMlpW3Off);
  float *b1 = reinterpret_cast<float *>(out + kMlpB1Off);
  float *b2 = reinterpret_cast<float *>(out + kMlpB2Off);
  float *b3 = reinterpret_cast<float *>(out + kMlpB3Off);
  for (int j = 0; j < kMlpH; ++j)
    for (int k = 0; k < kMlpIn; ++k) w1[j * 16 + k] = to_bf16(params[oW1 + j * kMlpIn + k]);
  for (int j = 0; j < kMlpH; ++j)
    for (int k = 0; k < kMlpH; ++k) w2[j * kMlpH + k] = to_bf16(params[oW2 + j * kMlpH + k]);
  for (int k = 0; k < kMlpH; ++k) w3[k] = to_bf16(params[oW3 + k]);
  for (int j = 0; j < kMlpH; ++j) {
    b1[j] = params[oB1 + j];
    b2[j] = params[oB2 + j];
  }
  *b3 = params[oB3];
  return ST_OK;
}

int st_mlp_grad(const float *params, const float *x, const float *y, int n, float *grad, float *loss_sum,
                void *stream) {
  if (!params || !grad || !loss_sum || n < 0 || (n > 0 && (!x || !y))) {
    set_error("st_mlp_grad: invalid arguments");
    return ST_ERR_INVALID;
  }
  if (n == 0) return ST_OK;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rounds = (n + kTB - 1) / kTB;
  const int grid = rounds < sms * 4 ? rounds : sms * 4;
  count_launch(), k_mlp_grad<<<grid, kGradThreads, 0, (cudaStream_t)stream>>>(params, x, y, n, grad, loss_sum);
  MLP_CK(cudaGetLastError());
  return ST_OK;
}

int st_mlp_grad_bf16(const float *params, const float *x, const float *y, int n, float *grad, float *loss_sum,
                     void *stream) {
  if (!params || !grad || !loss_sum || n < 0 || (n > 0 && (!x || !y))) {
    set_error("st_mlp_grad_bf16: invalid arguments");
    return ST_ERR_INVALID;
  }
  if (n == 0) return ST_OK;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // at least four 16-record tiles per warp, at most four CTAs per SM
  const long long tiles = (n + 15) / 16;
  const long long want = (tiles + 4 * kTcWarps - 1) / (4 * kTcWarps);
  const int grid = (int)(want < sms * 4 ? want : sms * 4);
  count_launch(), k_mlp_grad_tc<<<grid, kTcWarps * 32, 0, (cudaStream_t)stream>>>(params, x, y, n, grad, loss_sum);
  MLP_CK(cudaGetLastError());
  return ST_OK;
}

int st_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, float beta1, float beta2,
                float eps, float grad_scale, void *stream) {
  if (!params || !grad || !m || !v || step < 1) { set_error("st_mlp_adam: invalid arguments"); return ST_ERR_INVALID; }
  const float c1 = 1.f - std::pow(beta1, (float)step), c2 = 1.f - std::pow(beta2, (float)step);
  count_launch(), k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      params, grad, m, v, lr, beta1, beta2, eps, grad_scale, c1, c2);
  MLP_CK(cudaGetLastError());
  return ST_OK;
}

int st_mlp_infer(const void *packed, const float *x, int n, float *omega, void *stream) {
  if (!packed || n < 0 || (n > 0 && (!x || !omega))) { set_error("st_mlp_infer: invalid arguments"); return ST_ERR_INVALID; }
  if (n == 0) return ST_OK;
  const int blocks = (n + 255) / 256;
  count_launch(), k_mlp_infer<<<blocks < 1024 ? blocks : 1024, 128, 0, (cudaStream_t)stream>>>(packed, x, n, omega);
  MLP_CK(cudaGetLastError());
  return ST_OK;
}

}  // extern "C"
