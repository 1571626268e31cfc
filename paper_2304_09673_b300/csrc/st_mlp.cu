// st_mlp.cu -- training and inspection kernels of the learned relaxation
// factor (MLP 6 -> 32 -> 32 -> 1, ReLU, omega = 1 + sigmoid(o)).
//
//   k_mlp_grad   FP32 forward + backward over a batch of step records; the
//                loss is the asymmetric squared error sum_i w_i (omega_i - y_i)^2
//                with w_i = 4 when omega_i > y_i (an overshooting factor costs
//                a rejected step) and 1 otherwise; gradients of that sum.
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
