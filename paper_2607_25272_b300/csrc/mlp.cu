// The schedule model: a 4 -> 64 -> 64 -> n_out MLP (ReLU hidden layers) that
// predicts the log10 cost of each candidate sketch-size schedule from four
// features of a problem.  The paper leaves the choice of the schedule open
// (Sec. 4.3: automatic selection remains open); this network picks among
// candidates and the paper's schedule stays the fallback.
//
// Weights are used in BF16 (products and sums in FP32); training keeps an
// FP32 master copy and updates it with Adam (Kingma & Ba, 2015).  Parameter
// layout: W1 (64 x 4, row-major), b1 (64), W2 (64 x 64), b2 (64),
// W3 (n_out x 64), b3 (n_out).
//
// Kernels: k_mlp_forward (inference), k_mlp_grad_partial (forward and
// backward over a block of samples, per-CTA gradient sums), k_mlp_reduce
// (fixed-order sum over CTAs), k_mlp_adam (update and BF16 copy).
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.hpp"

namespace spcg {

constexpr int MH = 64, MIN = 4, MMAXOUT = 64, SPB = 16;   // samples per CTA

__host__ __device__ constexpr int p_W1() { return 0; }
__host__ __device__ constexpr int p_b1() { return MH * MIN; }
__host__ __device__ constexpr int p_W2() { return MH * MIN + MH; }
__host__ __device__ constexpr int p_b2() { return MH * MIN + MH + MH * MH; }
__host__ __device__ constexpr int p_W3() { return MH * MIN + 2 * MH + MH * MH; }
__host__ __device__ inline int p_b3(int nout) { return p_W3() + nout * MH; }
__host__ __device__ inline int n_params(int nout) { return p_b3(nout) + nout; }

struct MlpShared {
  float W1[MH * MIN], b1[MH], W2[MH * MH], b2[MH], W3[MMAXOUT * MH], b3[MMAXOUT];
  float x[MIN], z1[MH], h1[MH], z2[MH], h2[MH], y[MMAXOUT], dy[MMAXOUT], dz2[MH], dz1[MH];
};

__device__ void mlp_load(MlpShared& s, const __nv_bfloat16* __restrict__ Wb, int nout) {
  for (int i = threadIdx.x; i < MH * MIN; i += blockDim.x) s.W1[i] = __bfloat162float(Wb[p_W1() + i]);
  for (int i = threadIdx.x; i < MH; i += blockDim.x) {
    s.b1[i] = __bfloat162float(Wb[p_b1() + i]);
    s.b2[i] = __bfloat162float(Wb[p_b2() + i]);
  }
  for (int i = threadIdx.x; i < MH * MH; i += blockDim.x) s.W2[i] = __bfloat162float(Wb[p_W2() + i]);
  for (int i = threadIdx.x; i < nout * MH; i += blockDim.x) s.W3[i] = __bfloat162float(Wb[p_W3() + i]);
  for (int i = threadIdx.x; i < nout; i += blockDim.x) s.b3[i] = __bfloat162float(Wb[p_b3(nout) + i]);
  __syncthreads();
}

// Forward pass of one sample held in s.x; thread u owns hidden unit u.
__device__ void mlp_fwd(MlpShared& s, int nout) {
  const int u = threadIdx.x;
  float a = s.b1[u];
#pragma unroll
  for (int k = 0; k < MIN; ++k) a = fmaf(s.W1[u * MIN + k], s.x[k], a);
  s.z1[u] = a;
  s.h1[u] = fmaxf(a, 0.f);
  __syncthreads();
  a = s.b2[u];
  for (int j = 0; j < MH; ++j) a = fmaf(s.W2[u * MH + j], s.h1[j], a);
  s.z2[u] = a;
  s.h2[u] = fmaxf(a, 0.f);
  __syncthreads();
  if (u < nout) {
    a = s.b3[u];
    for (int j = 0; j < MH; ++j) a = fmaf(s.W3[u * MH + j], s.h2[j], a);
    s.y[u] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(MH) k_mlp_forward(const __nv_bfloat16* __restrict__ Wb, int nout,
                                                    const float* __restrict__ x, int64_t B,
                                                    float* __restrict__ y) {
  __shared__ MlpShared s;
  mlp_load(s, Wb, nout);
  for (int64_t n = blockIdx.x; n < B; n += gridDim.x) {
    if (threadIdx.x < MIN) s.x[threadIdx.x] = x[n * MIN + threadIdx.x];
    __syncthreads();
    mlp_fwd(s, nout);
    if (threadIdx.x < nout) y[n * nout + threadIdx.x] = s.y[threadIdx.x];
    __syncthreads();
  }
}

// Loss = mean over samples and outputs of (y - t)^2.  Each CTA adds the
// gradient of its SPB samples into one row of `partials` (n_params floats)
// and its share of the squared error into loss_part[blockIdx.x].
__global__ void __launch_bounds__(MH) k_mlp_grad_partial(const __nv_bfloat16* __restrict__ Wb,
                                                         int nout, const float* __restrict__ x,
                                                         const float* __restrict__ t, int64_t B,
                                                         float* __restrict__ partials,
                                                         float* __restrict__ loss_part) {
  __shared__ MlpShared s;
  __shared__ float red[MH];
  mlp_load(s, Wb, nout);
  const int u = threadIdx.x;
  const int P = n_params(nout);
  float gW1[MIN] = {0.f, 0.f, 0.f, 0.f}, gb1 = 0.f, gb2 = 0.f, gb3 = 0.f;
  float gW2[MH], gW3[MH];
#pragma unroll
  for (int j = 0; j < MH; ++j) gW2[j] = gW3[j] = 0.f;
  float sq = 0.f;
  const float scale = 2.f / (float)(B * nout);
  const int64_t n0 = (int64_t)blockIdx.x * SPB;
  for (int64_t n = n0; n < n0 + SPB && n < B; ++n) {
    if (u < MIN) s.x[u] = x[n * MIN + u];
    __syncthreads();
    mlp_fwd(s, nout);
    if (u < nout) {
      const float diff = s.y[u] - t[n * nout + u];
      sq = fmaf(diff, diff, sq);
      s.dy[u] = scale * diff;
    }
    __syncthreads();
    if (u < nout) {
      const float dyu = s.dy[u];
#pragma unroll
      for (int j = 0; j < MH; ++j) gW3[j] = fmaf(dyu, s.h2[j], gW3[j]);
      gb3 += dyu;
    }
    float dh = 0.f;   // d loss / d h2[u]
    for (int o = 0; o < nout; ++o) dh = fmaf(s.W3[o * MH + u], s.dy[o], dh);
    const float dz2 = s.z2[u] > 0.f ? dh : 0.f;
    s.dz2[u] = dz2;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MH; ++j) gW2[j] = fmaf(dz2, s.h1[j], gW2[j]);
    gb2 += dz2;
    float dh1 = 0.f;  // d loss / d h1[u]
    for (int v = 0; v < MH; ++v) dh1 = fmaf(s.W2[v * MH + u], s.dz2[v], dh1);
    const float dz1 = s.z1[u] > 0.f ? dh1 : 0.f;
#pragma unroll
    for (int k = 0; k < MIN; ++k) gW1[k] = fmaf(dz1, s.x[k], gW1[k]);
    gb1 += dz1;
    __syncthreads();
  }
  float* g = partials + (size_t)blockIdx.x * P;
#pragma unroll
  for (int k = 0; k < MIN; ++k) g[p_W1() + u * MIN + k] = gW1[k];
  g[p_b1() + u] = gb1;
#pragma unroll
  for (int j = 0; j < MH; ++j) g[p_W2() + u * MH + j] = gW2[j];
  g[p_b2() + u] = gb2;
  if (u < nout) {
#pragma unroll
    for (int j = 0; j < MH; ++j) g[p_W3() + u * MH + j] = gW3[j];
    g[p_b3(nout) + u] = gb3;
  }
  red[u] = sq;
  __syncthreads();
  if (u == 0) {
    float a = 0.f;
    for (int i = 0; i < MH; ++i) a += red[i];
    loss_part[blockIdx.x] = a;
  }
}

__global__ void k_mlp_reduce(const float* __restrict__ partials, int nb, int P,
                             float* __restrict__ grad, const float* __restrict__ loss_part,
                             float* __restrict__ loss, float loss_scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int b = 0; b < nb; ++b) a += partials[(size_t)b * P + i];
    grad[i] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
    float a = 0.f;
    for (int b = 0; b < nb; ++b) a += loss_part[b];
    *loss = a * loss_scale;
  }
}

__global__ void k_mlp_adam(float* __restrict__ theta, const float* __restrict__ grad,
                           float* __restrict__ m, float* __restrict__ v, int P, float lr,
                           float beta1, float beta2, float eps, float bc1, float bc2,
                           __nv_bfloat16* __restrict__ Wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * g;
    const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    theta[i] = th;
    Wb[i] = __float2bfloat16_rn(th);
  }
}

__global__ void k_mlp_to_bf16(const float* __restrict__ theta, int P, __nv_bfloat16* __restrict__ Wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    Wb[i] = __float2bfloat16_rn(theta[i]);
}

spcg_status mlp_forward_launch(const void* Wb, int nout, const float* x, int64_t B, float* y,
                               cudaStream_t st) {
  int g = (int)(B < 1024 ? B : 1024);
  if (g < 1) g = 1;
  k_mlp_forward<<<g, MH, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(Wb), nout, x, B, y);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

}  // namespace spcg

using namespace spcg;

extern "C" int64_t spcg_mlp_params(int32_t n_out) {
  if (n_out < 1 || n_out > MMAXOUT) return -1;
  return n_params(n_out);
}

extern "C" int64_t spcg_mlp_workspace_floats(int32_t n_out, int64_t B) {
  if (n_out < 1 || n_out > MMAXOUT || B < 0) return -1;
  const int64_t nb = (B + SPB - 1) / SPB;
  return nb * n_params(n_out) + nb + 1;
}

extern "C" spcg_status spcg_mlp_forward(const uint16_t* Wb, int32_t n_out, const float* x,
                                        int64_t B, float* y, void* stream) {
  if (!Wb || !x || !y || n_out < 1 || n_out > MMAXOUT || B < 0) return SPCG_E_INVALID_ARG;
  if (B == 0) return SPCG_OK;
  SPCG_TRY(mlp_forward_launch(Wb, n_out, x, B, y, (cudaStream_t)stream));
  SPCG_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SPCG_OK;
}

extern "C" spcg_status spcg_mlp_grad(const uint16_t* Wb, int32_t n_out, const float* x,
                                     const float* t, int64_t B, float* grad, float* loss,
                                     float* workspace, void* stream) {
  if (!Wb || !x || !t || !grad || !workspace || n_out < 1 || n_out > MMAXOUT || B < 1)
    return SPCG_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int P = n_params(n_out);
  const int nb = (int)((B + SPB - 1) / SPB);
  float* partials = workspace;
  float* loss_part = workspace + (size_t)nb * P;
  k_mlp_grad_partial<<<nb, MH, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(Wb), n_out, x, t,
                                        B, partials, loss_part);
  SPCG_CK(cudaGetLastError());
  k_mlp_reduce<<<(P + 255) / 256, 256, 0, st>>>(partials, nb, P, grad, loss_part, loss,
                                                1.f / (float)(B * n_out));
  SPCG_CK(cudaGetLastError());
  SPCG_CK(cudaStreamSynchronize(st));
  return SPCG_OK;
}

extern "C" spcg_status spcg_mlp_adam(float* theta, const float* grad, float* m, float* v,
                                     int64_t P, float lr, int32_t step, uint16_t* Wb,
                                     void* stream) {
  if (!theta || !grad || !m || !v || !Wb || P < 1 || step < 1) return SPCG_E_INVALID_ARG;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  k_mlp_adam<<<(int)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      theta, grad, m, v, (int)P, lr, b1, b2, 1e-8f, bc1, bc2,
      reinterpret_cast<__nv_bfloat16*>(Wb));
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

extern "C" spcg_status spcg_mlp_to_bf16(const float* theta, int64_t P, uint16_t* Wb, void* stream) {
  if (!theta || !Wb || P < 1) return SPCG_E_INVALID_ARG;
  k_mlp_to_bf16<<<(int)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      theta, (int)P, reinterpret_cast<__nv_bfloat16*>(Wb));
  SPCG_CK(cudaGetLastError());
  SPCG_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SPCG_OK;
}
