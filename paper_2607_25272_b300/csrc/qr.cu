// The preconditioner factor (Sec. 2.2; Sec. 4 applies H-hat through a QR):
// H-hat = (S-hat X)^T (S-hat X) = R^T R with R from a Householder QR of the
// r x d sketch S-hat X, then R^{-1} and R^{-T} for the two triangular
// products z = R^{-1} (R^{-T} g) of every PCG iteration.
//
// Householder step k (one launch): every CTA forms the reflector of column
// k from the untouched column (it only reads it), then applies it to the
// trailing columns it owns, one warp per column.  Column k itself is never
// written during step k, so the CTAs do not race; the diagonal alpha_k is
// recorded separately.  FP64 throughout: at kappa = 1e8 the sketch must be
// factored well below 1/kappa relative error.
#include "common.cuh"
#include "internal.hpp"

namespace spcg {

constexpr int QR_WARPS = 4;

// Deterministic block sum (fixed order over warps).
template <int NW>
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_allsum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NW; ++i) s += red[i];
  return s;
}

__global__ void __launch_bounds__(QR_WARPS * 32)
    k_householder_step(double* __restrict__ A, int64_t r, int d, int k,
                       double* __restrict__ Rdiag) {
  __shared__ double red[QR_WARPS];
  const double* colk = A + (int64_t)k * r;
  // sum of squares of x(k+1 : r)
  double s2 = 0.0;
  for (int64_t i = k + 1 + threadIdx.x; i < r; i += blockDim.x) s2 += colk[i] * colk[i];
  s2 = block_sum<QR_WARPS>(s2, red);
  const double x0 = colk[k];
  const double normx = sqrt(x0 * x0 + s2);
  const double alpha = (x0 >= 0.0) ? -normx : normx;
  const double v0 = x0 - alpha;
  const double vv = v0 * v0 + s2;
  if (blockIdx.x == 0 && threadIdx.x == 0) Rdiag[k] = alpha;
  if (vv == 0.0) return;
  const double tau = 2.0 / vv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // trailing columns j = k+1+gw, gw over all warps of the grid
  for (int j = k + 1 + blockIdx.x * QR_WARPS + warp; j < d; j += gridDim.x * QR_WARPS) {
    double* colj = A + (int64_t)j * r;
    double s = 0.0;
    for (int64_t i = k + 1 + lane; i < r; i += 32) s += colk[i] * colj[i];
    s = warp_allsum(s) + v0 * colj[k];
    const double f = tau * s;
    if (lane == 0) colj[k] -= f * v0;
    for (int64_t i = k + 1 + lane; i < r; i += 32) colj[i] -= f * colk[i];
  }
}

// R (row-major upper, diag > 0) from the reduced matrix: row i of R is row i
// of A after step i, times the sign that makes alpha_i positive.
__global__ void k_extract_R(const double* __restrict__ A, int64_t r, int d,
                            const double* __restrict__ Rdiag, double* __restrict__ R,
                            int* __restrict__ status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)d * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    const double a = Rdiag[i];
    const double sgn = (a < 0.0) ? -1.0 : 1.0;
    double v = 0.0;
    if (j == i) {
      v = fabs(a);
      if (!(v > 0.0) || !isfinite(v)) atomicExch(status, DEV_BREAKDOWN);
    } else if (j > i) {
      v = sgn * A[(int64_t)j * r + i];
    }
    R[e] = v;
  }
}

// R^{-1} column by column (one warp per column j): back substitution of
// R x = e_j, x_i = -(sum_{k=i+1..j} R_ik x_k) / R_ii, x_j = 1 / R_jj.
__global__ void __launch_bounds__(256) k_trtri_upper(const double* __restrict__ R, int d,
                                                   double* __restrict__ Rinv) {
  extern __shared__ double xs[];  // 8 warps x d
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 8 + warp;
  if (j >= d) return;
  double* x = xs + (size_t)warp * d;
  for (int i = lane; i < d; i += 32) x[i] = 0.0;
  __syncwarp();
  if (lane == 0) x[j] = 1.0 / R[(int64_t)j * d + j];
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    const double* Ri = R + (int64_t)i * d;
    double s = 0.0;
    for (int k = i + 1 + lane; k <= j; k += 32) s += Ri[k] * x[k];
    s = warp_allsum(s);
    if (lane == 0) x[i] = -s / Ri[i];
    __syncwarp();
  }
  for (int i = lane; i < d; i += 32) Rinv[(int64_t)i * d + j] = x[i];
}

__global__ void k_transpose(const double* __restrict__ S, int d, double* __restrict__ T) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int row = by + yy, col = bx + threadIdx.x;
    if (row < d && col < d) tile[yy][threadIdx.x] = S[(int64_t)row * d + col];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int row = bx + yy, col = by + threadIdx.x;
    if (row < d && col < d) T[(int64_t)row * d + col] = tile[threadIdx.x][yy];
  }
}

spcg_status launch_precond_factor(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int d = c->d;
  const int64_t r = s.sched.r;
  for (int k = 0; k < d; ++k) {
    const int cols = d - k - 1;
    int grid = (cols + QR_WARPS - 1) / QR_WARPS;
    if (grid < 1) grid = 1;
    k_householder_step<<<grid, QR_WARPS * 32, 0, c->stream>>>(s.Ahat, r, d, k, s.Rdiag);
  }
  c->n_launch += d + 3;
  SPCG_CK(cudaGetLastError());
  const int64_t dd = (int64_t)d * d;
  int g = (int)((dd + 255) / 256);
  if (g > 4096) g = 4096;
  k_extract_R<<<g, 256, 0, c->stream>>>(s.Ahat, r, d, s.Rdiag, s.R, &c->scal->status);
  SPCG_CK(cudaGetLastError());
  const size_t smem = (size_t)8 * d * sizeof(double);
  SPCG_CK(cudaFuncSetAttribute(k_trtri_upper, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  k_trtri_upper<<<(d + 7) / 8, 256, smem, c->stream>>>(s.R, d, s.Rinv);
  SPCG_CK(cudaGetLastError());
  dim3 tg((d + 31) / 32, (d + 31) / 32);
  k_transpose<<<tg, dim3(32, 8), 0, c->stream>>>(s.Rinv, d, s.RinvT);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

}  // namespace spcg
