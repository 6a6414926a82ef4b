// Estimate of nu = ||D R^{-1}||_2, D = diag(||R e_j||), used by the
// mixed-precision path to choose the precision of the Stage II operator.
//
// Why this number: storing X in a format with unit roundoff u perturbs each
// entry relatively, X~ = X + E with |E_ij| <= u |X_ij|.  The iterations run on
// the preconditioned operator R^{-T} X~^T X~ R^{-1}, whose distance from the
// exact one is about 2 ||E R^{-1}|| <= 2 ||E D_X^{-1}|| ||D_X R^{-1}||, with
// D_X the column norms of X and ||E D_X^{-1}|| about u.  R comes from a
// subspace embedding of X (Sec. 2.1), so ||R e_j|| matches ||X e_j|| up to the
// embedding distortion and D stands in for D_X.  Iterative refinement on the
// true gradient contracts while u nu stays well below one; the FP32 copy of X
// has u = 2^-24, the double-FP32 pair about 2^-48.
//
// nu is estimated by power iteration on B^T B, B = D R^{-1}: a few rounds of
// y = B v / ||v||, v = B^T y / ||y|| from a fixed, deterministic start vector;
// ||B v|| / ||v|| after the last round is a lower bound that converges to nu.
// Every CTA recomputes the norm of its input vector in a fixed order, so the
// estimate is deterministic and each round is one launch.
#include "common.cuh"
#include "internal.hpp"

namespace spcg {

namespace {

constexpr int kCondThreads = 256;
constexpr int kCondRows = kCondThreads / 32;   // one warp per output row
constexpr int kCondRounds = 6;

__device__ double block_norm2(const double* __restrict__ v, int d, double* red) {
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) s += v[j] * v[j];
  s = warp_allsum(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

// D_j = ||R e_j|| (R row-major upper triangular); v0 a fixed start vector.
__global__ void k_cond_init(const double* __restrict__ R, int d, double* __restrict__ D,
                            double* __restrict__ v) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  double s = 0.0;
  for (int i = 0; i <= j; ++i) s += R[(size_t)i * d + j] * R[(size_t)i * d + j];
  D[j] = sqrt(s);
  // golden-ratio sequence in [1, 2): no sign pattern or zero entries
  const double f = (double)j * 0.6180339887498949;
  v[j] = 1.0 + (f - floor(f));
}

// mode 0: y_i = D_i (R^{-1} v)_i / ||v||     (row i of R^{-1}: columns i..d-1)
// mode 1: y_j = (R^{-T} (D v))_j / ||v||     (row j of R^{-T}: columns 0..j)
__global__ void __launch_bounds__(kCondThreads)
    k_cond_mv(int mode, const double* __restrict__ M, const double* __restrict__ D, int d,
              const double* __restrict__ v, double* __restrict__ y) {
  __shared__ double red[kCondRows];
  const double nv = sqrt(block_norm2(v, d, red));
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kCondRows + (threadIdx.x >> 5);
  if (i >= d) return;
  const double* row = M + (size_t)i * d;
  const int j0 = mode == 0 ? i : 0, j1 = mode == 0 ? d : i + 1;
  double s = 0.0;
  for (int j = j0 + lane; j < j1; j += 32) s += row[j] * (mode == 0 ? v[j] : D[j] * v[j]);
  s = warp_allsum(s);
  if (lane == 0) {
    const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
    y[i] = (mode == 0 ? D[i] * s : s) * inv;
  }
}

// nu estimate = ||y|| for the last y = B v / ||v||.
__global__ void k_cond_final(const double* __restrict__ y, int d, DevScalars* scal) {
  __shared__ double red[kCondRows];
  const double n2 = block_norm2(y, d, red);
  if (threadIdx.x == 0) scal->cond = sqrt(n2);
}

}  // namespace

spcg_status launch_condest(spcg_ctx* c) {
  const int d = c->d;
  double* D = c->pb.u;   // d-space scratch: free between solves
  double* v = c->pb.z;
  double* y = c->pb.w;
  k_cond_init<<<(d + 255) / 256, 256, 0, c->stream>>>(c->sk.R, d, D, v);
  SPCG_CK(cudaGetLastError());
  const int nb = (d + kCondRows - 1) / kCondRows;
  for (int r = 0; r < kCondRounds; ++r) {
    k_cond_mv<<<nb, kCondThreads, 0, c->stream>>>(0, c->sk.Rinv, D, d, v, y);
    SPCG_CK(cudaGetLastError());
    if (r + 1 == kCondRounds) break;
    k_cond_mv<<<nb, kCondThreads, 0, c->stream>>>(1, c->sk.RinvT, D, d, y, v);
    SPCG_CK(cudaGetLastError());
  }
  k_cond_final<<<1, kCondThreads, 0, c->stream>>>(y, d, c->scal);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 2 * kCondRounds + 1;
  return SPCG_OK;
}

}  // namespace spcg
