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
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.hpp"

namespace cg = cooperative_groups;

namespace spcg {

constexpr int QR_WARPS = 8;

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

// Step k: s2 = ||x(k+1:r)||^2, alpha = -sign(x_k) ||x||, v = x - alpha e_k;
// every trailing column j gets a_j -= (2 / v.v) (v.a_j) v.  The reflector
// column is staged in shared memory when it fits; each warp owns trailing
// columns and keeps eight independent partial sums so that eight loads per
// lane are in flight (the step is bound by L2 latency, not arithmetic).
__global__ void __launch_bounds__(QR_WARPS * 32)
    k_householder_step(double* __restrict__ A, int64_t r, int d, int k,
                       double* __restrict__ Rdiag, int staged) {
  extern __shared__ double vs[];   // x(k : r) when staged
  __shared__ double red[QR_WARPS];
  const double* colk = A + (int64_t)k * r;
  const int64_t len = r - k;       // rows k .. r-1
  if (staged)
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) vs[i] = colk[k + i];
  __syncthreads();
  const double* v = staged ? vs : colk + k;   // v[i] = x_{k+i}
  double s2 = 0.0;
  for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) s2 += v[i] * v[i];
  s2 = block_sum<QR_WARPS>(s2, red);
  const double x0 = v[0];
  const double normx = sqrt(x0 * x0 + s2);
  const double alpha = (x0 >= 0.0) ? -normx : normx;
  const double v0 = x0 - alpha;
  const double vv = v0 * v0 + s2;
  if (blockIdx.x == 0 && threadIdx.x == 0) Rdiag[k] = alpha;
  if (vv == 0.0) return;
  const double tau = 2.0 / vv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = k + 1 + blockIdx.x * QR_WARPS + warp; j < d; j += gridDim.x * QR_WARPS) {
    double* cj = A + (int64_t)j * r + k;      // cj[i] = a_{k+i, j}
    double p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t i = 1 + lane;
    for (; i + 7 * 32 < len; i += 8 * 32) {
#pragma unroll
      for (int u = 0; u < 8; ++u) p[u] = fma(v[i + u * 32], cj[i + u * 32], p[u]);
    }
    for (; i < len; i += 32) p[0] = fma(v[i], cj[i], p[0]);
    double s = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
    s = warp_allsum(s) + v0 * cj[0];
    const double f = tau * s;
    if (lane == 0) cj[0] -= f * v0;
    for (int64_t i2 = 1 + lane; i2 < len; i2 += 32) cj[i2] = fma(-f, v[i2], cj[i2]);
  }
}

// Step k with the rows of the trailing matrix split over a cluster of 8 CTAs
// and its columns dealt round-robin to the clusters of the grid.  Each CTA
// sums its rows' share of ||x(k+1:r)||^2 and of every dot v.a_j; the shares
// meet through distributed shared memory and are added in rank order, so the
// result does not depend on timing.  The cluster barrier is the hardware
// barrier of the thread-block cluster (no software spin).
constexpr int QRC = 8;            // CTAs per cluster
constexpr int QRC_WARPS = 16;
constexpr int QRC_MAXCOLS = 128;  // trailing columns per cluster per step
constexpr int QRC_MAXCHUNK = 4096;  // rows of the reflector a CTA stages in shared memory

// The CTA's rows of column k (the reflector, v_0 replacing x_k) are staged in
// shared memory, so the update loop streams only the trailing column through
// global memory and its loads overlap (no aliasing with the reflector).
__global__ void __cluster_dims__(QRC, 1, 1) __launch_bounds__(QRC_WARPS * 32)
    k_householder_cluster(double* __restrict__ A, int64_t r, int d, int k,
                          double* __restrict__ Rdiag) {
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int ncl = gridDim.x / QRC, cl = blockIdx.x / QRC;
  extern __shared__ double vs[];   // chunk of column k
  __shared__ double part_s2;
  __shared__ double pdot[QRC_MAXCOLS];
  __shared__ double red[QRC_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* colk = A + (int64_t)k * r + k;          // colk[i] = x_{k+i}
  const int64_t len = r - k;
  const int64_t chunk = (len + QRC - 1) / QRC;
  const int64_t lo = q * chunk;
  const int64_t hi = (lo + chunk < len) ? lo + chunk : len;
  const int64_t n = hi > lo ? hi - lo : 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) vs[i] = colk[lo + i];
  __syncthreads();
  // share of sum x_i^2 over rows k+1..r-1
  double s2 = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    if (lo + i > 0) s2 = fma(vs[i], vs[i], s2);
  s2 = block_sum<QRC_WARPS>(s2, red);
  if (threadIdx.x == 0) part_s2 = s2;
  cluster.sync();
  double tot = 0.0;
  for (int rr = 0; rr < QRC; ++rr) tot += *cluster.map_shared_rank(&part_s2, rr);
  const double x0 = colk[0];
  const double normx = sqrt(x0 * x0 + tot);
  const double alpha = (x0 >= 0.0) ? -normx : normx;
  const double v0 = x0 - alpha;
  const double vv = v0 * v0 + tot;
  if (blockIdx.x == 0 && threadIdx.x == 0) Rdiag[k] = alpha;
  if (lo == 0 && n > 0 && threadIdx.x == 0) vs[0] = v0;   // the reflector's first entry
  __syncthreads();
  const int ncols = d - k - 1;
  const int mycols = ncols > cl ? (ncols - cl + ncl - 1) / ncl : 0;
  if (vv != 0.0) {
    for (int c = warp; c < mycols; c += QRC_WARPS) {
      const double* cj = A + (int64_t)(k + 1 + cl + c * ncl) * r + k + lo;
      double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
      int64_t i = lane;
      for (; i + 96 < n; i += 128) {
        p0 = fma(vs[i], cj[i], p0);
        p1 = fma(vs[i + 32], cj[i + 32], p1);
        p2 = fma(vs[i + 64], cj[i + 64], p2);
        p3 = fma(vs[i + 96], cj[i + 96], p3);
      }
      for (; i < n; i += 32) p0 = fma(vs[i], cj[i], p0);
      const double p = warp_allsum((p0 + p1) + (p2 + p3));
      if (lane == 0) pdot[c] = p;
    }
  }
  cluster.sync();
  if (vv != 0.0) {
    const double tau = 2.0 / vv;
    for (int c = warp; c < mycols; c += QRC_WARPS) {
      double sj = 0.0;
      for (int rr = 0; rr < QRC; ++rr) sj += *cluster.map_shared_rank(&pdot[c], rr);
      const double f = tau * sj;
      double* cj = A + (int64_t)(k + 1 + cl + c * ncl) * r + k + lo;
      int64_t i = lane;
      for (; i + 96 < n; i += 128) {
        const double c0 = cj[i], c1 = cj[i + 32], c2 = cj[i + 64], c3 = cj[i + 96];
        cj[i] = fma(-f, vs[i], c0);
        cj[i + 32] = fma(-f, vs[i + 32], c1);
        cj[i + 64] = fma(-f, vs[i + 64], c2);
        cj[i + 96] = fma(-f, vs[i + 96], c3);
      }
      for (; i < n; i += 32) cj[i] = fma(-f, vs[i], cj[i]);
    }
  }
  cluster.sync();   // no CTA leaves while another still reads its shared memory
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
  int ncl = c->num_sms / QRC;
  if (ncl < 1) ncl = 1;
  const bool use_cluster = ((d - 1 + ncl - 1) / ncl) <= QRC_MAXCOLS &&
                           (r + QRC - 1) / QRC <= QRC_MAXCHUNK;
  if (use_cluster)
    SPCG_CK(cudaFuncSetAttribute(k_householder_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(QRC_MAXCHUNK * sizeof(double))));
  const size_t stage_cap = 200 * 1024;
  const int staged = (size_t)r * 8 <= stage_cap;
  if (!use_cluster && staged)
    SPCG_CK(cudaFuncSetAttribute(k_householder_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)r * 8)));
  for (int k = 0; k < d; ++k) {
    const int cols = d - k - 1;
    if (use_cluster) {
      int g = cols < ncl ? cols : ncl;   // clusters with at least one column
      if (g < 1) g = 1;
      const size_t chunk_bytes = (size_t)((r - k + QRC - 1) / QRC) * sizeof(double);
      k_householder_cluster<<<g * QRC, QRC_WARPS * 32, chunk_bytes, c->stream>>>(s.Ahat, r, d, k,
                                                                                s.Rdiag);
    } else {
      int grid = (cols + QR_WARPS - 1) / QR_WARPS;
      if (grid < 1) grid = 1;
      const size_t smem = staged ? (size_t)(r - k) * 8 : 0;
      k_householder_step<<<grid, QR_WARPS * 32, smem, c->stream>>>(s.Ahat, r, d, k, s.Rdiag,
                                                                   staged);
    }
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
