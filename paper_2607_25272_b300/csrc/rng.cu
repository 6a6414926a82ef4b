// Counter-based draws of the SRHT (Sec. 2.1): Rademacher signs D, the
// permutation P, the nested order pi of I_1 c ... c I_K (Sec. 2.2) and the
// independent preconditioner rows I-hat, all from Philox4x32-10 keyed by the
// seed.  The permutations are Feistel networks over index bits, so every
// index is mapped (or inverted) in O(1) without a sort.
#include "common.cuh"
#include "internal.hpp"

namespace spcg {

__global__ void k_philox(const uint32_t* __restrict__ ctr, uint64_t seed, int64_t n,
                         uint32_t* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    u32x4 c{ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3]};
    u32x4 o = philox10(c, seed);
    out[4 * j] = o.x;
    out[4 * j + 1] = o.y;
    out[4 * j + 2] = o.z;
    out[4 * j + 3] = o.w;
  }
}

__global__ void k_feistel(uint64_t seed, int nbits, uint32_t tag, int64_t count, int inverse,
                          int64_t* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (int64_t)feistel((uint32_t)t, nbits, tag, seed, inverse != 0);
}

__global__ void k_signs(uint64_t seed, int64_t n, double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (double)rademacher((uint64_t)k, seed);
}

// For every row j of the padded transform:
//   gather[j] = P(j) with bit 31 set when D_j = -1 ((D P X')_j = D_j X'_{P(j)})
//   dest[j]   = pi^{-1}(j) if it is < m_K (row j belongs to I_K), else -1
//   hdest[j]  = sigma_hat^{-1}(j) if it is < r (row j belongs to I-hat), else -1
// dest and hdest are stored in the row order of the transform's last pass
// (its rows j = low + t 2^last_shift, t < 2^last_logl, at index
// low 2^last_logl + t), so that the pass reads its tile's entries
// contiguously; with one pass that order is j itself.
__global__ void k_sketch_maps(int nbits, uint64_t seed, int64_t n_pad, int64_t mK, int64_t r,
                              int last_shift, int last_logl, uint32_t* __restrict__ gather,
                              int32_t* __restrict__ dest, int32_t* __restrict__ hdest) {
  const int64_t low_mask = (int64_t(1) << last_shift) - 1;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_pad;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t src = feistel((uint32_t)j, nbits, TAG_P, seed, false);
    const int sgn = rademacher((uint64_t)j, seed);
    gather[j] = src | (sgn < 0 ? 0x80000000u : 0u);
    const int64_t jl = ((j & low_mask) << last_logl) | (j >> last_shift);
    const uint32_t t = feistel((uint32_t)j, nbits, TAG_PI, seed, true);
    dest[jl] = ((int64_t)t < mK) ? (int32_t)t : -1;
    const uint32_t th = feistel((uint32_t)j, nbits, TAG_HAT, seed, true);
    hdest[jl] = ((int64_t)th < r) ? (int32_t)th : -1;
  }
}

static int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 148 * 32) g = 148 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

spcg_status launch_sketch_maps(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int64_t mK = s.sched.K > 0 ? s.sched.m[s.sched.K - 1] : 0;
  int logl[8];
  const int passes = fwht_pass_plan(s.nbits, logl, c->opts.fwht_first_levels);
  const int last_logl = logl[passes - 1], last_shift = s.nbits - last_logl;
  k_sketch_maps<<<grid_for(s.n_pad, 256), 256, 0, c->stream>>>(
      s.nbits, s.seed, s.n_pad, mK, s.sched.r, last_shift, last_logl, s.gather, s.dest, s.hdest);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 1;
  return SPCG_OK;
}

}  // namespace spcg

using namespace spcg;

extern "C" spcg_status spcg_philox(const uint32_t* ctr, uint64_t seed, int64_t n, uint32_t* out,
                                   void* stream) {
  if (n < 0 || ((!ctr || !out) && n > 0)) return SPCG_E_INVALID_ARG;
  if (n == 0) return SPCG_OK;
  k_philox<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(ctr, seed, n, out);
  SPCG_CK(cudaGetLastError());
  SPCG_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SPCG_OK;
}

extern "C" spcg_status spcg_feistel(uint64_t seed, int32_t nbits, int32_t tag, int64_t count,
                                    int32_t inverse, int64_t* out, void* stream) {
  if (nbits < 0 || nbits > 30 || count < 0 || count > (int64_t(1) << nbits) || tag < 0 ||
      (!out && count > 0))
    return SPCG_E_INVALID_ARG;
  if (count == 0) return SPCG_OK;
  k_feistel<<<grid_for(count, 256), 256, 0, (cudaStream_t)stream>>>(seed, nbits, (uint32_t)tag,
                                                                    count, inverse, out);
  SPCG_CK(cudaGetLastError());
  SPCG_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SPCG_OK;
}

extern "C" spcg_status spcg_signs(uint64_t seed, int64_t n, double* out, void* stream) {
  if (n < 0 || (!out && n > 0)) return SPCG_E_INVALID_ARG;
  if (n == 0) return SPCG_OK;
  k_signs<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(seed, n, out);
  SPCG_CK(cudaGetLastError());
  SPCG_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SPCG_OK;
}
