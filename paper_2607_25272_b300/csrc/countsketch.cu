// CountSketch initialisation of SPCG-CS (Sec. 3 after Theorem 3.4, Sec. 4.3):
// S has one +-1 per column, in a uniform bucket h(j), so S [X Y] is a
// scatter-add of signed rows and costs O(Nd).  Stage i uses h(j) mod m_i
// (all m_i powers of two), i.e. bucket t of stage i collects buckets
// t, t + m_i, ... of the top stage: the stages come from folding one
// scatter.  The preconditioner S-hat is an independent r-bucket CountSketch.
//
// The scatter adds 64-bit fixed-point values (the per-column scales of the
// transform, which keep every sum of N terms below 2^62) with integer
// atomics: integer addition is associative, so the bucket sums are exact
// and independent of the order in which rows arrive.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.hpp"

namespace spcg {

__device__ __forceinline__ long long fx(double x, int s) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;
  const unsigned long long mant = (unsigned long long)(b & 0xFFFFFFFFFFFFFll) | (1ull << 52);
  const int sh = e - 1075 + s;
  unsigned long long q;
  if (sh >= 0) q = mant << sh;
  else if (sh > -64) q = (mant + (1ull << (-sh - 1))) >> (-sh);
  else q = 0;
  return (b < 0) ? -(long long)q : (long long)q;
}

__device__ __forceinline__ double unfx(long long q, int s) {
  if (q == 0) return 0.0;
  const unsigned long long sign = q < 0 ? 1ull : 0ull;
  const unsigned long long v = sign ? (unsigned long long)(-q) : (unsigned long long)q;
  int top = 63 - __clzll((long long)v);
  unsigned long long m;
  if (top <= 52) {
    m = v << (52 - top);
  } else {
    const int drop = top - 52;
    m = v >> drop;
    const unsigned long long rem = v & ((1ull << drop) - 1), half = 1ull << (drop - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++top;
    }
  }
  const int biased = top - s + 1023;
  if (biased <= 0) return 0.0;
  return __longlong_as_double(
      (long long)((sign << 63) | ((unsigned long long)biased << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

constexpr uint32_t TAG_CS = 4, TAG_CS_HAT = 5;

// One warp per row: lane 0 draws the buckets and signs, every lane adds a
// slice of the row's columns to the two sketches.
__global__ void __launch_bounds__(256) k_cs_scatter(const double* __restrict__ X, int64_t ldx,
                                                    const double* __restrict__ Y, int64_t N,
                                                    int d, uint64_t seed, int64_t mK, int64_t r,
                                                    const int* __restrict__ shift,
                                                    unsigned long long* __restrict__ top,
                                                    unsigned long long* __restrict__ hat) {
  const int lane = threadIdx.x & 31;
  const int C = d + 1;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t j = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); j < N; j += warps) {
    uint32_t b = 0, bh = 0, sg = 0, sgh = 0;
    if (lane == 0) {
      const u32x4 w = philox10(u32x4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), TAG_CS, 0u}, seed);
      b = w.x & (uint32_t)(mK - 1);
      sg = w.y & 1u;
      const u32x4 wh =
          philox10(u32x4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), TAG_CS_HAT, 0u}, seed);
      bh = (uint32_t)(((uint64_t)wh.x * (uint64_t)r) >> 32);
      sgh = wh.y & 1u;
    }
    b = __shfl_sync(0xffffffffu, b, 0);
    sg = __shfl_sync(0xffffffffu, sg, 0);
    bh = __shfl_sync(0xffffffffu, bh, 0);
    sgh = __shfl_sync(0xffffffffu, sgh, 0);
    for (int c = lane; c < C; c += 32) {
      const long long q = fx((c < d) ? X[j * ldx + c] : Y[j], shift[c]);
      atomicAdd(top + (int64_t)b * C + c, (unsigned long long)(sg ? -q : q));
      if (c < d) atomicAdd(hat + (int64_t)bh * C + c, (unsigned long long)(sgh ? -q : q));
    }
  }
}

// Fold the top buckets in half: row t += row t + half, t < half.
__global__ void k_cs_fold(long long* __restrict__ top, int64_t half, int C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < half * C;
       e += (int64_t)gridDim.x * blockDim.x)
    top[e] += top[e + half * C];
}

// Rows [0, m) of the folded buckets to a stage's FP64 or BF16 matrix and b.
__global__ void k_cs_convert(const long long* __restrict__ top, int64_t m, int d,
                             const int* __restrict__ shift, double* __restrict__ A, int64_t lda,
                             __nv_bfloat16* __restrict__ A16, int64_t lda16,
                             double* __restrict__ b) {
  const int C = d + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * C;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / C;
    const int c = (int)(e % C);
    const double z = unfx(top[e], shift[c]);
    if (c < d) {
      if (A) A[t * lda + c] = z;
      if (A16) A16[t * lda16 + c] = __double2bfloat16(z);
    } else {
      b[t] = z;
    }
  }
}

// S-hat X to the column-major r x d matrix the QR reduces.
__global__ void k_cs_hat_convert(const long long* __restrict__ hat, int64_t r, int d,
                                 const int* __restrict__ shift, double* __restrict__ Ahat) {
  const int C = d + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / d;
    const int c = (int)(e % d);
    Ahat[(int64_t)c * r + t] = unfx(hat[t * C + c], shift[c]);
  }
}

spcg_status launch_countsketch(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int d = c->d, C = d + 1;
  const spcg_schedule& sc = s.sched;
  const int64_t mK = sc.m[sc.K - 1];
  const int64_t r = sc.r;
  long long* top = reinterpret_cast<long long*>(s.work);
  long long* hat = top + mK * C;
  SPCG_CK(cudaMemsetAsync(top, 0, (size_t)(mK + r) * C * 8, c->stream));
  // the fixed-point scales: per-column maxima as for the transform
  SPCG_TRY(launch_colscales(c));
  const int grid = 8 * c->num_sms;
  k_cs_scatter<<<grid, 256, 0, c->stream>>>(c->X, c->ldx, c->Y, c->N, d, s.seed, mK, r,
                                            s.colshift, reinterpret_cast<unsigned long long*>(top),
                                            reinterpret_cast<unsigned long long*>(hat));
  SPCG_CK(cudaGetLastError());
  k_cs_hat_convert<<<grid, 256, 0, c->stream>>>(hat, r, d, s.colshift, s.Ahat);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 2;
  int64_t cur = mK;
  for (int i = sc.K - 1; i >= 0; --i) {
    while (cur > sc.m[i]) {
      cur /= 2;
      k_cs_fold<<<grid, 256, 0, c->stream>>>(top, cur, C);
      SPCG_CK(cudaGetLastError());
      c->n_launch += 1;
    }
    double* A = s.mixed ? nullptr : s.AK + s.stage_off[i] * s.ldak;
    __nv_bfloat16* A16 =
        s.mixed ? reinterpret_cast<__nv_bfloat16*>(s.AK16) + s.stage_off[i] * s.ldak16 : nullptr;
    k_cs_convert<<<grid, 256, 0, c->stream>>>(top, cur, d, s.colshift, A, s.ldak, A16, s.ldak16,
                                              s.bK + s.stage_off[i]);
    SPCG_CK(cudaGetLastError());
    c->n_launch += 1;
  }
  return SPCG_OK;
}

}  // namespace spcg
