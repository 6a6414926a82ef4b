// Batched SPCG: many independent least-squares problems of uneven N and d,
// FP32 storage, solved by one persistent kernel.
//
// Each CTA is a complete SPCG solver: it takes the next problem from a work
// queue (problems sorted largest first, so the longest solves start first)
// and runs the whole method on it with CTA-level synchronisation only, then
// takes the next.  No CTA ever waits on another.
//
// Per problem (Algorithm 1 with the CountSketch initialisation of SPCG-CS,
// Sec. 4.3, whose O(Nd) cost suits problems this small):
//   1. column maxima of [X Y] -> 64-bit fixed-point scales;
//   2. one read of [X Y]: signed rows scattered into m_K + r buckets with
//      exact integer atomics (stage hash and independent preconditioner hash);
//   3. stage matrices by folding the buckets modulo m_i, as FP32;
//   4. Householder QR of the r x d preconditioner sketch (FP32), R^{-1};
//   5. warm-started PCG on every stage and Stage II on X with the stopping
//      rule of the single-problem path: the streaming passes read row chunks
//      with bulk asynchronous copies (cp.async.bulk) into a shared-memory
//      ring guarded by mbarriers; the true gradients X^T (Y - X beta) use
//      double-FP32 arithmetic (TwoProd/TwoSum) so that the stopping rule sees
//      an FP64-accurate gradient of the FP32-valued problem.
// The rows per chunk (the tile) are chosen per width class by an autotuner
// on the host.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.hpp"

namespace spcg {

constexpr int BW = 16;                    // consumer warps
constexpr int BT = 32 * (BW + 1);         // + one producer warp
constexpr int B_STAGES = 6;
constexpr int B_MAXD = 256;
constexpr int B_NI = B_MAXD / 32;         // columns per lane
constexpr int B_RU = 4;                   // rows (or elements) a thread loads at once outside the ring
constexpr int B_SR = 4;                   // rows of a stage bucket loaded at once (lane per bucket)
constexpr int B_CCH = 8;                  // columns per chunk of a stage bucket (lane per bucket)

struct BatchProblemDev {
  const float* X;
  const float* Y;
  int64_t N;
  int64_t ldx;
  int d;
  int K;
  int64_t m[SPCG_MAX_STAGES];
  int a[SPCG_MAX_STAGES];
  int64_t r;
  int tile_rows;            // rows per streamed chunk (autotuned)
  double* beta;             // output
  int* status;              // output: 0 ok, 4 breakdown, 5 not converged, 6 timeout
  int* iters;               // output: Stage II iterations
};

struct BatchArgs {
  const BatchProblemDev* probs;
  int n;
  int* queue;
  unsigned char* scratch;   // gridDim.x x scratch_bytes
  size_t scratch_bytes;
  int64_t max_rows_int;     // rows of the int64 bucket area (max m_K + r)
  int64_t max_stage_rows;   // rows of the FP32 stage area (max sum m_i)
  int64_t max_r;
  uint64_t seed;
  double tol;
  int max_iters;
  int max_restarts;
  long long spin;
  int64_t max_n;            // rows of the largest problem (row lists)
  long long* phase_cycles;  // n x 8 clock cycles per phase of each problem, or null
};

// ---------------- small helpers ----------------
__device__ __forceinline__ uint32_t b_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void b_mbar_init(uint64_t* bar, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_smem(bar)), "r"(c) : "memory");
}
__device__ __forceinline__ void b_mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b_smem(bar)) : "memory");
}
__device__ __forceinline__ void b_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b_smem(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void b_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b_smem(bar)) : "memory");
}
__device__ __forceinline__ bool b_try(uint64_t* bar, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(b_smem(bar)), "r"(par)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool b_wait(uint64_t* bar, uint32_t par, long long budget) {
  if (b_try(bar, par)) return true;
  const long long t0 = clock64();
  while (!b_try(bar, par))
    if (clock64() - t0 > budget) return false;
  return true;
}
__device__ __forceinline__ void b_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(b_smem(dst)),
      "l"(src), "r"(bytes), "r"(b_smem(bar))
      : "memory");
}

// Exact conversions between FP32 values and 64-bit fixed point with integer
// operations only (the FP64 pipe of this GPU is slow).  q = x 2^s rounded half
// away from zero, from the FP32 bit pattern (subnormals included).
__device__ __forceinline__ long long fixed_from_f32(float x, int s) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFFu);
  uint64_t m = b & 0x7FFFFFu;
  int E;                      // x = m 2^E
  if (e == 0) {
    if (m == 0) return 0;
    E = -149;
  } else {
    m |= 0x800000u;
    E = e - 150;
  }
  const int sh = E + s;
  uint64_t q;
  if (sh >= 0) q = m << sh;                         // the scale keeps q below 2^62
  else if (sh > -40) q = (m + (1ull << (-sh - 1))) >> (-sh);
  else q = 0;
  return (b >> 31) ? -(long long)q : (long long)q;
}

// |q| 2^-s with the 53 (FP64) or 24 (FP32) leading bits, round to nearest
// even; results below the normal range flush to zero.
__device__ __forceinline__ void fixed_split(long long q, int s, int mbits, uint32_t& sign,
                                            uint64_t& mant, int& exp2) {
  sign = q < 0 ? 1u : 0u;
  const uint64_t v = sign ? (uint64_t)(-q) : (uint64_t)q;
  int top = 63 - __clzll((long long)v);
  uint64_t m;
  if (top < mbits) {
    m = v << (mbits - 1 - top);
  } else {
    const int drop = top - (mbits - 1);
    m = v >> drop;
    const uint64_t rem = drop > 0 ? v & ((1ull << drop) - 1) : 0, half = drop > 0 ? 1ull << (drop - 1) : 0;
    if (drop > 0 && (rem > half || (rem == half && (m & 1ull)))) ++m;
    if (m == (1ull << mbits)) {
      m >>= 1;
      ++top;
    }
  }
  mant = m;
  exp2 = top - s;             // value = m 2^(exp2 - (mbits - 1))
}

__device__ __forceinline__ float f32_from_fixed(long long q, int s) {
  if (q == 0) return 0.f;
  uint32_t sign;
  uint64_t m;
  int e2;
  fixed_split(q, s, 24, sign, m, e2);
  const int biased = e2 + 127;
  if (biased <= 0) return 0.f;
  if (biased >= 255) return __uint_as_float((sign << 31) | 0x7F800000u);
  return __uint_as_float((sign << 31) | ((uint32_t)biased << 23) | (uint32_t)(m & 0x7FFFFFu));
}

__device__ __forceinline__ double f64_from_fixed(long long q, int s) {
  if (q == 0) return 0.0;
  uint32_t sign;
  uint64_t m;
  int e2;
  fixed_split(q, s, 53, sign, m, e2);
  const int biased = e2 + 1023;
  if (biased <= 0) return 0.0;
  return __longlong_as_double((long long)(((uint64_t)sign << 63) | ((uint64_t)biased << 52) |
                                          (m & 0xFFFFFFFFFFFFFull)));
}

// double-FP32 helpers (error-free transformations); the _rn intrinsics keep
// the compiler from contracting a product and a sum into one FMA, which
// would break the error terms
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}

struct BShared {
  uint64_t full[B_STAGES], empty[B_STAGES];
  double dvec[6][B_MAXD];     // beta, g, z, p, w, u (FP64 d-space)
  float pf[B_MAXD];           // p (FP32) for the passes
  float bh[B_MAXD], bl[B_MAXD];   // beta as double-FP32 for true gradients
  double red[BW][B_MAXD];     // per-warp partial sums
  double scal[8];
  int colshift[B_MAXD + 1];
  uint32_t colmax32[B_MAXD + 1];    // largest |x| per column, FP32 bit pattern
  int flag;
};

// One streamed pass over rows [0, m) of a row-major FP32 matrix A (ld floats,
// 16-byte rows).  mode 0: w = A^T (A p);  mode 1: g = A^T (b - A beta) with
// b FP64 (stage start, FP32 arithmetic);  mode 2: true gradient in
// double-FP32.  The result lands in sh.red (per warp) and is summed into
// out (FP64) in warp order.
//
// A row is handled by LW lanes (LW = 32 / rows per warp, the smallest power
// of two with 8 LW >= d): lane s of a group owns columns s, s + LW, ...,
// s + 7 LW, so narrow problems put several rows in one warp instead of
// leaving most lanes idle.  Row dot products reduce over the LW lanes of a
// group (xor shuffles below LW); at the end the groups' column sums are
// added across the warp (xor shuffles at LW and above) in a fixed order.
template <int LW>
__device__ bool stream_pass_lw(BShared& sh, unsigned char* ring, size_t ring_bytes,
                               const float* A, int64_t m, int64_t ld, int d, int tile_rows,
                               int mode, const double* bvec64, const float* bvec32, double* out,
                               long long spin) {
  constexpr int RPW = 32 / LW;              // rows per warp
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sub = lane % LW, grp = lane / LW;
  const int64_t chunk_rows = tile_rows;
  const size_t chunk_bytes = (size_t)chunk_rows * ld * 4;
  const int nst = (int)((ring_bytes / chunk_bytes) < B_STAGES ? (ring_bytes / chunk_bytes) : B_STAGES);
  const int64_t nchunks = (m + chunk_rows - 1) / chunk_rows;
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      b_mbar_init(&sh.full[s], 1);
      b_mbar_init(&sh.empty[s], BW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    sh.flag = 0;
  }
  __syncthreads();
  float acc[B_NI], cmp[B_NI];
#pragma unroll
  for (int i = 0; i < B_NI; ++i) acc[i] = cmp[i] = 0.f;
  // this lane's columns of p or beta (zero beyond d)
  float pv[B_NI], blo[B_NI];
#pragma unroll
  for (int i = 0; i < B_NI; ++i) {
    const int c = sub + LW * i;
    pv[i] = (c < B_MAXD) ? (mode == 0 ? sh.pf[c] : sh.bh[c]) : 0.f;
    blo[i] = (c < B_MAXD && mode == 2) ? sh.bl[c] : 0.f;
  }
  bool ok = true;
  if (warp == BW) {
    if (lane == 0) {
      for (int64_t k = 0; k < nchunks; ++k) {
        const int s = (int)(k % nst);
        if (k >= nst && !b_wait(&sh.empty[s], (uint32_t)(((k / nst) - 1) & 1), spin)) {
          sh.flag = 1;
          break;
        }
        if (*(volatile int*)&sh.flag) break;
        const int64_t r0 = k * chunk_rows;
        const int64_t rows = (m - r0 < chunk_rows) ? m - r0 : chunk_rows;
        const uint32_t bytes = (uint32_t)(rows * ld * 4);
        b_expect(&sh.full[s], bytes);
        b_bulk(ring + (size_t)s * chunk_bytes, A + r0 * ld, bytes, &sh.full[s]);
      }
    }
  } else {
    for (int64_t k = 0; k < nchunks; ++k) {
      const int s = (int)(k % nst);
      if (!b_wait(&sh.full[s], (uint32_t)((k / nst) & 1), spin)) {
        sh.flag = 1;
        ok = false;
        break;
      }
      const float* tile = reinterpret_cast<const float*>(ring + (size_t)s * chunk_bytes);
      const int64_t r0 = k * chunk_rows;
      const int64_t rows = (m - r0 < chunk_rows) ? m - r0 : chunk_rows;
      for (int64_t base = (int64_t)warp * RPW; base < rows; base += (int64_t)BW * RPW) {
        const int64_t rr = base + grp;
        const bool live = rr < rows;
        const float* row = tile + (size_t)(live ? rr : 0) * ld;
        float x[B_NI];
#pragma unroll
        for (int i = 0; i < B_NI; ++i) {
          const int c = sub + LW * i;
          x[i] = (live && c < d) ? row[c] : 0.f;
        }
        if (mode == 0 || mode == 1) {
          float t = 0.f;
#pragma unroll
          for (int i = 0; i < B_NI; ++i) t = fmaf(x[i], pv[i], t);
#pragma unroll
          for (int o = LW / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (mode == 1) t = live ? (float)bvec64[r0 + rr] - t : 0.f;
#pragma unroll
          for (int i = 0; i < B_NI; ++i) {
            float pr, pe, s2, se;
            two_prod(t, x[i], pr, pe);
            two_sum(acc[i], pr, s2, se);
            acc[i] = s2;
            cmp[i] += pe + se;
          }
        } else {
          // t = y - x . beta in double-FP32 (Dot2 on the hi part, the lo part plain)
          float sh_ = 0.f, sl = 0.f;
#pragma unroll
          for (int i = 0; i < B_NI; ++i) {
            float pr, pe, s2, se;
            two_prod(x[i], pv[i], pr, pe);
            two_sum(sh_, pr, s2, se);
            sh_ = s2;
            sl += pe + se + x[i] * blo[i];
          }
          // group all-reduce of the pair (hi, lo): hi with TwoSum, lo plainly,
          // commutative so both partner lanes end with the same bits
#pragma unroll
          for (int o = LW / 2; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh_, o);
            const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
            float s2, se;
            two_sum(sh_, oh, s2, se);
            sh_ = s2;
            sl = __fadd_rn(__fadd_rn(sl, ol), se);
          }
          const float y = live ? bvec32[r0 + rr] : 0.f;
          float th, tl;
          two_sum(y, -sh_, th, tl);
          tl -= sl;
#pragma unroll
          for (int i = 0; i < B_NI; ++i) {
            float pr, pe, s2, se;
            two_prod(th, x[i], pr, pe);
            two_sum(acc[i], pr, s2, se);
            acc[i] = s2;
            cmp[i] += pe + se + tl * x[i];
          }
        }
      }
      __syncwarp();
      if (lane == 0) b_arrive(&sh.empty[s]);
    }
  }
  __syncthreads();
  if (sh.flag) ok = false;
  if (warp < BW) {
#pragma unroll
    for (int i = 0; i < B_NI; ++i) {
      double v = (double)acc[i] + (double)cmp[i];
      // add the groups' sums of the same column (fixed xor order)
#pragma unroll
      for (int o = LW; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const int c = sub + LW * i;
      if (grp == 0 && c < d) sh.red[warp][c] = v;
    }
  }
  __syncthreads();
  for (int c = tid; c < d; c += blockDim.x) {
    double sacc = 0.0;
    for (int w = 0; w < BW; ++w) sacc += sh.red[w][c];
    out[c] = sacc;
  }
  if (tid == 0)
    for (int s = 0; s < nst; ++s) {
      b_mbar_inval(&sh.full[s]);
      b_mbar_inval(&sh.empty[s]);
    }
  __syncthreads();
  return ok;
}

__device__ bool stream_pass(BShared& sh, unsigned char* ring, size_t ring_bytes, const float* A,
                            int64_t m, int64_t ld, int d, int tile_rows, int mode,
                            const double* bvec64, const float* bvec32, double* out,
                            long long spin) {
  if (d <= 8)
    return stream_pass_lw<1>(sh, ring, ring_bytes, A, m, ld, d, tile_rows, mode, bvec64, bvec32,
                             out, spin);
  if (d <= 16)
    return stream_pass_lw<2>(sh, ring, ring_bytes, A, m, ld, d, tile_rows, mode, bvec64, bvec32,
                             out, spin);
  if (d <= 32)
    return stream_pass_lw<4>(sh, ring, ring_bytes, A, m, ld, d, tile_rows, mode, bvec64, bvec32,
                             out, spin);
  if (d <= 64)
    return stream_pass_lw<8>(sh, ring, ring_bytes, A, m, ld, d, tile_rows, mode, bvec64, bvec32,
                             out, spin);
  if (d <= 128)
    return stream_pass_lw<16>(sh, ring, ring_bytes, A, m, ld, d, tile_rows, mode, bvec64, bvec32,
                              out, spin);
  return stream_pass_lw<32>(sh, ring, ring_bytes, A, m, ld, d, tile_rows, mode, bvec64, bvec32,
                            out, spin);
}

// Block-wide deterministic sum of one double per thread.
__device__ double bsum(double v, double* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_allsum(v);
  __syncthreads();
  if (lane == 0) tmp[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += tmp[w];
  __syncthreads();
  return s;
}

// z = R^{-1} (R^{-T} g) with FP32 triangular factors (u = scratch).
__device__ void precond(const float* Rinv, const float* RinvT, int d, const double* g, double* u,
                        double* z) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < d; i += nw) {
    const float* row = RinvT + (size_t)i * d;
    float s = 0.f;
    for (int j = lane; j <= i; j += 32) s = fmaf(row[j], (float)g[j], s);
    s = warp_allsum(s);
    if (lane == 0) u[i] = s;
  }
  __syncthreads();
  for (int i = warp; i < d; i += nw) {
    const float* row = Rinv + (size_t)i * d;
    float s = 0.f;
    for (int j = i + lane; j < d; j += 32) s = fmaf(row[j], (float)u[j], s);
    s = warp_allsum(s);
    if (lane == 0) z[i] = s;
  }
  __syncthreads();
}

constexpr size_t B_RING = (size_t)B_STAGES * 16384;
static_assert((size_t)6 * B_MAXD * sizeof(float) <= B_RING,
              "the QR stages a reflector of r = 6d <= 1536 rows in the ring");
constexpr size_t B_SMEM = B_RING + ((sizeof(BShared) + 127) & ~(size_t)127) + 128;

__global__ void __launch_bounds__(BT, 1) k_batched_spcg(const BatchArgs a) {
  extern __shared__ unsigned char dyn_raw[];
  unsigned char* dyn = dyn_raw + ((128u - (b_smem(dyn_raw) & 127u)) & 127u);
  unsigned char* ring = dyn;
  BShared& sh = *reinterpret_cast<BShared*>(dyn + B_RING);
  __shared__ int s_p;
  __shared__ double tmp[BT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = BT / 32;
  const size_t ring_bytes = B_RING;
  unsigned char* scr = a.scratch + (size_t)blockIdx.x * a.scratch_bytes;
  long long* buckets = reinterpret_cast<long long*>(scr);
  float* stages = reinterpret_cast<float*>(scr + (size_t)a.max_rows_int * (B_MAXD + 1) * 8);
  double* bst = reinterpret_cast<double*>(stages + (size_t)a.max_stage_rows * B_MAXD);
  float* Ahat = reinterpret_cast<float*>(bst + a.max_stage_rows);
  float* R = Ahat + (size_t)a.max_r * B_MAXD;
  float* Rinv = R + B_MAXD * B_MAXD;
  float* RinvT = Rinv + B_MAXD * B_MAXD;
  int* cnt = reinterpret_cast<int*>(RinvT + B_MAXD * B_MAXD);   // bucket sizes, then offsets
  int* cur = cnt + a.max_rows_int;                              // bucket fill cursors
  int32_t* rlist = cur + a.max_rows_int;                        // row lists (2 x max_n)
  __shared__ int sh_scan[BT];

  for (;;) {
    if (tid == 0) s_p = atomicAdd(a.queue, 1);
    __syncthreads();
    const int p = s_p;
    if (p >= a.n) break;
    const BatchProblemDev& P = a.probs[p];
    const int d = P.d, C = d + 1;
    const int64_t N = P.N, ldx = P.ldx;
    const int64_t n_pad = (int64_t)1 << (64 - __clzll((long long)(N - 1)));
    const int nbits = 63 - __clzll((long long)n_pad);
    const int K = P.K;
    const int64_t mK = K > 0 ? P.m[K - 1] : 0, r = P.r;
    const int ld = (d + 3) & ~3;   // stage rows: 16-byte aligned
    const uint64_t key = a.seed + (uint64_t)p;
    int status = 0;

    long long t_phase = clock64();
    auto phase_mark = [&](int k) {
      if (a.phase_cycles && tid == 0) {
        const long long t = clock64();
        a.phase_cycles[(size_t)p * 8 + k] = t - t_phase;
        t_phase = t;
      }
    };
    // 1. column maxima of |[X Y]| (FP32 bit patterns: integer order is numeric
    //    order for non-negative floats) -> fixed-point scales
    for (int c = tid; c < C; c += blockDim.x) sh.colmax32[c] = 0u;
    __syncthreads();
    {
      uint32_t mx[(B_MAXD + 1 + 31) / 32];
#pragma unroll
      for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) mx[u] = 0u;
      // B_RU rows per warp and step, all loads issued before the maxima
      for (int64_t i0 = (int64_t)warp * B_RU; i0 < N; i0 += (int64_t)nw * B_RU) {
        float v[B_RU][(B_MAXD + 1 + 31) / 32];
#pragma unroll
        for (int q = 0; q < B_RU; ++q)
#pragma unroll
          for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) {
            const int c = lane + 32 * u;
            const int64_t i = i0 + q;
            v[q][u] = (c < C && i < N) ? ((c < d) ? P.X[i * ldx + c] : P.Y[i]) : 0.f;
          }
#pragma unroll
        for (int q = 0; q < B_RU; ++q)
#pragma unroll
          for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) {
            const uint32_t bits = __float_as_uint(v[q][u]) & 0x7FFFFFFFu;
            mx[u] = bits > mx[u] ? bits : mx[u];
          }
      }
#pragma unroll
      for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) {
        const int c = lane + 32 * u;
        if (c < C && mx[u]) atomicMax(&sh.colmax32[c], mx[u]);
      }
    }
    __syncthreads();
    for (int c = tid; c < C; c += blockDim.x) {
      // s_c = 61 - n - E_c with 2^{E_c} <= max_c < 2^{E_c+1}: every sum of
      // N' <= 2^n terms stays below 2^62
      const uint32_t bits = sh.colmax32[c];
      const int e = (int)(bits >> 23);
      int E = 0;
      if (e > 0) E = e - 127;
      else if (bits) E = (31 - __clz((int)bits)) - 149;
      sh.colshift[c] = bits == 0 ? 0 : 61 - nbits - E;
    }
    phase_mark(0);
    // 2. CountSketch by gathering: bucket sizes (one integer atomic per row and
    //    sketch, on arrays small enough to stay in L2), offsets, a row list
    //    per bucket, then every bucket sums its rows in 64-bit registers and
    //    is written once.  Integer sums: the order of the rows in a bucket
    //    does not change a bit.
    const int64_t nb = mK + r;
    for (int64_t e = tid; e < nb; e += blockDim.x) cnt[e] = 0;
    __syncthreads();
    for (int64_t j = tid; j < N; j += blockDim.x) {
      const u32x4 w = philox10(u32x4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 4u, 0u}, key);
      const u32x4 wh = philox10(u32x4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 5u, 0u}, key);
      if (mK > 0) atomicAdd(&cnt[w.x & (uint32_t)(mK - 1)], 1);
      atomicAdd(&cnt[mK + (int64_t)(((uint64_t)wh.x * (uint64_t)r) >> 32)], 1);
    }
    __syncthreads();
    {
      // exclusive scan of cnt[0, nb) (stage buckets, then preconditioner
      // buckets, so those offsets start at N): per-thread chunks, then the
      // chunk totals
      const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
      const int64_t lo = (int64_t)tid * per, hi = lo + per < nb ? lo + per : nb;
      int tsum = 0;
      for (int64_t e = lo; e < hi; ++e) tsum += cnt[e];
      sh_scan[tid] = tsum;
      __syncthreads();
      if (tid == 0) {
        int run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
          const int v = sh_scan[k];
          sh_scan[k] = run;
          run += v;
        }
      }
      __syncthreads();
      int run = sh_scan[tid];
      for (int64_t e = lo; e < hi; ++e) {
        const int v = cnt[e];
        cnt[e] = run;
        cur[e] = run;
        run += v;
      }
    }
    __syncthreads();
    for (int64_t j = tid; j < N; j += blockDim.x) {
      const u32x4 w = philox10(u32x4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 4u, 0u}, key);
      const u32x4 wh = philox10(u32x4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 5u, 0u}, key);
      if (mK > 0) {
        const int slot = atomicAdd(&cur[w.x & (uint32_t)(mK - 1)], 1);
        rlist[slot] = (int32_t)((uint32_t)j | ((w.y & 1u) << 31));
      }
      const int slot = atomicAdd(&cur[mK + (int64_t)(((uint64_t)wh.x * (uint64_t)r) >> 32)], 1);
      rlist[slot] = (int32_t)((uint32_t)j | ((wh.y & 1u) << 31));
    }
    __syncthreads();
    phase_mark(1);
    // bucket sums.  Stage buckets (about two rows each, N'/2 of them): a lane
    // per bucket, columns in chunks of 8 (two 16-byte loads per row), the
    // first B_SR rows' loads of a chunk issued before their sums, so that a
    // CTA keeps hundreds of buckets' rows in flight.  Preconditioner buckets
    // (N / r rows each): a warp per bucket, lanes over the columns, the loads
    // of B_RU rows issued before their sums.
    {
      constexpr int CCH = B_CCH;
      for (int64_t tb = (int64_t)warp * 32; tb < mK; tb += (int64_t)nw * 32) {
        const int64_t t = tb + lane;
        const bool live = t < mK;
        const int k0 = live ? cnt[t] : 0, k1 = live ? cur[t] : 0;
        uint32_t ent[B_SR];
#pragma unroll
        for (int q = 0; q < B_SR; ++q) ent[q] = k0 + q < k1 ? (uint32_t)rlist[k0 + q] : 0u;
        for (int c0 = 0; c0 < C; c0 += CCH) {
          long long acc[CCH];
#pragma unroll
          for (int u = 0; u < CCH; ++u) acc[u] = 0;
          const bool vec = c0 + CCH <= d;   // eight columns of X, 16-byte aligned
          for (int kb = k0; kb < k1; kb += B_SR) {
            float v[B_SR][CCH];
#pragma unroll
            for (int q = 0; q < B_SR; ++q) {
              const uint32_t e = kb == k0 ? ent[q] : (kb + q < k1 ? (uint32_t)rlist[kb + q] : 0u);
              const int64_t j = e & 0x7FFFFFFFu;   // rows past the bucket read row 0
              if (vec) {
#pragma unroll
                for (int h = 0; h < CCH / 4; ++h) {
                  const float4 a4 = *reinterpret_cast<const float4*>(P.X + j * ldx + c0 + 4 * h);
                  v[q][4 * h] = a4.x;
                  v[q][4 * h + 1] = a4.y;
                  v[q][4 * h + 2] = a4.z;
                  v[q][4 * h + 3] = a4.w;
                }
              } else {
#pragma unroll
                for (int u = 0; u < CCH; ++u) {
                  const int c = c0 + u;
                  v[q][u] = c < d ? P.X[j * ldx + c] : (c == d ? P.Y[j] : 0.f);
                }
              }
            }
#pragma unroll
            for (int q = 0; q < B_SR; ++q) {
              if (kb + q >= k1) break;
              const uint32_t e = kb == k0 ? ent[q] : (uint32_t)rlist[kb + q];
#pragma unroll
              for (int u = 0; u < CCH; ++u) {
                const int c = c0 + u;
                if (c < C) {
                  const long long fq = fixed_from_f32(v[q][u], sh.colshift[c]);
                  acc[u] += (e >> 31) ? -fq : fq;
                }
              }
            }
          }
          if (live)
#pragma unroll
            for (int u = 0; u < CCH; ++u)
              if (c0 + u < C) buckets[t * C + c0 + u] = acc[u];
        }
      }
      for (int64_t t = mK + warp; t < nb; t += nw) {
        long long acc[(B_MAXD + 1 + 31) / 32];
#pragma unroll
        for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) acc[u] = 0;
        const int k1 = cur[t];
        for (int k0 = cnt[t]; k0 < k1; k0 += B_RU) {
          float v[B_RU][(B_MAXD + 1 + 31) / 32];
          uint32_t ent[B_RU];
#pragma unroll
          for (int q = 0; q < B_RU; ++q) ent[q] = k0 + q < k1 ? (uint32_t)rlist[k0 + q] : 0u;
#pragma unroll
          for (int q = 0; q < B_RU; ++q) {
            const int64_t j = ent[q] & 0x7FFFFFFFu;
#pragma unroll
            for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) {
              const int c = lane + 32 * u;
              v[q][u] = (c < C && k0 + q < k1) ? ((c < d) ? P.X[j * ldx + c] : P.Y[j]) : 0.f;
            }
          }
#pragma unroll
          for (int q = 0; q < B_RU; ++q)
#pragma unroll
            for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) {
              const int c = lane + 32 * u;
              if (c < C) {
                const long long fq = fixed_from_f32(v[q][u], sh.colshift[c]);
                acc[u] += (ent[q] >> 31) ? -fq : fq;   // rows past the bucket hold 0
              }
            }
        }
#pragma unroll
        for (int u = 0; u < (B_MAXD + 1 + 31) / 32; ++u) {
          const int c = lane + 32 * u;
          if (c < d) Ahat[(int64_t)c * r + (t - mK)] = f32_from_fixed(acc[u], sh.colshift[c]);
        }
      }
    }
    __syncthreads();
    phase_mark(2);
    // 3. stage matrices by folding the buckets modulo m_i (integer adds)
    int64_t off[SPCG_MAX_STAGES];
    {
      int64_t o = 0;
      for (int i = 0; i < K; ++i) {
        off[i] = o;
        o += P.m[i];
      }
    }
    int64_t cur_m = mK;
    for (int i = K - 1; i >= 0; --i) {
      while (cur_m > P.m[i]) {
        cur_m >>= 1;
        const int64_t ne = cur_m * C;
        for (int64_t e0 = tid; e0 < ne; e0 += (int64_t)blockDim.x * 2 * B_RU) {   // loads in flight
          long long hi[2 * B_RU], lo[2 * B_RU];
#pragma unroll
          for (int q = 0; q < 2 * B_RU; ++q) {
            const int64_t e = e0 + (int64_t)q * blockDim.x;
            hi[q] = e < ne ? buckets[e + ne] : 0;
            lo[q] = e < ne ? buckets[e] : 0;
          }
#pragma unroll
          for (int q = 0; q < 2 * B_RU; ++q) {
            const int64_t e = e0 + (int64_t)q * blockDim.x;
            if (e < ne) buckets[e] = lo[q] + hi[q];
          }
        }
        __syncthreads();
      }
      float* S_i = stages + off[i] * ld;
      double* b_i = bst + off[i];
      // a warp per stage row, lanes over its columns (no index division)
      for (int64_t t = warp; t < cur_m; t += nw) {
        const long long* src = buckets + t * C;
        float* dst = S_i + t * ld;
        long long qv[(B_MAXD + 4 + 31) / 32];
#pragma unroll
        for (int u = 0; u < (B_MAXD + 4 + 31) / 32; ++u) {
          const int c = lane + 32 * u;
          qv[u] = c < d ? src[c] : 0;
        }
#pragma unroll
        for (int u = 0; u < (B_MAXD + 4 + 31) / 32; ++u) {
          const int c = lane + 32 * u;
          if (c < ld) dst[c] = c < d ? f32_from_fixed(qv[u], sh.colshift[c]) : 0.f;
        }
        if (lane == 0) b_i[t] = f64_from_fixed(src[d], sh.colshift[d]);
      }
      __syncthreads();
    }
    __syncthreads();
    phase_mark(3);
    // 4. Householder QR of S-hat X (FP32), R with positive diagonal, R^{-1}
    float* vk = reinterpret_cast<float*>(ring);   // x(k : r) of step k (the ring is idle here)
    for (int k = 0; k < d; ++k) {
      const float* colk = Ahat + (int64_t)k * r;
      for (int64_t i = k + tid; i < r; i += blockDim.x) vk[i] = colk[i];
      __syncthreads();
      double s2 = 0.0;
      for (int64_t i = k + 1 + tid; i < r; i += blockDim.x) s2 += (double)vk[i] * vk[i];
      s2 = bsum(s2, tmp);
      const double x0 = vk[k];
      const double normx = sqrt(x0 * x0 + s2);
      const double alpha = (x0 >= 0.0) ? -normx : normx;
      const double v0 = x0 - alpha;
      const double vv = v0 * v0 + s2;
      if (tid == 0) R[k * d + k] = (float)alpha;
      if (vv > 0.0) {
        const float tau = (float)(2.0 / vv), v0f = (float)v0;
        for (int j = k + 1 + warp; j < d; j += nw) {
          float* cj = Ahat + (int64_t)j * r;
          // eight independent partial sums: eight loads of the column in
          // flight, the reflector from shared memory
          float sp[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) sp[u] = 0.f;
          int64_t i = k + 1 + lane;
          for (; i + 224 < r; i += 256) {
            float cv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) cv[u] = cj[i + 32 * u];
#pragma unroll
            for (int u = 0; u < 8; ++u) sp[u] = fmaf(vk[i + 32 * u], cv[u], sp[u]);
          }
          for (; i < r; i += 32) sp[0] = fmaf(vk[i], cj[i], sp[0]);
          const float sd =
              warp_allsum(((sp[0] + sp[1]) + (sp[2] + sp[3])) + ((sp[4] + sp[5]) + (sp[6] + sp[7]))) +
              v0f * cj[k];
          const float f = tau * sd;
          if (lane == 0) cj[k] -= f * v0f;
          i = k + 1 + lane;
          for (; i + 224 < r; i += 256) {
            float cv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) cv[u] = cj[i + 32 * u];
#pragma unroll
            for (int u = 0; u < 8; ++u) cj[i + 32 * u] = fmaf(-f, vk[i + 32 * u], cv[u]);
          }
          for (; i < r; i += 32) cj[i] = fmaf(-f, vk[i], cj[i]);
        }
      }
      __syncthreads();
    }
    for (int64_t e = tid; e < (int64_t)d * d; e += blockDim.x) {
      const int i = (int)(e / d), j = (int)(e % d);
      const float di = R[i * d + i];
      const float sg = di < 0.f ? -1.f : 1.f;
      if (j > i) R[e] = sg * Ahat[(int64_t)j * r + i];
      else if (j < i) R[e] = 0.f;
    }
    __syncthreads();
    if (tid == 0) sh.flag = 0;
    __syncthreads();
    for (int i = tid; i < d; i += blockDim.x) {
      const float v = fabsf(R[i * d + i]);
      if (!(v > 0.f) || !isfinite(v)) sh.flag = 2;
      R[i * d + i] = v;
    }
    __syncthreads();
    if (sh.flag == 2) status = 4;
    __syncthreads();
    // R^{-1}: one warp per column, back substitution
    if (status == 0) {
      for (int j = warp; j < d; j += nw) {
        for (int i = lane; i < d; i += 32) Rinv[(int64_t)i * d + j] = 0.f;
        __syncwarp();
        if (lane == 0) Rinv[(int64_t)j * d + j] = 1.f / R[j * d + j];
        __syncwarp();
        for (int i = j - 1; i >= 0; --i) {
          float s = 0.f;
          for (int kk = i + 1 + lane; kk <= j; kk += 32) s = fmaf(R[i * d + kk], Rinv[(int64_t)kk * d + j], s);
          s = warp_allsum(s);
          if (lane == 0) Rinv[(int64_t)i * d + j] = -s / R[i * d + i];
          __syncwarp();
        }
      }
      __syncthreads();
      for (int64_t e = tid; e < (int64_t)d * d; e += blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);
        RinvT[e] = Rinv[(int64_t)j * d + i];
      }
      __syncthreads();
    }
    phase_mark(4);
    double* beta = sh.dvec[0];
    double* g = sh.dvec[1];
    double* z = sh.dvec[2];
    double* pv = sh.dvec[3];
    double* wv = sh.dvec[4];
    double* u = sh.dvec[5];
    for (int c = tid; c < d; c += blockDim.x) beta[c] = 0.0;
    __syncthreads();
    // one PCG run of `iters` iterations on (A, b); check: stopping rule
    // (returns 1 when the recursive test holds), 0 otherwise, -1 on error
    auto start = [&](const float* A, int64_t m, int64_t lda, int mode, const double* b64,
                     const float* b32) -> bool {
      for (int c = tid; c < B_MAXD; c += blockDim.x) {   // zero beyond d: 0 * x stays 0
        const float hi = c < d ? (float)beta[c] : 0.f;
        sh.bh[c] = hi;
        sh.bl[c] = c < d ? (float)(beta[c] - (double)hi) : 0.f;
      }
      __syncthreads();
      if (!stream_pass(sh, ring, ring_bytes, A, m, lda, d, P.tile_rows, mode, b64, b32, g, a.spin))
        return false;
      precond(Rinv, RinvT, d, g, u, z);
      for (int c = tid; c < d; c += blockDim.x) pv[c] = z[c];
      __syncthreads();
      return true;
    };
    auto gamma_rb = [&](double& gam, double& rb) {
      double x = 0.0, y = 0.0;
      for (int i = tid; i < d; i += blockDim.x) {
        x += g[i] * z[i];
        double q = 0.0;
        for (int j = i; j < d; ++j) q += (double)R[i * d + j] * beta[j];
        y += q * q;
      }
      gam = bsum(x, tmp);
      rb = sqrt(bsum(y, tmp));
    };
    auto iterate = [&](const float* A, int64_t m, int64_t lda, double& gam) -> bool {
      for (int c = tid; c < B_MAXD; c += blockDim.x) sh.pf[c] = c < d ? (float)pv[c] : 0.f;
      __syncthreads();
      if (!stream_pass(sh, ring, ring_bytes, A, m, lda, d, P.tile_rows, 0, nullptr, nullptr, wv,
                       a.spin))
        return false;
      double pw = 0.0;
      for (int i = tid; i < d; i += blockDim.x) pw += pv[i] * wv[i];
      pw = bsum(pw, tmp);
      const double alpha = gam / pw;
      if (!(pw > 0.0) || !isfinite(alpha)) return false;
      for (int i = tid; i < d; i += blockDim.x) {
        beta[i] += alpha * pv[i];
        g[i] -= alpha * wv[i];
      }
      __syncthreads();
      precond(Rinv, RinvT, d, g, u, z);
      double gz = 0.0;
      for (int i = tid; i < d; i += blockDim.x) gz += g[i] * z[i];
      const double gam2 = bsum(gz, tmp);
      const double ratio = gam2 / gam;
      for (int i = tid; i < d; i += blockDim.x) pv[i] = z[i] + ratio * pv[i];
      __syncthreads();
      gam = gam2;
      return true;
    };
    // 5. Stage I
    for (int i = 0; i < K && status == 0; ++i) {
      const float* S_i = stages + off[i] * ld;
      if (!start(S_i, P.m[i], ld, 1, bst + off[i], nullptr)) {
        status = 6;
        break;
      }
      double gam, rb;
      gamma_rb(gam, rb);
      for (int it = 0; it < P.a[i] && gam > 0.0; ++it)
        if (!iterate(S_i, P.m[i], ld, gam)) {
          status = 4;
          break;
        }
    }
    phase_mark(5);
    // 6. Stage II with the stopping rule confirmed on true gradients
    int total = 0, restarts = 0, converged = 0;
    const double tau = a.tol / 2.0;
    while (status == 0) {
      if (!start(P.X, N, ldx, 2, nullptr, P.Y)) {
        status = 6;
        break;
      }
      double gam, rb;
      gamma_rb(gam, rb);
      if (gam == 0.0 || sqrt(fmax(gam, 0.0)) <= tau * rb) {
        converged = 1;
        break;
      }
      if (total >= a.max_iters || restarts > a.max_restarts) break;
      bool hit = false;
      while (total < a.max_iters) {
        if (!iterate(P.X, N, ldx, gam)) {
          status = 4;
          break;
        }
        ++total;
        gamma_rb(gam, rb);
        if (gam == 0.0 || sqrt(fmax(gam, 0.0)) <= tau * rb) {
          hit = true;
          break;
        }
      }
      if (!hit) break;
      ++restarts;
    }
    if (status == 0 && !converged) status = 5;
    phase_mark(6);
    for (int c = tid; c < d; c += blockDim.x) P.beta[c] = beta[c];
    if (tid == 0) {
      *P.status = status;
      *P.iters = total;
    }
    __syncthreads();
  }
}

}  // namespace spcg

// ---------------------------------------------------------------------------
// Host side: batch context, autotuner, CUDA graph.
// ---------------------------------------------------------------------------
#include <algorithm>
#include <vector>

struct spcg_batch {
  cudaStream_t stream = nullptr;   // the caller's stream (ordering only)
  cudaStream_t own = nullptr;      // non-blocking stream the graph is captured and run on
  cudaEvent_t eu = nullptr;
  int n = 0;
  std::vector<spcg::BatchProblemDev> host;   // in solve order (largest first)
  std::vector<int> order;                     // host[k] is problem order[k]
  spcg::BatchProblemDev* dprobs = nullptr;
  int* dstatus = nullptr;
  int* diters = nullptr;
  int* queue = nullptr;
  unsigned char* scratch = nullptr;
  size_t scratch_bytes = 0;
  int grid = 0;
  int64_t max_rows_int = 0, max_stage_rows = 0, max_r = 0, max_n = 0;
  long long* dphase = nullptr;     // n x 8 phase cycles of the last solve
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t g_seed = 0;
  double g_tol = 0.0;
  int g_tiles_version = -1;
  int tiles_version = 0;
  int tile_class[4] = {0, 0, 0, 0};   // chunk bytes per width class (0 = default)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {
int width_class(int d) { return d <= 32 ? 0 : d <= 64 ? 1 : d <= 128 ? 2 : 3; }
int tile_rows_for(int d, int chunk_bytes) {
  const int ld = (d + 3) & ~3;
  int rows = chunk_bytes / (ld * 4);
  if (rows < 1) rows = 1;
  return rows;
}
}  // namespace

using namespace spcg;

static spcg_status batch_upload(spcg_batch* b) {
  for (auto& P : b->host) {
    const int cls = width_class(P.d);
    const int bytes = b->tile_class[cls] > 0 ? b->tile_class[cls] : 16384;
    P.tile_rows = tile_rows_for(P.d, bytes);
  }
  SPCG_CK(cudaMemcpyAsync(b->dprobs, b->host.data(), sizeof(BatchProblemDev) * b->n,
                          cudaMemcpyHostToDevice, b->stream));
  b->tiles_version++;
  return SPCG_OK;
}

extern "C" spcg_status spcg_batch_create(const spcg_problem_f32* probs, int32_t n, void* stream,
                                         spcg_batch** out) {
  if (!out || !probs || n < 1) return SPCG_E_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {   // every problem, before any CUDA call
    const spcg_problem_f32& q = probs[i];
    if (!q.X || !q.Y || !q.beta || q.d < 1 || q.d > 256 || q.N <= q.d || q.N > (1 << 24) ||
        q.ldx < q.d || (q.ldx * 4) % 16 != 0 || ((uintptr_t)q.X & 15u) != 0)
      return SPCG_E_INVALID_ARG;
  }
  spcg_batch* b = new spcg_batch();
  b->stream = (cudaStream_t)stream;
  b->n = n;
  auto fail = [&](spcg_status s) {
    spcg_batch_destroy(b);
    return s;
  };
  // solve order: largest N d first (longest-processing-time first)
  b->order.resize(n);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    return probs[x].N * probs[x].d > probs[y].N * probs[y].d;
  });
  if (cudaMalloc(&b->dstatus, sizeof(int) * n) != cudaSuccess) return fail(SPCG_E_OOM);
  if (cudaMalloc(&b->diters, sizeof(int) * n) != cudaSuccess) return fail(SPCG_E_OOM);
  b->host.resize(n);
  for (int k = 0; k < n; ++k) {
    const spcg_problem_f32& q = probs[b->order[k]];
    BatchProblemDev P{};
    P.X = q.X;
    P.Y = q.Y;
    P.N = q.N;
    P.ldx = q.ldx;
    P.d = q.d;
    spcg_schedule sc;
    if (spcg_default_schedule(q.N, q.d, &sc) != SPCG_OK) return fail(SPCG_E_INVALID_ARG);
    P.K = sc.K;
    for (int i = 0; i < sc.K; ++i) {
      P.m[i] = sc.m[i];
      P.a[i] = sc.a[i];
    }
    P.r = sc.r;
    P.beta = q.beta;
    P.status = b->dstatus + k;
    P.iters = b->diters + k;
    const int64_t mK = sc.K > 0 ? sc.m[sc.K - 1] : 0;
    int64_t sum_m = 0;
    for (int i = 0; i < sc.K; ++i) sum_m += sc.m[i];
    b->max_rows_int = std::max(b->max_rows_int, mK + sc.r);
    b->max_stage_rows = std::max(b->max_stage_rows, sum_m);
    b->max_r = std::max(b->max_r, (int64_t)sc.r);
    b->max_n = std::max(b->max_n, (int64_t)q.N);
    b->host[k] = P;
  }
  b->max_rows_int = (b->max_rows_int + 15) & ~int64_t(15);
  b->max_stage_rows = (b->max_stage_rows + 15) & ~int64_t(15);
  b->max_r = (b->max_r + 15) & ~int64_t(15);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(SPCG_E_CUDA);
  b->grid = std::min(sms, n);
  size_t bytes = (size_t)b->max_rows_int * (B_MAXD + 1) * 8 + (size_t)b->max_stage_rows * B_MAXD * 4 +
                 (size_t)b->max_stage_rows * 8 + (size_t)b->max_r * B_MAXD * 4 +
                 (size_t)3 * B_MAXD * B_MAXD * 4 + (size_t)2 * b->max_rows_int * 4 +
                 (size_t)2 * b->max_n * 4;
  b->scratch_bytes = (bytes + 255) & ~(size_t)255;
  if (cudaMalloc(&b->scratch, b->scratch_bytes * b->grid) != cudaSuccess) return fail(SPCG_E_OOM);
  if (cudaMalloc(&b->dprobs, sizeof(BatchProblemDev) * n) != cudaSuccess) return fail(SPCG_E_OOM);
  if (cudaMalloc(&b->queue, sizeof(int)) != cudaSuccess) return fail(SPCG_E_OOM);
  if (cudaMalloc(&b->dphase, sizeof(long long) * 8 * n) != cudaSuccess) return fail(SPCG_E_OOM);
  if (cudaMemset(b->dphase, 0, sizeof(long long) * 8 * n) != cudaSuccess) return fail(SPCG_E_CUDA);
  if (cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->eu, cudaEventDisableTiming) != cudaSuccess)
    return fail(SPCG_E_CUDA);
  // a capture needs a stream with no implicit ordering against the legacy stream
  if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess)
    return fail(SPCG_E_CUDA);
  if (cudaFuncSetAttribute(k_batched_spcg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)B_SMEM) != cudaSuccess)
    return fail(SPCG_E_CUDA);
  spcg_status st = batch_upload(b);
  if (st != SPCG_OK) return fail(st);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(SPCG_E_CUDA);
  *out = b;
  return SPCG_OK;
}

extern "C" void spcg_batch_destroy(spcg_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->own) cudaStreamSynchronize(b->own);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->eu) cudaEventDestroy(b->eu);
  if (b->own) cudaStreamDestroy(b->own);
  cudaFree(b->dprobs);
  cudaFree(b->dstatus);
  cudaFree(b->diters);
  cudaFree(b->queue);
  cudaFree(b->dphase);
  cudaFree(b->scratch);
  delete b;
}

// Capture (memset of the queue, the persistent kernel) as a CUDA graph.
static spcg_status batch_capture(spcg_batch* b, uint64_t seed, double tol) {
  if (b->exec && b->g_seed == seed && b->g_tol == tol && b->g_tiles_version == b->tiles_version)
    return SPCG_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  BatchArgs a{};
  a.probs = b->dprobs;
  a.n = b->n;
  a.queue = b->queue;
  a.scratch = b->scratch;
  a.scratch_bytes = b->scratch_bytes;
  a.max_rows_int = b->max_rows_int;
  a.max_stage_rows = b->max_stage_rows;
  a.max_r = b->max_r;
  a.max_n = b->max_n;
  a.phase_cycles = b->dphase;
  a.seed = seed;
  a.tol = tol;
  a.max_iters = 100;
  a.max_restarts = 5;
  a.spin = 1ll << 31;
  SPCG_CK(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(b->queue, 0, sizeof(int), b->own);
  k_batched_spcg<<<b->grid, BT, B_SMEM, b->own>>>(a);
  cudaError_t le = cudaGetLastError();
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->own, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return from_cuda(le != cudaSuccess ? le : ce);
  }
  b->graph = g;
  SPCG_CK(cudaGraphInstantiate(&b->exec, g, 0));
  b->g_seed = seed;
  b->g_tol = tol;
  b->g_tiles_version = b->tiles_version;
  return SPCG_OK;
}

extern "C" spcg_status spcg_batch_solve(spcg_batch* b, uint64_t seed, double tol,
                                        int32_t* status_out, int32_t* iters_out, double* ms_out) {
  if (!b || !(tol > 0.0)) return SPCG_E_INVALID_ARG;
  SPCG_TRY(batch_capture(b, seed, tol));
  SPCG_CK(cudaEventRecord(b->eu, b->stream));      // after the caller's prior work
  SPCG_CK(cudaStreamWaitEvent(b->own, b->eu, 0));
  SPCG_CK(cudaEventRecord(b->e0, b->own));
  SPCG_CK(cudaGraphLaunch(b->exec, b->own));
  SPCG_CK(cudaEventRecord(b->e1, b->own));
  SPCG_CK(cudaStreamSynchronize(b->own));
  if (ms_out) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->e0, b->e1);
    *ms_out = ms;
  }
  std::vector<int> st(b->n), it(b->n);
  SPCG_CK(cudaMemcpy(st.data(), b->dstatus, sizeof(int) * b->n, cudaMemcpyDeviceToHost));
  SPCG_CK(cudaMemcpy(it.data(), b->diters, sizeof(int) * b->n, cudaMemcpyDeviceToHost));
  spcg_status worst = SPCG_OK;
  for (int k = 0; k < b->n; ++k) {
    const int i = b->order[k];
    if (status_out) status_out[i] = st[k];
    if (iters_out) iters_out[i] = it[k];
    if (st[k] != 0 && worst == SPCG_OK) worst = (spcg_status)st[k];
  }
  return worst;
}

extern "C" spcg_status spcg_solve_batched(const spcg_problem_f32* probs, int32_t n, uint64_t seed,
                                          double tol, void* stream, int32_t* status_out,
                                          int32_t* iters_out) {
  spcg_batch* b = nullptr;
  SPCG_TRY(spcg_batch_create(probs, n, stream, &b));
  const spcg_status st = spcg_batch_solve(b, seed, tol, status_out, iters_out, nullptr);
  spcg_batch_destroy(b);
  return st;
}

extern "C" spcg_status spcg_batch_phase_cycles(spcg_batch* b, int64_t* cycles_out) {
  if (!b || !cycles_out) return SPCG_E_INVALID_ARG;
  std::vector<long long> h((size_t)8 * b->n);
  SPCG_CK(cudaMemcpy(h.data(), b->dphase, sizeof(long long) * 8 * b->n, cudaMemcpyDeviceToHost));
  for (int k = 0; k < b->n; ++k)
    for (int q = 0; q < 8; ++q) cycles_out[(size_t)b->order[k] * 8 + q] = h[(size_t)k * 8 + q];
  return SPCG_OK;
}

extern "C" spcg_status spcg_batch_set_tiles(spcg_batch* b, const int32_t* chunk_bytes4) {
  if (!b || !chunk_bytes4) return SPCG_E_INVALID_ARG;
  for (int i = 0; i < 4; ++i) {
    const int v = chunk_bytes4[i];
    if (v != 0 && (v < 1024 || v > 16384 || (v & 15))) return SPCG_E_INVALID_ARG;
    b->tile_class[i] = v;
  }
  SPCG_TRY(batch_upload(b));
  SPCG_CK(cudaStreamSynchronize(b->stream));
  return SPCG_OK;
}

// The autotuner: for every width class present, time the batch with each
// candidate chunk size (the other classes at their current choice) and keep
// the fastest.  Candidate chunks: 4, 8 and 16 KB of rows.
extern "C" spcg_status spcg_batch_autotune(spcg_batch* b, uint64_t seed, double tol,
                                           int32_t* chosen4) {
  if (!b) return SPCG_E_INVALID_ARG;
  const int cands[3] = {4096, 8192, 16384};
  bool present[4] = {false, false, false, false};
  for (auto& P : b->host) present[width_class(P.d)] = true;
  for (int cls = 0; cls < 4; ++cls) {
    if (!present[cls]) continue;
    double best = 1e300;
    int pick = 16384;
    for (int c : cands) {
      b->tile_class[cls] = c;
      SPCG_TRY(batch_upload(b));
      double ms = 0.0;
      spcg_batch_solve(b, seed, tol, nullptr, nullptr, &ms);   // warm
      spcg_batch_solve(b, seed, tol, nullptr, nullptr, &ms);
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    b->tile_class[cls] = pick;
  }
  SPCG_TRY(batch_upload(b));
  SPCG_CK(cudaStreamSynchronize(b->stream));
  if (chosen4)
    for (int i = 0; i < 4; ++i) chosen4[i] = b->tile_class[i];
  return SPCG_OK;
}
