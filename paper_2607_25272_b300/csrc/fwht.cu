// The nested SRHT transform (Sec. 2.2): Z = H D P [X Y; 0] over N' = 2^n
// padded rows, H the Sylvester Walsh-Hadamard matrix.
//
// Arithmetic.  H has entries +-1, so the transform is additions only.  Each
// column c is converted once to 64-bit fixed point, q = round(x 2^{s_c}),
// with s_c chosen from the column's largest magnitude so that no partial
// sum of N' terms can reach 2^62; every butterfly is then an exact integer
// add, and the only rounding is the conversion in and out (error at most
// half a quantum 2^{-s_c} per input element, and one rounding to FP64 per
// output).  This keeps the B300's slow FP64 pipe out of the transform.
//
// Passes.  H_{N'} factors over groups of index bits: a pass that owns bits
// [s, s + b) runs the 2^b-point transform on every set of rows that differ
// only in those bits.  Each CTA stages one such set (2^b rows, 2^s apart)
// for a slab of TC adjacent columns.  Inside the tile, threads take 2^g
// values of one column into registers and run g butterfly levels there
// (g <= 4), so a 10-level tile needs three register rounds and four passes
// over shared memory.  The first pass fuses the signed row gather (D P) and
// the conversion to fixed point; the last pass converts back and scatters
// the rows of I_K (to their position in pi order) and of I-hat (scaled by
// 1/sqrt(r), column-major for the QR).  Y is column d.
//
// Scale.  The stage rows are stored as H' D P X' with the unnormalised +-1
// matrix H' (PCG iterates do not change under a joint scaling of A and b);
// S-hat X = sqrt(N'/r) H D P X' [I-hat] = H' D P X' [I-hat] / sqrt(r).
#include <cuda_bf16.h>

#include <atomic>

#include "common.cuh"
#include "internal.hpp"

namespace spcg {

// ---- exact conversions between FP64 and 64-bit fixed point ----
// q = x 2^s rounded half away from zero (subnormal inputs count as zero).
__device__ __forceinline__ long long to_fixed(double x, int s) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;
  const unsigned long long mant = (unsigned long long)(b & 0xFFFFFFFFFFFFFll) | (1ull << 52);
  const int sh = e - 1075 + s;   // x 2^s = mant 2^sh
  unsigned long long q;
  if (sh >= 0) q = mant << sh;   // the scale bound keeps this below 2^62
  else if (sh > -64) q = (mant + (1ull << (-sh - 1))) >> (-sh);
  else q = 0;
  return (b < 0) ? -(long long)q : (long long)q;
}

// q 2^{-s} rounded to nearest even (results below the normal range flush to 0).
__device__ __forceinline__ double from_fixed(long long q, int s) {
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
  const unsigned long long bits =
      (sign << 63) | ((unsigned long long)biased << 52) | (m & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// Per-column largest magnitude (as IEEE bit patterns: for non-negative
// doubles the integer order is the numeric order, so atomicMax is exact).
__global__ void __launch_bounds__(256) k_colmax(const double* __restrict__ X, int64_t ldx,
                                                const double* __restrict__ Y, int64_t N, int d,
                                                unsigned long long* __restrict__ colmax) {
  const int C = d + 1;
  const int64_t G = gridDim.x;
  for (int c0 = 0; c0 < C; c0 += blockDim.x) {
    const int c = c0 + threadIdx.x;
    unsigned long long mx = 0;
    if (c < C) {
      // four rows in flight per thread
      for (int64_t i = blockIdx.x; i < N; i += 4 * G) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t row = i + u * G;
          v[u] = (row < N) ? ((c < d) ? X[row * ldx + c] : Y[row]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned long long b =
              (unsigned long long)__double_as_longlong(v[u]) & 0x7FFFFFFFFFFFFFFFull;
          mx = b > mx ? b : mx;
        }
      }
      atomicMax(colmax + c, mx);
    }
  }
}

// s_c = 61 - n - E_c with 2^{E_c} <= max_c < 2^{E_c+1}: every partial sum of
// N' <= 2^n terms stays below 2^62 in magnitude.  A column holding an Inf or
// a NaN (the largest bit pattern then has the all-ones exponent) has no such
// scale: the device status becomes BREAKDOWN and the column gets shift 0, so
// the transform still only moves values (no shift or index depends on them).
__global__ void k_colscale(const unsigned long long* __restrict__ colmax, int C, int nbits,
                           int* __restrict__ shift, int* __restrict__ status) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    const unsigned long long b = colmax[c];
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) atomicExch(status, DEV_BREAKDOWN);
    shift[c] = (e == 0 || e == 0x7FF) ? 0 : 61 - nbits - (e - 1023);
  }
}

struct FwhtArgs {
  const double* X;
  int64_t ldx;
  const double* Y;
  int64_t N;
  const uint32_t* gather;
  const int* shift;      // per-column fixed-point scale exponent
  long long* W;          // work buffer N' x ldw (multi-pass only)
  int64_t ldw;
  int C;                 // d + 1 columns (Y last)
  int d;
  int shift_lo;          // low index bit of this pass
  int first, last;
  int ncoltiles;
  const int32_t* dest;
  const int32_t* hdest;
  double* AK;            // FP64 prefix (or null)
  int64_t ldak;
  __nv_bfloat16* AK16;   // BF16 prefix (or null)
  int64_t ldak16;
  double* bK;
  double* Ahat;          // column-major, ld = r
  int64_t r;
  double hat_scale;      // 1/sqrt(r)
};

template <int LOGL>
struct FwhtShape {
  static constexpr int L = 1 << LOGL;
  static constexpr int TC = (L <= 1024) ? 16 : (L == 2048 ? 8 : 4);
  static constexpr int THREADS = 512;
  static constexpr int ROUNDS = (LOGL + 3) / 4;
  static constexpr size_t SMEM = (size_t)L * TC * 8 + (size_t)L * 3 * 4;
};

// g-level butterfly on 2^g registers (index bits 0..g-1 of the register index).
template <int G>
__device__ __forceinline__ void bfly(long long (&v)[1 << G]) {
#pragma unroll
  for (int b = 0; b < G; ++b) {
#pragma unroll
    for (int k = 0; k < (1 << G); ++k) {
      if (k & (1 << b)) continue;
      const long long x = v[k], y = v[k | (1 << b)];
      v[k] = x + y;
      v[k | (1 << b)] = x - y;
    }
  }
}

// Register rounds of a LOGL-level pass: R rounds of g(rnd) levels (g <= 4),
// round rnd starting at tile-row bit lev(rnd).  All compile-time, so every
// shared-memory offset of a round is an immediate.
template <int LOGL>
struct FwhtRounds {
  static constexpr int R = FwhtShape<LOGL>::ROUNDS;
  static constexpr int g(int rnd) { return LOGL / R + (rnd < LOGL % R ? 1 : 0); }
  static constexpr int lev(int rnd) {
    int l = 0;
    for (int i = 0; i < rnd; ++i) l += g(i);
    return l;
  }
};

// What one thread of k_fwht_pass needs for its column (threads keep one tile
// column c = tid mod TC for the whole pass).  Global rows of the tile,
// low | t << shift_lo | high << (shift_lo + LOGL), are low + high 2^(shift_lo + LOGL)
// plus t 2^shift_lo (the bit fields do not overlap), so a work-buffer element
// of tile row t sits at wb + t * wst.
struct PassCol {
  long long* tc;          // this column of the shared-memory tile
  bool ok;                // column < C
  bool isx;               // column < d (a column of X, not Y)
  int s;                  // fixed-point scale exponent of the column
  uint32_t nrows;         // N (rows of X and Y; at most 2^30)
  const char* src;        // first pass: the column's first element
  uint64_t sstride;       // first pass: bytes between rows of that column
  long long* wb;          // work buffer, tile row 0 of this column
  int64_t wst;            // elements between tile rows in the work buffer
  double* ak;             // last pass: column of A_K (FP64), or null
  __nv_bfloat16* ak16;    // last pass: column of A_K (BF16), or null
  double* ahat;           // last pass: column of S-hat X
};

template <int LOGL, int RND>
__device__ __forceinline__ void pass_round(const FwhtArgs& a, const PassCol& pc,
                                           const int32_t* gmap, const int32_t* dmap,
                                           const int32_t* hmap) {
  using S = FwhtShape<LOGL>;
  using RS = FwhtRounds<LOGL>;
  constexpr int L = S::L, TC = S::TC, NT = S::THREADS;
  constexpr int G = RS::g(RND), LEV = RS::lev(RND), H = 1 << LEV, GN = 1 << G;
  constexpr bool FROM = (RND == 0), TO = (RND == RS::R - 1);
  constexpr int NG = L / GN, GS = NT / TC;
  const int64_t hst = (int64_t)H * pc.wst;
  for (int gi = threadIdx.x / TC; gi < NG; gi += GS) {
    const int t0 = (gi & (H - 1)) | ((gi >> LEV) << (LEV + G));
    long long v[GN];
    if constexpr (FROM) {
      if (a.first) {
        // All GN loads are issued before any is used: rows past N read row 0
        // and are zeroed afterwards, so no load waits behind a branch.  The
        // sign of D is applied to the FP64 sign bit before the conversion
        // (which rounds the magnitude), the same as negating its result.
        uint32_t gm[GN];
        double raw[GN];
#pragma unroll
        for (int k = 0; k < GN; ++k) {
          gm[k] = (uint32_t)gmap[t0 + k * H];
          const uint32_t src = gm[k] & 0x7FFFFFFFu;
          const uint32_t srcc = src < pc.nrows ? src : 0u;
          raw[k] = __ldg(reinterpret_cast<const double*>(pc.src + (uint64_t)srcc * pc.sstride));
        }
#pragma unroll
        for (int k = 0; k < GN; ++k) {
          const bool live = pc.ok && (gm[k] & 0x7FFFFFFFu) < pc.nrows;
          unsigned long long b = (unsigned long long)__double_as_longlong(raw[k]) ^
                                 ((unsigned long long)(gm[k] & 0x80000000u) << 32);
          b = live ? b : 0ull;
          v[k] = to_fixed(__longlong_as_double((long long)b), pc.s);
        }
      } else {
        const long long* p = pc.wb + (int64_t)t0 * pc.wst;
#pragma unroll
        for (int k = 0; k < GN; ++k) v[k] = p[k * hst];
        if (!pc.ok)
#pragma unroll
          for (int k = 0; k < GN; ++k) v[k] = 0;
      }
    } else {
#pragma unroll
      for (int k = 0; k < GN; ++k) v[k] = pc.tc[(t0 + k * H) * TC];
    }
    bfly<G>(v);
    if constexpr (!TO) {
#pragma unroll
      for (int k = 0; k < GN; ++k) pc.tc[(t0 + k * H) * TC] = v[k];
    } else if (pc.ok) {
      if (!a.last) {
        long long* p = pc.wb + (int64_t)t0 * pc.wst;
#pragma unroll
        for (int k = 0; k < GN; ++k) p[k * hst] = v[k];
      } else {
#pragma unroll
        for (int k = 0; k < GN; ++k) {
          const int t = t0 + k * H;
          const int32_t dst = dmap[t], hd = hmap[t];
          if (dst >= 0 || hd >= 0) {
            const double z = from_fixed(v[k], pc.s);
            if (dst >= 0) {
              if (pc.isx) {
                if (pc.ak) pc.ak[(int64_t)dst * a.ldak] = z;
                if (pc.ak16) pc.ak16[(int64_t)dst * a.ldak16] = __double2bfloat16(z);
              } else {
                a.bK[dst] = z;
              }
            }
            if (hd >= 0 && pc.isx) pc.ahat[hd] = z * a.hat_scale;
          }
        }
      }
    }
  }
}

template <int LOGL, int RND>
__device__ __forceinline__ void pass_rounds(const FwhtArgs& a, const PassCol& pc,
                                            const int32_t* gmap, const int32_t* dmap,
                                            const int32_t* hmap) {
  if constexpr (RND < FwhtRounds<LOGL>::R) {
    pass_round<LOGL, RND>(a, pc, gmap, dmap, hmap);
    if constexpr (RND + 1 < FwhtRounds<LOGL>::R) {
      __syncthreads();
      pass_rounds<LOGL, RND + 1>(a, pc, gmap, dmap, hmap);
    }
  }
}

template <int LOGL>
__global__ void __launch_bounds__(512) k_fwht_pass(const FwhtArgs a) {
  using S = FwhtShape<LOGL>;
  constexpr int L = S::L, TC = S::TC, NT = S::THREADS;
  static_assert(NT % TC == 0, "a thread keeps one column");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* tile = reinterpret_cast<long long*>(smem_raw);
  int32_t* gmap = reinterpret_cast<int32_t*>(tile + (size_t)L * TC);
  int32_t* dmap = gmap + L;
  int32_t* hmap = dmap + L;

  const int64_t blk = blockIdx.x;
  const int ct = (int)(blk % a.ncoltiles);
  const int64_t base = blk / a.ncoltiles;
  const int c0 = ct * TC;
  const int64_t low = base & ((int64_t(1) << a.shift_lo) - 1);
  const int64_t high = base >> a.shift_lo;
  const int tid = threadIdx.x;
  if (a.first)
    for (int t = tid; t < L; t += NT)
      gmap[t] = (int32_t)a.gather[low | ((int64_t)t << a.shift_lo) | (high << (a.shift_lo + LOGL))];
  if (a.last)   // the maps are stored in the last pass's row order
    for (int t = tid; t < L; t += NT) {
      dmap[t] = a.dest[base * L + t];
      hmap[t] = a.hdest[base * L + t];
    }

  PassCol pc;
  const int c = tid % TC;
  const int col = c0 + c;
  pc.tc = tile + c;
  pc.ok = col < a.C;
  const int colc = pc.ok ? col : 0;   // a valid column for the masked loads
  pc.isx = colc < a.d;
  pc.s = a.shift[colc];
  pc.nrows = (uint32_t)a.N;
  pc.src = pc.isx ? reinterpret_cast<const char*>(a.X + colc) : reinterpret_cast<const char*>(a.Y);
  pc.sstride = pc.isx ? (uint64_t)a.ldx * sizeof(double) : sizeof(double);
  pc.wst = a.ldw << a.shift_lo;
  pc.wb = a.W ? a.W + (low + (high << (a.shift_lo + LOGL))) * a.ldw + colc : nullptr;
  pc.ak = a.AK ? a.AK + colc : nullptr;
  pc.ak16 = a.AK16 ? a.AK16 + colc : nullptr;
  pc.ahat = a.Ahat ? a.Ahat + (int64_t)colc * a.r : nullptr;
  __syncthreads();
  pass_rounds<LOGL, 0>(a, pc, gmap, dmap, hmap);
}

// ---------------------------------------------------------------------------
// Tiled pass for 9..12 levels (the passes of every N' >= 2^18).  A CTA holds
// one 128 KB tile: L = 2^LOGL rows (2^shift_lo apart) x TC adjacent columns.
// Every thread keeps one column c for the whole pass, so the column's
// fixed-point shift stays in a register, and owns VPT = L TC / NT values per
// round (32 or 64 registers of int64).  Two register rounds cover the pass:
// round 0 runs levels [0, G0) on 2^G0 consecutive tile rows, round 1 levels
// [G0, LOGL) on rows 2^G0 apart, with one trip through shared memory between
// them.  Tile rows are padded every 2^G0 rows so that the 64-bit accesses of a
// half-warp fall in distinct banks in both rounds.
// ---------------------------------------------------------------------------
// Tile variants: V = 1, 128 KB tiles and 64 values a thread (one CTA per
// SM); V = 2, 64 KB tiles and 32 values a thread (two CTAs per SM, so one
// CTA's loads overlap the other's butterflies; 9 and 10 levels only).
template <int LOGL, int V> struct TileCfg;
template <> struct TileCfg<9, 1> { static constexpr int TC = 32, NT = 256, G0 = 6, MINB = 1; };
template <> struct TileCfg<10, 1> { static constexpr int TC = 16, NT = 256, G0 = 6, MINB = 1; };
template <> struct TileCfg<11, 1> { static constexpr int TC = 8, NT = 256, G0 = 6, MINB = 1; };
template <> struct TileCfg<12, 1> { static constexpr int TC = 4, NT = 256, G0 = 6, MINB = 1; };
template <> struct TileCfg<9, 2> { static constexpr int TC = 16, NT = 256, G0 = 5, MINB = 2; };
template <> struct TileCfg<10, 2> { static constexpr int TC = 8, NT = 256, G0 = 5, MINB = 2; };

template <int LOGL, int V>
struct TileShape {
  using C = TileCfg<LOGL, V>;
  static constexpr int MINB = C::MINB;
  static constexpr int L = 1 << LOGL, TC = C::TC, NT = C::NT, G0 = C::G0, G1 = LOGL - G0;
  static constexpr int TPC = NT / TC;                   // threads per column
  static constexpr int VPT = L * TC / NT;               // values per thread and round
  static constexpr int NG1 = (1 << G0) / TPC;           // round-1 groups per thread
  static constexpr int PAD = TC < 16 ? 16 - TC : 0;     // words per 2^G0 tile rows
  static constexpr size_t WORDS = (size_t)L * TC + (size_t)(L >> G0) * PAD;
  static constexpr size_t SMEM = WORDS * 8 + (size_t)L * 3 * 4;
  static_assert(VPT == (1 << G0), "round 0 is one group per thread");
  static_assert(NG1 * (1 << G1) == VPT, "round 1 covers the thread's values");
  static_assert(G1 >= 1 && G1 <= G0, "levels per round");
};

template <int LOGL, int V>
__device__ __forceinline__ int tile_word(int t, int c) {
  using S = TileShape<LOGL, V>;
  return t * S::TC + c + (t >> S::G0) * S::PAD;
}

template <int LOGL, int V>
__global__ void __launch_bounds__(TileShape<LOGL, V>::NT, TileShape<LOGL, V>::MINB)
    k_fwht_tile(const FwhtArgs a) {
  using S = TileShape<LOGL, V>;
  constexpr int L = S::L, TC = S::TC, G0 = S::G0, G1 = S::G1, VPT = S::VPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* tile = reinterpret_cast<long long*>(smem_raw);
  int32_t* gmap = reinterpret_cast<int32_t*>(tile + S::WORDS);
  int32_t* dmap = gmap + L;
  int32_t* hmap = dmap + L;
  const int tid = threadIdx.x;
  const int64_t blk = blockIdx.x;
  const int ct = (int)(blk % a.ncoltiles);
  const int64_t base = blk / a.ncoltiles;
  const int64_t low = base & ((int64_t(1) << a.shift_lo) - 1);
  const int64_t high = base >> a.shift_lo;
  // global row of tile row t: j0 + t * step
  const int64_t j0 = low | (high << (a.shift_lo + LOGL));
  const int64_t step = int64_t(1) << a.shift_lo;
  const int c = tid % TC, r = tid / TC;
  const int col = ct * TC + c;
  const bool colok = col < a.C;
  const int sh = colok ? a.shift[col] : 0;
  if (a.first)
    for (int t = tid; t < L; t += S::NT) gmap[t] = (int32_t)a.gather[j0 + t * step];
  if (a.last)   // the maps are stored in the last pass's row order
    for (int t = tid; t < L; t += S::NT) {
      dmap[t] = a.dest[base * L + t];
      hmap[t] = a.hdest[base * L + t];
    }
  __syncthreads();
  long long v[VPT];
  // ---- round 0: rows t = r 2^G0 + k ----
  {
    const int t0 = r << G0;
    if (a.first) {
      // column pointer and row stride of this thread's column (Y is column d)
      const double* cp = (colok && col < a.d) ? a.X + col : a.Y;
      const int64_t cstride = (colok && col < a.d) ? a.ldx : 1;
      // all loads first (the raw bits held in v; sign and padding-row flags
      // as bit masks), then the conversions
      unsigned long long negm = 0ull, okm = 0ull;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const uint32_t gm = (uint32_t)gmap[t0 + k];
        const int64_t src = (int64_t)(gm & 0x7FFFFFFFu);
        const bool ok = src < a.N;
        negm |= (unsigned long long)(gm >> 31) << k;
        okm |= (unsigned long long)ok << k;
        v[k] = __double_as_longlong(__ldg(cp + (ok ? src : 0) * cstride));
      }
      if (!colok) okm = 0ull;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const long long x = ((okm >> k) & 1ull) ? to_fixed(__longlong_as_double(v[k]), sh) : 0;
        v[k] = ((negm >> k) & 1ull) ? -x : x;
      }
    } else {
      const long long* wp = reinterpret_cast<const long long*>(a.W) + (colok ? col : 0);
#pragma unroll
      for (int k = 0; k < VPT; ++k) v[k] = wp[(j0 + (int64_t)(t0 + k) * step) * a.ldw];
      if (!colok)
#pragma unroll
        for (int k = 0; k < VPT; ++k) v[k] = 0;
    }
    bfly<G0>(v);
#pragma unroll
    for (int k = 0; k < VPT; ++k) tile[tile_word<LOGL, V>(t0 + k, c)] = v[k];
  }
  __syncthreads();
  // ---- round 1: NG1 groups, rows t = gi + k 2^G0 with gi < 2^G0 ----
#pragma unroll
  for (int m = 0; m < S::NG1; ++m) {
    const int gi = r + m * S::TPC;
    long long u[1 << G1];
#pragma unroll
    for (int k = 0; k < (1 << G1); ++k) u[k] = tile[tile_word<LOGL, V>(gi + (k << G0), c)];
    bfly<G1>(u);
#pragma unroll
    for (int k = 0; k < (1 << G1); ++k) {
      const int t = gi + (k << G0);
      if (!colok) continue;
      if (!a.last) {
        reinterpret_cast<long long*>(a.W)[(j0 + (int64_t)t * step) * a.ldw + col] = u[k];
      } else {
        const int32_t dst = dmap[t], hd = hmap[t];
        if (dst >= 0 || hd >= 0) {
          const double z = from_fixed(u[k], sh);
          if (dst >= 0) {
            if (col < a.d) {
              if (a.AK) a.AK[(int64_t)dst * a.ldak + col] = z;
              if (a.AK16) a.AK16[(int64_t)dst * a.ldak16 + col] = __double2bfloat16(z);
            } else {
              a.bK[dst] = z;
            }
          }
          if (hd >= 0 && col < a.d) a.Ahat[(int64_t)col * a.r + hd] = z * a.hat_scale;
        }
      }
    }
  }
}

template <int LOGL, int V>
static spcg_status launch_tile(const FwhtArgs& a, int64_t nbases, cudaStream_t st) {
  using S = TileShape<LOGL, V>;
  FwhtArgs b = a;
  b.ncoltiles = (a.C + S::TC - 1) / S::TC;
  SPCG_CK(cudaFuncSetAttribute(k_fwht_tile<LOGL, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)S::SMEM));
  k_fwht_tile<LOGL, V><<<(unsigned)(nbases * b.ncoltiles), S::NT, S::SMEM, st>>>(b);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

template <int LOGL>
static spcg_status launch_one(const FwhtArgs& a, int64_t nbases, cudaStream_t st) {
  using S = FwhtShape<LOGL>;
  FwhtArgs b = a;
  b.ncoltiles = (a.C + S::TC - 1) / S::TC;
  SPCG_CK(cudaFuncSetAttribute(k_fwht_pass<LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)S::SMEM));
  const int64_t nblk = nbases * b.ncoltiles;
  k_fwht_pass<LOGL><<<(unsigned)nblk, S::THREADS, S::SMEM, st>>>(b);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

// variant: 0 = the per-round kernel k_fwht_pass for every pass, 1 or 2 = the
// tiled kernel (TileCfg variant) for passes of 9..12 levels.
static spcg_status launch_logl(int logl, const FwhtArgs& a, int64_t nbases, cudaStream_t st,
                               int variant) {
  if (variant == 2) {
    if (logl == 9) return launch_tile<9, 2>(a, nbases, st);
    if (logl == 10) return launch_tile<10, 2>(a, nbases, st);
  }
  if (variant == 1 || variant == 2) {
    switch (logl) {
      case 9: return launch_tile<9, 1>(a, nbases, st);
      case 10: return launch_tile<10, 1>(a, nbases, st);
      case 11: return launch_tile<11, 1>(a, nbases, st);
      case 12: return launch_tile<12, 1>(a, nbases, st);
    }
  }
  switch (logl) {
    case 1: return launch_one<1>(a, nbases, st);
    case 2: return launch_one<2>(a, nbases, st);
    case 3: return launch_one<3>(a, nbases, st);
    case 4: return launch_one<4>(a, nbases, st);
    case 5: return launch_one<5>(a, nbases, st);
    case 6: return launch_one<6>(a, nbases, st);
    case 7: return launch_one<7>(a, nbases, st);
    case 8: return launch_one<8>(a, nbases, st);
    case 9: return launch_one<9>(a, nbases, st);
    case 10: return launch_one<10>(a, nbases, st);
    case 11: return launch_one<11>(a, nbases, st);
    case 12: return launch_one<12>(a, nbases, st);
    default: return SPCG_E_INVALID_ARG;
  }
}

// Split n index bits into passes of at most 12 bits, as even as possible,
// the larger passes first, except that a two-pass plan gives its last pass
// (the scatter to the nested positions) 9 levels when the first then has at
// most 11: a 9-level tile takes 70 KB, so two CTAs share an SM and one's
// loads overlap the other's butterflies (at n = 20, 11 + 9 levels measured
// faster than 10 + 10).  first_levels (> 0) fixes the first pass of a
// two-pass plan instead.
int fwht_pass_plan(int n, int* logl, int first_levels) {
  const int passes = (n + 11) / 12;
  for (int p = 0; p < passes; ++p) logl[p] = n / passes + (p < n % passes ? 1 : 0);
  if (passes == 2 && logl[1] > 9 && n - 9 <= 11) {
    logl[0] = n - 9;
    logl[1] = 9;
  }
  if (passes == 2 && first_levels > 0 && first_levels <= 12 && n - first_levels >= 1 &&
      n - first_levels <= 12) {
    logl[0] = first_levels;
    logl[1] = n - first_levels;
  }
  return passes;
}

// Per-column fixed-point scales: sums of up to 2^nbits terms stay below 2^62.
spcg_status launch_colscales(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int C = c->d + 1;
  if (!s.colmax_pre) {
    SPCG_CK(cudaMemsetAsync(s.colmax, 0, (size_t)C * sizeof(unsigned long long), c->stream));
    int cg = (int)((c->N + 63) / 64);
    if (cg > 8 * c->num_sms) cg = 8 * c->num_sms;
    if (cg < 1) cg = 1;
    k_colmax<<<cg, 256, 0, c->stream>>>(c->X, c->ldx, c->Y, c->N, c->d, s.colmax);
    SPCG_CK(cudaGetLastError());
    c->n_launch += 1;
  }
  s.colmax_pre = false;
  k_colscale<<<(C + 255) / 256, 256, 0, c->stream>>>(s.colmax, C, s.nbits, s.colshift,
                                                 &c->scal->status);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 1;
  return SPCG_OK;
}

spcg_status launch_transform(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int C = c->d + 1;
  SPCG_TRY(launch_colscales(c));
  int logl[8];
  const int passes = fwht_pass_plan(s.nbits, logl, c->opts.fwht_first_levels);
  // default: the per-round kernel for every pass (measured at least as fast as
  // either tile variant at 2^20 x 500 and 2^22 x 1000)
  const int variant = (c->opts.fwht_tile == 0 || c->opts.fwht_tile == 3) ? 0 : c->opts.fwht_tile;
  FwhtArgs a{};
  a.X = c->X;
  a.ldx = c->ldx;
  a.Y = c->Y;
  a.N = c->N;
  a.gather = s.gather;
  a.shift = s.colshift;
  a.W = reinterpret_cast<long long*>(s.work);
  a.ldw = s.ldw;
  a.C = C;
  a.d = c->d;
  a.dest = s.dest;
  a.hdest = s.hdest;
  a.AK = s.mixed ? nullptr : s.AK;
  a.ldak = s.ldak;
  a.AK16 = s.mixed ? reinterpret_cast<__nv_bfloat16*>(s.AK16) : nullptr;
  a.ldak16 = s.ldak16;
  a.bK = s.bK;
  a.Ahat = s.Ahat;
  a.r = s.sched.r;
  a.hat_scale = 1.0 / sqrt((double)s.sched.r);
  int shift = 0;
  for (int p = 0; p < passes; ++p) {
    a.shift_lo = shift;
    a.first = (p == 0);
    a.last = (p == passes - 1);
    const int64_t nbases = s.n_pad >> logl[p];
    SPCG_TRY(launch_logl(logl[p], a, nbases, c->stream, variant));
    c->n_launch += 1;
    shift += logl[p];
  }
  return SPCG_OK;
}

// Rows [row0, row0 + n) of the prefix, scaled to Z = H D P X' (normalised H).
__global__ void k_export_rows(const double* __restrict__ AK, int64_t ldak,
                              const __nv_bfloat16* __restrict__ AK16, int64_t ldak16,
                              const double* __restrict__ bK, int64_t row0, int64_t n, int d,
                              double scale, double* __restrict__ A, double* __restrict__ b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * (d + 1);
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / (d + 1);
    const int j = (int)(e % (d + 1));
    if (j < d) {
      if (A) {
        const double v = AK ? AK[(row0 + i) * ldak + j]
                            : (double)__bfloat162float(AK16[(row0 + i) * ldak16 + j]);
        A[i * d + j] = v * scale;
      }
    } else if (b) {
      b[i] = bK[row0 + i] * scale;
    }
  }
}

spcg_status launch_export_rows(spcg_ctx* c, int64_t row0, int64_t n, double* A, double* b) {
  const Sketch& s = c->sk;
  const bool cs = s.sched.sketch == SPCG_SKETCH_COUNT;
  const double scale = cs ? 1.0 : 1.0 / sqrt((double)s.n_pad);
  const int64_t off = s.sched.K > 0 ? s.stage_off[s.sched.K - 1] : 0;
  k_export_rows<<<512, 256, 0, c->stream>>>(
      s.mixed ? nullptr : s.AK + off * s.ldak, s.ldak,
      reinterpret_cast<const __nv_bfloat16*>(s.AK16) + off * s.ldak16, s.ldak16, s.bK + off, row0,
      n, c->d, scale, A, b);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

// The FP32 split X = Xh + Xl of the mixed-precision Stage II: the iterations
// read Xh, the true gradients read both halves.
// Xh = fl32(x) and Xl = fl32(x - Xh), round to nearest even, from the bit
// pattern of x with integer and FP32 operations: this GPU's FP64 pipe (and
// the double conversions) run at a small fraction of its integer and FP32
// rates.  The float image keeps the top 24 significant bits; the 29 dropped
// bits decide the rounding and, minus 2^29 when it rounded up, are the
// remainder x - Xh in units of 2^(e-52): an integer below 2^29 in magnitude,
// rounded once to FP32 and scaled exactly by a power of two.  Values outside
// 2^-74 <= |x| < 2^127 (zero, subnormal, huge, Inf, NaN) take the
// conversion instructions.
__device__ __forceinline__ void split_f32(double x, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -74 || e > 126) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
    return;
  }
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long frac = b & 0xFFFFFFFFFFFFFull;   // 52 fraction bits
  const unsigned dropped = (unsigned)(frac & 0x1FFFFFFFull);  // the low 29 bits
  unsigned mag = ((unsigned)(e + 127) << 23) | (unsigned)(frac >> 29);
  const bool up = dropped > 0x10000000u || (dropped == 0x10000000u && (mag & 1u));
  mag += up ? 1u : 0u;   // a carry into the exponent field is the correct rounding
  h = __uint_as_float(sign | mag);
  const int rem = (int)dropped - (up ? (1 << 29) : 0);
  const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);   // 2^(e-52), normal
  l = (float)(sign ? -rem : rem) * scale;   // an exact zero stays +0, as x - Xh does
}

// Xh, Xl for an N x d block: one warp per row, 16-byte loads, four loads in
// flight per lane before the stores.  With CM, the same read of X also yields
// per-column maxima for the fixed-point scales: the largest high word (sign
// cleared) of the IEEE patterns of each column of X and of Y.  The high word
// holds the exponent, and k_colscale reads only the exponent, so the scales
// equal those from k_colmax's full maxima.  A lane keeps the maxima of its
// fixed column pairs in registers, a CTA merges them in shared memory and
// posts one atomicMax per column (as high word << 32).
template <bool CM>
__global__ void __launch_bounds__(256) k_to_f32(const double* __restrict__ X, int64_t ldx,
                                                int64_t N, int d, float* __restrict__ Xf,
                                                float* __restrict__ Xl, int64_t ldxf,
                                                const double* __restrict__ Y,
                                                unsigned long long* __restrict__ colmax) {
  constexpr int U = 4;
  constexpr int S = (SPCG_MAX_D / 2 + 32 * U - 1) / (32 * U);   // column-pair steps
  __shared__ unsigned smax[CM ? SPCG_MAX_D + 1 : 1];
  const int lane = threadIdx.x & 31;
  const int full = d / 2;   // complete column pairs
  unsigned mx[S][U][2], mtail = 0, my = 0;
  if (CM) {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int u = 0; u < U; ++u) mx[s][u][0] = mx[s][u][1] = 0;
    for (int c = threadIdx.x; c <= d; c += blockDim.x) smax[c] = 0;
  }
  for (int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); i < N;
       i += (int64_t)gridDim.x * 8) {
    const double* xr = X + i * ldx;
    float* hr = Xf + i * ldxf;
    float* lr = Xl + i * ldxf;
    // one block of S steps covers d <= SPCG_MAX_D (the CM case); the plain
    // split takes any d
    for (int qb = 0; qb < full; qb += S * 32 * U)
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int q0 = qb + s * 32 * U;
      if (q0 < full) {
        double2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = q0 + u * 32 + lane;
          if (q < full) v[u] = __ldcs(reinterpret_cast<const double2*>(xr) + q);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = q0 + u * 32 + lane;
          if (q < full) {
            float h0, l0, h1, l1;
            split_f32(v[u].x, h0, l0);
            split_f32(v[u].y, h1, l1);
            reinterpret_cast<float2*>(hr)[q] = make_float2(h0, h1);
            reinterpret_cast<float2*>(lr)[q] = make_float2(l0, l1);
            if (CM) {
              mx[s][u][0] = max(mx[s][u][0], (unsigned)__double2hiint(v[u].x) & 0x7FFFFFFFu);
              mx[s][u][1] = max(mx[s][u][1], (unsigned)__double2hiint(v[u].y) & 0x7FFFFFFFu);
            }
          }
        }
      }
    }
    if ((d & 1) && lane == 0) {
      const double x = xr[d - 1];
      float h, l;
      split_f32(x, h, l);
      hr[d - 1] = h;
      lr[d - 1] = l;
      if (CM) {
        mtail = max(mtail, (unsigned)__double2hiint(x) & 0x7FFFFFFFu);
      }
    }
    if (CM && lane == 1) {
      my = max(my, (unsigned)__double2hiint(Y[i]) & 0x7FFFFFFFu);
    }
  }
  if (CM) {
    __syncthreads();   // smax cleared
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = s * 32 * U + u * 32 + lane;
        if (q < full) {
          if (mx[s][u][0]) atomicMax(&smax[2 * q], mx[s][u][0]);
          if (mx[s][u][1]) atomicMax(&smax[2 * q + 1], mx[s][u][1]);
        }
      }
    if (mtail) atomicMax(&smax[d - 1], mtail);
    if (my) atomicMax(&smax[d], my);
    __syncthreads();
    for (int c = threadIdx.x; c <= d; c += blockDim.x)
      if (smax[c]) atomicMax(colmax + c, (unsigned long long)smax[c] << 32);
  }
}

// Resident CTAs per SM of k_to_f32<CM> on the current device, computed once
// per device and variant (the answer depends on the device's limits; a racing
// first call on two threads computes the same value twice).
template <bool CM>
static int to_f32_blocks_per_sm() {
  static std::atomic<int> per_dev[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int v = per_dev[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_to_f32<CM>, 256, 0) != cudaSuccess ||
      v < 1) {
    (void)cudaGetLastError();
    return 1;
  }
  per_dev[dev].store(v, std::memory_order_relaxed);
  return v;
}

spcg_status launch_to_f32(spcg_ctx* c) {
  // one wave of resident CTAs: the grid-stride loop then has no tail wave
  k_to_f32<false><<<to_f32_blocks_per_sm<false>() * c->num_sms, 256, 0, c->stream>>>(
      c->X, c->ldx, c->N, c->d, c->Xf, c->Xl, c->ldxf, nullptr, nullptr);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 1;
  return SPCG_OK;
}

// The split and the column maxima of the next sketch in one read of X; the
// next launch_colscales (within the same spcg_sketch call) then skips k_colmax.
spcg_status launch_to_f32_colmax(spcg_ctx* c) {
  Sketch& s = c->sk;
  SPCG_CK(cudaMemsetAsync(s.colmax, 0, (size_t)(c->d + 1) * sizeof(unsigned long long),
                          c->stream));
  k_to_f32<true><<<to_f32_blocks_per_sm<true>() * c->num_sms, 256, 0, c->stream>>>(
      c->X, c->ldx, c->N, c->d, c->Xf, c->Xl, c->ldxf, c->Y, s.colmax);
  SPCG_CK(cudaGetLastError());
  s.colmax_pre = true;
  c->n_launch += 1;
  return SPCG_OK;
}

}  // namespace spcg

extern "C" spcg_status spcg_split_f32(const double* X, int64_t N, int32_t d, int64_t ldx,
                                      float* Xh, float* Xl, int64_t ldxf, void* stream) {
  if (N < 0 || d < 1 || ldx < d || ldxf < d) return SPCG_E_INVALID_ARG;
  if (N == 0) return SPCG_OK;
  if (!X || !Xh || !Xl || (ldx & 1) || (ldxf & 1) || ((uintptr_t)X & 15u) ||
      ((uintptr_t)Xh & 7u) || ((uintptr_t)Xl & 7u))
    return SPCG_E_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPCG_E_CUDA;
  spcg::k_to_f32<false><<<spcg::to_f32_blocks_per_sm<false>() * sms, 256, 0, (cudaStream_t)stream>>>(
      X, ldx, N, d, Xh, Xl, ldxf, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return SPCG_E_CUDA;
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? SPCG_OK : SPCG_E_CUDA;
}
