// Shared device helpers of the SPCG CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spcg.h"

#define SPCG_WARP 32

// Device-side error codes written to the context's status word; the host
// maps them to spcg_status.
enum : int {
  DEV_OK = 0,
  DEV_BREAKDOWN = 1,
  DEV_TIMEOUT = 2,
};

namespace spcg {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds; each round forms the 64-bit products
// of counter words 0 and 2 with two odd multipliers and mixes their halves
// with the key and words 1 and 3; the key advances by two Weyl increments
// between rounds.
// ---------------------------------------------------------------------------
struct u32x4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ u32x4 philox10(u32x4 c, uint64_t seed) {
  const uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  const uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kWeylA;
      k1 += kWeylB;
    }
    const uint64_t pa = (uint64_t)kMulA * c.x;
    const uint64_t pb = (uint64_t)kMulB * c.z;
    const uint32_t hia = (uint32_t)(pa >> 32), loa = (uint32_t)pa;
    const uint32_t hib = (uint32_t)(pb >> 32), lob = (uint32_t)pb;
    u32x4 n;
    n.x = hib ^ c.y ^ k0;
    n.y = lob;
    n.z = hia ^ c.w ^ k1;
    n.w = loa;
    c = n;
  }
  return c;
}

// Tags of the four independent draws of the sketch.
enum : uint32_t { TAG_P = 0, TAG_SIGN = 1, TAG_PI = 2, TAG_HAT = 3 };
constexpr int kFeistelRounds = 8;

// Rademacher sign of row k: +1 if bit 0 of word 0 of
// philox(ctr = (k lo, k hi, TAG_SIGN, 0)) is clear, else -1.
__host__ __device__ __forceinline__ int rademacher(uint64_t k, uint64_t seed) {
  u32x4 c{(uint32_t)k, (uint32_t)(k >> 32), TAG_SIGN, 0u};
  return (philox10(c, seed).x & 1u) ? -1 : 1;
}

// Alternating Feistel network on nbits-bit indices: high half L (nbits -
// nbits/2 bits), low half Rr (nbits/2 bits); even rounds L ^= F(Rr), odd
// rounds Rr ^= F(L), with F = word 0 of philox(ctr = (half, round, tag,
// nbits)) masked to the half's width.  Each round is its own inverse, so
// the map is a bijection and the inverse runs the rounds backwards.
__host__ __device__ __forceinline__ uint32_t feistel(uint32_t x, int nbits, uint32_t tag,
                                                     uint64_t seed, bool inverse) {
  const int lo_bits = nbits / 2, hi_bits = nbits - lo_bits;
  const uint32_t mask_hi = (hi_bits >= 32) ? 0xFFFFFFFFu : ((1u << hi_bits) - 1u);
  const uint32_t mask_lo = (1u << lo_bits) - 1u;
  uint32_t L = (x >> lo_bits) & mask_hi;
  uint32_t Rr = x & mask_lo;
  for (int i = 0; i < kFeistelRounds; ++i) {
    const int r = inverse ? (kFeistelRounds - 1 - i) : i;
    if ((r & 1) == 0) {
      u32x4 c{Rr, (uint32_t)r, tag, (uint32_t)nbits};
      L ^= philox10(c, seed).x & mask_hi;
    } else {
      u32x4 c{L, (uint32_t)r, tag, (uint32_t)nbits};
      Rr ^= philox10(c, seed).x & mask_lo;
    }
  }
  return (L << lo_bits) | Rr;
}

// ---------------------------------------------------------------------------
// Warp reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Grid barrier of a cooperative launch (every CTA of the grid is resident).
// bar[0] counts arrivals and bar[kBarGen] is the generation, on separate
// 128-byte lines so that the polling does not contend with the arrivals.
// Arrival is an acquire-release atomic add (it publishes the CTA's writes,
// ordered before it by the CTA barrier); the last CTA to arrive resets the
// count and releases the next generation; the others poll the generation
// with acquire loads and a short back-off, at most `spin` clock cycles.
// Returns false when the wait expired: the status word is set to DEV_TIMEOUT
// and the CTA must leave (the other CTAs then time out at their next
// barrier).  Called by every thread of the CTA; *s_fail is a shared flag, 0
// at kernel start.
// ---------------------------------------------------------------------------
constexpr int kBarGen = 32;      // word index of the generation
constexpr int kBarWords = 64;    // words a barrier occupies

__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(p), "r"(v)
               : "memory");
  return old;
}
__device__ __forceinline__ void st_release_gpu_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of the first `nparts` CTAs of the grid (the others must not call
// it with the same bar); grid_sync_bounded is the whole grid.
__device__ __forceinline__ bool group_sync_bounded(unsigned* bar, unsigned nparts, int* status,
                                                   long long spin, int* s_fail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* gen = bar + kBarGen;
    const unsigned g = ld_acquire_gpu_u32(gen);
    const unsigned prev = atom_add_acq_rel_gpu_u32(bar, 1u);
    if (prev == nparts - 1) {
      bar[0] = 0u;                      // ordered before the release below
      st_release_gpu_u32(gen, g + 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_gpu_u32(gen) == g) {
        if (clock64() - t0 > spin) {
          atomicExch(status, DEV_TIMEOUT);
          *s_fail = 1;
          break;
        }
        __nanosleep(32);
      }
    }
  }
  __syncthreads();
  return *s_fail == 0;
}

__device__ __forceinline__ bool grid_sync_bounded(unsigned* bar, int* status, long long spin,
                                                  int* s_fail) {
  return group_sync_bounded(bar, gridDim.x, status, spin, s_fail);
}

}  // namespace spcg
