// PCG(A, b, H-hat, beta_init, a) of Sec. 2.2 on the normal equations,
// preconditioned by H-hat = R^T R.  One iteration is
//   w = A^T (A p); alpha = gamma / (p.w); beta += alpha p; g -= alpha w;
//   z = R^{-1} (R^{-T} g); gamma' = g.z; p = z + (gamma'/gamma) p
// (the d-space recurrence whose cost is the (4m + 13)d + 2d^2 flops that
// Sec. 2.2 charges per iteration).  Kernels per iteration:
//   k_pass      fused prologue (gamma', new p, stopping test) + one read of A:
//               per-CTA partials of A^T (A p), row tiles staged by TMA
//   k_dspace    one cooperative launch: partials -> w and p.w; alpha, g and
//               beta updates, u = R^{-T} g; z = R^{-1} u and the partial dots
//               g.z and ||R beta||^2 that the next pass's prologue adds
// The stage start uses the same pass in residual mode: g = A^T (b - A beta).
// (k_reduce, the partials -> w sum alone, serves the plain-pass entry points.)
// All reductions run in a fixed order, so two runs give identical bits.
//
// Stopping state (DevScalars::done), kept on the device so that a Stage II
// schedule can be enqueued without reading it back: 1 when a pass prologue
// finds the recursive test met (iterations then do nothing), 2 when k_check
// confirms it on a true gradient (then everything does nothing); k_check sets
// 0 again when the true gradient fails the test, and iterations resume from it.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.hpp"

namespace spcg {

// --------------------------------------------------------------------------
// mbarrier / TMA helpers (inline PTX, sm_90+ instructions used on sm_103a)
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false once `budget` clock cycles have passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}
// L2 policy for operand tiles that are read once per pass: evict first, so
// that a pass streaming gigabytes does not push the d x d factors, the
// per-CTA partials and the d-vectors (read between passes) out of L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

constexpr int kConsumers = 12;                // consumer warps of the FP64 and FP32 passes
constexpr int kMaxConsumers = 15;             // the most any pass uses (scratch sizing)
// Consumer warps per CTA: fewer for the widest rows, whose accumulators need
// the registers; BF16 rows, and FP32 rows up to 512 columns, take 15 (more
// warps hide the latency of short rows: BF16 10-17 % faster than with 12 at
// 128-1000 columns, FP32 13-15 % at 128-256 columns).
// (Registers come in blocks of four warps: 13 warps get no more registers
// than 16 would, 12 warps get as many as 12.)
template <int NI, int ES = 8>   // ES: element size of the operand
struct PassCfg {
  static constexpr int C = ES == 2 ? kMaxConsumers
                          : (NI < 32 ? (ES == 4 ? kMaxConsumers : kConsumers) : (ES == 8 ? 8 : 11));
  static constexpr int THREADS = 32 * (C + 1);
};
constexpr int kMaxStages = 8;

enum PassMode : int { PASS_PLAIN = 0, PASS_ITER = 1, PASS_RESID = 2 };

struct PassArgs {
  int64_t m;
  int d, nbox, boxc, tm, ntiles, stages;
  uint32_t tx_bytes;       // bytes one stage's boxes deliver
  uint32_t slot_elems;     // elements between box slots (128-byte multiple)
  uint32_t stage_elems;    // elements between stages
  uint32_t region_bytes;   // bytes of the staging region (also the reduction scratch)
  int mode;
  const double* vec;       // PLAIN: p; RESID: beta
  const double* b;         // RESID: right-hand side
  double* partials;
  int ldp;
  // PASS_ITER prologue
  const double* z;
  const double* p_prev;
  double* p_next;
  const double* dots_gz;
  const double* dots_rb;
  int n_dots;
  int gp;                  // gamma ping-pong index of the previous direction
  int start;               // 1: p = z (first iteration after a (re)start)
  int check;               // 1: stop when sqrt(gamma) <= tau ||R beta||
  double tau;
  DevScalars* scal;
  long long spin;
  int inject_stall;        // test hook: CTA 0 never issues its first tile
};

// Fixed-order sum of n values by one warp: lanes stride, then xor tree.
__device__ __forceinline__ double warp_sum_array(const double* v, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += v[i];
  return warp_allsum(s);
}

// PASS_ITER prologue of both fused passes: gamma = g.z and ||R beta||^2 from
// the previous launch's per-block partial dots, the breakdown and stopping
// tests, and the CG ratio gamma / gamma_prev.  Called by every thread of the
// CTA; false means the pass must not run (the caller returns before issuing a
// copy).  The decision is uniform over the grid: every CTA reads the same
// partials.
__device__ bool iter_prologue(const PassArgs& a, double* s_scal, double& ratio) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    const double gam = warp_sum_array(a.dots_gz, a.n_dots);
    const double rb2 = warp_sum_array(a.dots_rb, a.n_dots);
    if (lane == 0) {
      s_scal[0] = gam;
      s_scal[1] = sqrt(rb2);
    }
  }
  __syncthreads();
  const double gam = s_scal[0], rb = s_scal[1];
  int flag = 0;
  if (!isfinite(gam) || gam < 0.0) flag = 2;
  else if (gam == 0.0 || (a.check && sqrt(gam) <= a.tau * rb)) flag = 1;
  if (flag) {
    if (blockIdx.x == 0 && tid == 0) {
      if (flag == 2) atomicExch(&a.scal->status, DEV_BREAKDOWN);
      else {
        a.scal->done = 1;
        a.scal->sqrt_gamma = sqrt(gam);
        a.scal->norm_rb = rb;
      }
    }
    return false;
  }
  ratio = a.start ? 0.0 : gam / a.scal->gam[a.gp];
  if (blockIdx.x == 0 && tid == 0) {
    a.scal->gam[a.gp ^ 1] = gam;
    a.scal->iters += 1;
  }
  return true;
}

// Element types of the operand and the accumulation they use: FP64 rows
// accumulate in FP64; FP32 rows (the refinement copy of X) form t = a.p in
// FP32 and add t a into FP32 block sums that are folded into a compensated
// (TwoSum) accumulator every few tiles, so the long sums over rows keep about
// twice the FP32 precision; BF16 rows (the sketched prefix of Stage I) use
// plain FP32 throughout.
template <typename T> struct PassElem;
template <> struct PassElem<double> {
  using acc = double;
  static constexpr bool compensated = false;
  __device__ static double load(double x) { return x; }
  __device__ static void load_vec(const double* p, double (&x)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x;
    x[1] = v.y;
  }
};
template <> struct PassElem<float> {
  using acc = float;
  static constexpr bool compensated = true;
  __device__ static float load(float x) { return x; }
  __device__ static void load_vec(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  }
};
template <> struct PassElem<__nv_bfloat16> {
  using acc = float;
  static constexpr bool compensated = false;
  __device__ static float load(__nv_bfloat16 x) { return __bfloat162float(x); }
  __device__ static void load_vec(const __nv_bfloat16* p, float (&x)[8]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {   // a BF16 is the top half of an FP32
      x[2 * i] = __uint_as_float(w[i] << 16);
      x[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};

template <typename T, int NI>
__global__ void __launch_bounds__(PassCfg<NI, sizeof(T)>::THREADS, 1)
    k_pass(const __grid_constant__ CUtensorMap tmap, const PassArgs a) {
  constexpr int kConsumers = PassCfg<NI, sizeof(T)>::C;
  using E = PassElem<T>;
  // Each consumer lane owns runs of V consecutive columns (one 16-byte vector
  // of the row in shared memory), NG runs in all, RS columns covered.
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int NG = (NI * 32 + 32 * V - 1) / (32 * V);
  constexpr int RS = NG * 32 * V;
  using acc_t = typename E::acc;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_addr = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((128u - (base_addr & 127u)) & 127u);
  T* tiles = reinterpret_cast<T*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.region_bytes);
  uint64_t* empty = full + kMaxStages;
  acc_t* vec_s = reinterpret_cast<acc_t*>(empty + kMaxStages);  // RS values
  __shared__ int s_flag;       // 1 = skip the pass (done / error)
  __shared__ int s_abort;
  __shared__ double s_scal[2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // uniform over the grid: an error, or the stopping test passed (done 1: the
  // recursive test, only a residual pass still runs, to confirm; done 2:
  // confirmed on the true gradient)
  if (a.scal->status != 0 || a.scal->done > (a.mode == PASS_RESID ? 1 : 0)) return;

  if (tid == 0) {
    s_flag = 0;
    s_abort = 0;
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }

  // ---- prologue: the direction this pass multiplies ----
  double ratio = 0.0;
  if (a.mode == PASS_ITER && !iter_prologue(a, s_scal, ratio)) return;   // no TMA issued yet
  for (int j = tid; j < RS; j += blockDim.x) {
    double v = 0.0;
    if (j < a.d) {
      if (a.mode == PASS_ITER) {
        v = a.z[j] + ratio * a.p_prev[j];
        if (blockIdx.x == 0) a.p_next[j] = v;
      } else {
        v = a.vec[j];
      }
    }
    vec_s[j] = (acc_t)v;
  }
  __syncthreads();

  const int my_tiles =
      (blockIdx.x < a.ntiles) ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  acc_t wv[NG][V], wb[E::compensated ? NG : 1][V], wc[E::compensated ? NG : 1][V];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      wv[g][v] = (acc_t)0;
      if constexpr (E::compensated) wb[g][v] = wc[g][v] = (acc_t)0;
    }
  int issued = 0, skipped = -1;   // producer thread (tid 0) only

  if (warp == 0) {
    // ---- producer: one lane issues the TMA box loads of each row tile ----
    if (lane == 0) {
      const uint64_t pol = l2_evict_first_policy();
      for (int k = 0; k < my_tiles; ++k) {
        const int s = k % a.stages;
        if (k >= a.stages) {
          if (!mbar_wait_bounded(&empty[s], ((k / a.stages) - 1) & 1, a.spin)) {
            atomicExch(&a.scal->status, DEV_TIMEOUT);
            s_abort = 1;
            break;
          }
        }
        if (*(volatile int*)&s_abort) break;
        issued = k + 1;
        if (a.inject_stall && blockIdx.x == 0 && k == 0) {
          skipped = 0;   // the consumers' wait on this tile can only time out
          continue;
        }
        const int tile = blockIdx.x + k * gridDim.x;
        mbar_expect_tx(&full[s], a.tx_bytes);
        T* dst = tiles + (size_t)s * a.stage_elems;
        for (int bx = 0; bx < a.nbox; ++bx)
          tma_load_2d(dst + (size_t)bx * a.slot_elems, &tmap, bx * a.boxc, tile * a.tm,
                      &full[s], pol);
      }
    }
  } else {
    // ---- consumers: t = a_row . v (warp all-reduce), acc += t a_row ----
    // WIDE: p and the row come from shared memory (FP64 rows, and FP32 rows
    // of more than 512 columns, whose compensated accumulators fill the
    // registers); otherwise both stay in registers
    constexpr bool WIDE = (NI >= 32 && E::compensated) || sizeof(acc_t) == 8;
    constexpr int RW = (sizeof(acc_t) == 4 && !WIDE && NI < 32) ? 2 : 1;   // rows in flight
    constexpr int FLUSH = 8;                                     // tiles per compensated flush
    const int cw = warp - 1;
    int off[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int c0 = g * 32 * V + lane * V;
      off[g] = (c0 < a.d) ? (c0 / a.boxc) * (int)a.slot_elems + (c0 % a.boxc) : -1;
    }
    acc_t pv[WIDE ? 1 : NG][V];
    if constexpr (!WIDE) {
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int v = 0; v < V; ++v) pv[g][v] = vec_s[g * 32 * V + lane * V + v];
    }
    for (int k = 0; k < my_tiles; ++k) {
      const int s = k % a.stages;
      if (!mbar_wait_bounded(&full[s], (k / a.stages) & 1, a.spin)) {
        atomicExch(&a.scal->status, DEV_TIMEOUT);
        s_abort = 1;
        break;
      }
      const int tile = blockIdx.x + k * gridDim.x;
      const int64_t row0 = (int64_t)tile * a.tm;
      const T* st = tiles + (size_t)s * a.stage_elems;
      // row r of the CTA's row stream (tile k, row rr) belongs to consumer
      // r mod C: every consumer stays busy when a tile has fewer rows than
      // there are consumers (wide FP64 rows)
      const int r0 = (int)(((int64_t)cw - (int64_t)k * a.tm) % kConsumers + kConsumers) % kConsumers;
      for (int rr = r0; rr < a.tm; rr += RW * kConsumers) {
        if (row0 + rr >= a.m) break;
        const T* rowp[RW];
        bool live[RW];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
          const int rq = rr + q * kConsumers;
          live[q] = (q == 0) || (rq < a.tm && row0 + rq < a.m);
          rowp[q] = st + (live[q] ? rq : rr) * a.boxc;
        }
        acc_t xr[WIDE ? 1 : RW][WIDE ? 1 : NG][V];
        acc_t t[RW];
#pragma unroll
        for (int q = 0; q < RW; ++q) t[q] = (acc_t)0;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (off[g] < 0) continue;
          acc_t pq[V];
          if constexpr (WIDE) {   // 16-byte loads of this lane's V entries of p
            const int4* src = reinterpret_cast<const int4*>(vec_s + g * 32 * V + lane * V);
            constexpr int NV = (int)(V * sizeof(acc_t) / 16);
#pragma unroll
            for (int u = 0; u < NV; ++u) {
              const int4 raw = src[u];
              memcpy(&pq[u * (16 / sizeof(acc_t))], &raw, 16);
            }
          } else {
#pragma unroll
            for (int v = 0; v < V; ++v) pq[v] = pv[WIDE ? 0 : g][v];
          }
#pragma unroll
          for (int q = 0; q < RW; ++q) {
            acc_t x[V];
            E::load_vec(rowp[q] + off[g], x);
#pragma unroll
            for (int v = 0; v < V; ++v) {
              t[q] = fma(x[v], pq[v], t[q]);
              if constexpr (!WIDE) xr[q][g][v] = x[v];
            }
          }
        }
#pragma unroll
        for (int q = 0; q < RW; ++q) {
          t[q] = warp_allsum(t[q]);
          // b is read only for a live row: the second row in flight may lie
          // past the operand's last row (b has exactly m entries)
          if (!live[q]) t[q] = (acc_t)0;
          else if (a.mode == PASS_RESID) t[q] = (acc_t)a.b[row0 + rr + q * kConsumers] - t[q];
        }
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (off[g] < 0) continue;
#pragma unroll
          for (int q = 0; q < RW; ++q) {
            acc_t x[V];
            if constexpr (WIDE) E::load_vec(rowp[q] + off[g], x);
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const acc_t xx = WIDE ? x[v] : xr[WIDE ? 0 : q][WIDE ? 0 : g][v];
              wv[g][v] = fma(t[q], xx, wv[g][v]);
            }
          }
        }
      }
      if constexpr (E::compensated) {
        // fold the block sums into the compensated accumulator (TwoSum)
        if ((k % FLUSH) == FLUSH - 1 || k == my_tiles - 1) {
#pragma unroll
          for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const acc_t sm = wb[g][v] + wv[g][v];
              const acc_t bb = sm - wb[g][v];
              wc[g][v] += (wb[g][v] - (sm - bb)) + (wv[g][v] - bb);
              wb[g][v] = sm;
              wv[g][v] = (acc_t)0;
            }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();

  if (s_abort && tid == 0) {
    // let every copy still in flight land before the CTA leaves (generous
    // bound, independent of the caller's spin budget)
    const int first = issued > a.stages ? issued - a.stages : 0;
    for (int k = first; k < issued; ++k)
      if (k != skipped)
        (void)mbar_wait_bounded(&full[k % a.stages], (k / a.stages) & 1, 1ll << 31);
  }
  __syncthreads();

  // ---- CTA partial: fixed-order sum over the consumer warps ----
  double* red = reinterpret_cast<double*>(smem);   // reuse stage memory: kConsumers x RS
  if (warp > 0) {
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        double val;
        if constexpr (E::compensated) val = ((double)wb[g][v] + (double)wc[g][v]) + (double)wv[g][v];
        else val = (double)wv[g][v];
        red[(size_t)(warp - 1) * RS + g * 32 * V + lane * V + v] = val;
      }
  }
  __syncthreads();
  for (int j = tid; j < a.d; j += blockDim.x) {
    double sum = 0.0;
#pragma unroll 4
    for (int w = 0; w < kConsumers; ++w) sum += red[(size_t)w * RS + j];
    a.partials[(size_t)blockIdx.x * a.ldp + j] = sum;
  }
}

// partials (nb x ldp) -> out[d]; optional per-CTA dots out.dotvec
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ partials, int nb,
                                                int ldp, int d, double* __restrict__ out,
                                                const double* __restrict__ dotvec,
                                                double* __restrict__ dots_out,
                                                const DevScalars* __restrict__ scal) {
  if (scal->status != 0 || scal->done != 0) return;
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (col < d)
    for (int b = warp; b < nb; b += 8) s += partials[(size_t)b * ldp + col];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    if (col < d) out[col] = t;
    if (dotvec) {
      double v = (col < d) ? t * dotvec[col] : 0.0;
      v = warp_allsum(v);
      if (lane == 0) dots_out[blockIdx.x] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// The d-space work between two fused passes in ONE cooperative launch.  It
// replaces k_reduce + k_precondT + k_precond (three launches) with three
// phases separated by bounded grid barriers:
//   1. columns of the pass output: w = sum of the per-CTA partials (the
//      residual pass of a (re)start gives g directly), share of p.w;
//   2. alpha = gamma / p.w, g' = g - alpha w (every CTA forms all of g'),
//      beta += alpha p (own columns), u = R^{-T} g' (own rows);
//   3. z = R^{-1} u and (R beta)_i (own rows), shares of g'.z and ||R beta||^2.
// The next pass's prologue adds the shares (gamma', the stopping test, p).
// Rows of the triangular products are dealt round-robin to all warps of the
// grid, so long and short rows mix; every sum runs in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kDsThreads = 256;
constexpr int kDsWarps = kDsThreads / 32;
constexpr int kDsUnroll = 8;   // independent loads a lane has in flight

struct DspaceArgs {
  int d;
  int iter;                 // 0: (re)start from a residual pass; 1: PCG iteration
  const double* partials;   // nb x ldp per-CTA partials of the pass
  int nb, ldp;
  const double* R;          // d x d row-major upper
  const double* Rinv;       // d x d row-major upper
  const double* RinvT;      // d x d row-major lower
  const double* g_cur;      // iter: current gradient
  double* g_nxt;            // the new gradient (start: the reduced pass output)
  double* w;                // iter: A^T A p
  const double* p;          // iter: the direction the pass multiplied
  double* beta;
  double* u;
  double* z;
  double* dots_pw;          // gridDim.x shares
  double* dots_gz;
  double* dots_rb;
  int gp;                   // gamma index of the current direction
  DevScalars* scal;
  unsigned* bar;
  long long spin;
};

// Fixed-order sum of one value per warp (lane 0's) over the CTA, by thread 0.
__device__ __forceinline__ void ds_block_sum2(double a0, double a1, double (*red)[2], double* o0,
                                              double* o1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp][0] = a0;
    red[warp][1] = a1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int k = 0; k < kDsWarps; ++k) {
      s0 += red[k][0];
      s1 += red[k][1];
    }
    if (o0) *o0 = s0;
    if (o1) *o1 = s1;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kDsThreads) k_dspace(const DspaceArgs a) {
  extern __shared__ double ds_sm[];
  double* gs = ds_sm;          // g' (all d)
  double* us = gs + a.d;       // u (all d)
  double* bs = us + a.d;       // beta (all d)
  __shared__ int s_fail;
  __shared__ double s_red[kDsWarps][2];
  __shared__ double s_alpha;
  // uniform over the grid; a (re)start still runs after the recursive test
  // passed (done 1), to confirm it on the true gradient
  if (a.scal->status != 0 || a.scal->done > (a.iter ? 0 : 1)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, q = blockIdx.x, d = a.d;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  const int cs = (d + G - 1) / G;
  const int c_lo = q * cs, c_hi = c_lo + cs < d ? c_lo + cs : d;
  // 1. own columns of the pass output
  double pw = 0.0;
  for (int j = c_lo + warp; j < c_hi; j += kDsWarps) {
    double sacc = 0.0;
    for (int b0 = 0; b0 < a.nb; b0 += 32 * kDsUnroll) {   // loads first, then the sums in order
      double v[kDsUnroll];
#pragma unroll
      for (int k = 0; k < kDsUnroll; ++k) {
        const int b = b0 + lane + 32 * k;
        v[k] = b < a.nb ? a.partials[(size_t)b * a.ldp + j] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kDsUnroll; ++k) sacc += v[k];
    }
    sacc = warp_allsum(sacc);
    if (lane == 0) {
      if (a.iter) {
        a.w[j] = sacc;
        pw = fma(sacc, a.p[j], pw);
      } else {
        a.g_nxt[j] = sacc;
      }
    }
  }
  if (a.iter) ds_block_sum2(pw, 0.0, s_red, &a.dots_pw[q], nullptr);
  if (!grid_sync_bounded(a.bar, &a.scal->status, a.spin, &s_fail)) return;
  // 2. alpha, g', beta, u = R^{-T} g'
  double alpha = 0.0;
  if (a.iter) {
    if (warp == 0) {
      double t = 0.0;
      for (int k = lane; k < G; k += 32) t += a.dots_pw[k];
      t = warp_allsum(t);
      if (lane == 0) {
        const double al = a.scal->gam[a.gp] / t;
        s_alpha = (t > 0.0 && isfinite(al)) ? al : NAN;
      }
    }
    __syncthreads();
    alpha = s_alpha;
    if (isnan(alpha)) {   // the same value in every CTA: all leave here
      if (q == 0 && tid == 0) atomicExch(&a.scal->status, DEV_BREAKDOWN);
      return;
    }
    for (int j = tid; j < d; j += kDsThreads) gs[j] = fma(-alpha, a.w[j], a.g_cur[j]);
    for (int j = c_lo + tid; j < c_hi; j += kDsThreads) {
      a.g_nxt[j] = fma(-alpha, a.w[j], a.g_cur[j]);
      a.beta[j] = fma(alpha, a.p[j], a.beta[j]);
    }
  } else {
    for (int j = tid; j < d; j += kDsThreads) gs[j] = a.g_nxt[j];
  }
  __syncthreads();
  const int W = G * kDsWarps, gw = q * kDsWarps + warp;
  for (int i = gw; i < d; i += W) {
    const double* Ri = a.RinvT + (size_t)i * d;
    double sacc = 0.0;
    for (int j0 = 0; j0 <= i; j0 += 32 * kDsUnroll) {   // row entries 0..i
      double v[kDsUnroll];
#pragma unroll
      for (int k = 0; k < kDsUnroll; ++k) {
        const int j = j0 + lane + 32 * k;
        v[k] = j <= i ? Ri[j] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kDsUnroll; ++k) {
        const int j = j0 + lane + 32 * k;
        if (j <= i) sacc = fma(v[k], gs[j], sacc);
      }
    }
    sacc = warp_allsum(sacc);
    if (lane == 0) a.u[i] = sacc;
  }
  if (!grid_sync_bounded(a.bar, &a.scal->status, a.spin, &s_fail)) return;
  // 3. z = R^{-1} u, (R beta)_i, shares of g'.z and ||R beta||^2
  for (int j = tid; j < d; j += kDsThreads) {
    us[j] = a.u[j];
    bs[j] = a.beta[j];
  }
  __syncthreads();
  double gz = 0.0, rb2 = 0.0;
  for (int i = gw; i < d; i += W) {
    const double* Ri = a.Rinv + (size_t)i * d;
    const double* Rr = a.R + (size_t)i * d;
    double zs = 0.0, rs = 0.0;
    for (int j0 = i; j0 < d; j0 += 32 * kDsUnroll) {   // row entries i..d-1
      double vz[kDsUnroll], vr[kDsUnroll];
#pragma unroll
      for (int k = 0; k < kDsUnroll; ++k) {
        const int j = j0 + lane + 32 * k;
        vz[k] = j < d ? Ri[j] : 0.0;
        vr[k] = j < d ? Rr[j] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kDsUnroll; ++k) {
        const int j = j0 + lane + 32 * k;
        if (j < d) {
          zs = fma(vz[k], us[j], zs);
          rs = fma(vr[k], bs[j], rs);
        }
      }
    }
    zs = warp_allsum(zs);
    rs = warp_allsum(rs);
    if (lane == 0) {
      a.z[i] = zs;
      gz = fma(gs[i], zs, gz);
      rb2 = fma(rs, rs, rb2);
    }
  }
  ds_block_sum2(gz, rb2, s_red, &a.dots_gz[q], &a.dots_rb[q]);
}

// The stopping test on freshly computed dots of a true gradient (same sums as
// the pass prologue): done = 2 (confirmed) when it holds, else 0 (iterate on
// from this gradient).  Nothing to do once confirmed.
__global__ void k_check(const double* __restrict__ dots_gz, const double* __restrict__ dots_rb,
                        int n, double tau, DevScalars* __restrict__ scal) {
  if (scal->status != 0 || scal->done == 2) return;
  const double gam = warp_sum_array(dots_gz, n);
  const double rb2 = warp_sum_array(dots_rb, n);
  if (threadIdx.x == 0) {
    const double rb = sqrt(rb2);
    scal->sqrt_gamma = sqrt(fmax(gam, 0.0));
    scal->norm_rb = rb;
    if (!isfinite(gam) || gam < 0.0) scal->status = DEV_BREAKDOWN;
    else scal->done = (gam == 0.0 || sqrt(gam) <= tau * rb) ? 2 : 0;
  }
}

__global__ void k_reset(DevScalars* scal, int clear_status, unsigned* bar) {
  if (clear_status) scal->status = 0;
  scal->done = 0;
  scal->iters = 0;
  if (bar) bar[0] = 0u;   // arrivals of the grid barrier (a timed-out wait leaves a count)
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver entry point, looked up once (a function-local static is
// initialised exactly once even when several host threads get here first).
static EncodeTiledFn get_encode() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return nullptr;
  }();
  return fn;
}

static int ni_for(int d) {
  const int n = (d + 31) / 32;
  int ni = 1;
  while (ni < n) ni <<= 1;
  return ni;
}

spcg_status make_pass_geom_t(const void* A, int64_t m, int d, int64_t lda, int dtype,
                             PassGeom* g) {
  const int es = dtype == DT_F64 ? 8 : (dtype == DT_F32 ? 4 : 2);
  if (m < 1 || d < 1 || d > SPCG_MAX_D || lda < d || (lda * es) % 16 != 0 ||
      ((uintptr_t)A & 15u) != 0)
    return SPCG_E_INVALID_ARG;
  g->m = m;
  g->d = d;
  g->dtype = dtype;
  g->esize = es;
  g->nbox = (d + 255) / 256;
  const int align = 16 / es;   // box inner extent: a multiple of 16 bytes
  int bc = (d + g->nbox - 1) / g->nbox;
  bc = (bc + align - 1) / align * align;
  g->boxc = bc;
  const int row_bytes = g->nbox * bc * es;
  int tm = 32768 / row_bytes;
  if (tm > 8) tm &= ~7;
  if (tm < 1) tm = 1;
  if (tm > 256) tm = 256;
  if (tm > m) tm = (int)m;
  g->tm = tm;
  g->ntiles = (int)((m + tm - 1) / tm);
  const size_t slot = (((size_t)tm * bc * es) + 127) & ~(size_t)127;
  const size_t stage = slot * g->nbox;
  int stages = (int)((192 * 1024) / stage);
  if (stages > kMaxStages) stages = kMaxStages;
  if (stages < 2) stages = 2;
  g->stages = stages;
  g->stage_bytes = stage;
  const size_t ni32 = (size_t)ni_for(d) * 32;
  const size_t cover = ni32 > 256 ? ni32 : 256;   // columns a consumer warp covers
  size_t red = (size_t)kMaxConsumers * cover * 8;
  size_t tiles = stage * stages;
  if (tiles < red) tiles = red;
  g->region_bytes = tiles;
  g->smem_bytes = 128 + tiles + 2 * kMaxStages * 8 + cover * 8;
  EncodeTiledFn enc = get_encode();
  if (!enc) return SPCG_E_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)(lda * es)};
  cuuint32_t box[2] = {(cuuint32_t)bc, (cuuint32_t)tm};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType tdt = dtype == DT_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                  : dtype == DT_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = enc(&g->tmap, tdt, 2, const_cast<void*>(A), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SPCG_OK : SPCG_E_CUDA;
}

spcg_status make_pass_geom(const double* A, int64_t m, int d, int64_t lda, PassGeom* g) {
  return make_pass_geom_t(A, m, d, lda, DT_F64, g);
}

template <typename T, int NI>
static spcg_status launch_pass_ni(spcg_ctx* c, const PassGeom& g, const PassArgs& a, int grid) {
  SPCG_CK(cudaFuncSetAttribute(k_pass<T, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)g.smem_bytes));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int op = g.dtype == DT_F64 ? OP_F64 : (g.dtype == DT_F32 ? OP_F32 : OP_BF16);
  if (c->opts.profile) SPCG_TRY(prof_events(c, &e0, &e1, op));
  if (e0) SPCG_CK(cudaEventRecord(e0, c->stream));
  k_pass<T, NI><<<grid, PassCfg<NI, sizeof(T)>::THREADS, g.smem_bytes, c->stream>>>(g.tmap, a);
  SPCG_CK(cudaGetLastError());
  if (e1) SPCG_CK(cudaEventRecord(e1, c->stream));
  c->n_launch += 1;
  c->n_pass += 1;
  c->pass_bytes += (uint64_t)g.m * g.d * g.esize;
  c->n_pass_op[op] += 1;
  c->pass_bytes_op[op] += (uint64_t)g.m * g.d * g.esize;
  return SPCG_OK;
}

template <typename T>
static spcg_status dispatch_ni(spcg_ctx* c, const PassGeom& g, const PassArgs& a, int grid) {
  switch (ni_for(g.d)) {
    case 1: return launch_pass_ni<T, 1>(c, g, a, grid);
    case 2: return launch_pass_ni<T, 2>(c, g, a, grid);
    case 4: return launch_pass_ni<T, 4>(c, g, a, grid);
    case 8: return launch_pass_ni<T, 8>(c, g, a, grid);
    case 16: return launch_pass_ni<T, 16>(c, g, a, grid);
    case 32: return launch_pass_ni<T, 32>(c, g, a, grid);
    default: return SPCG_E_INVALID_ARG;
  }
}

static spcg_status launch_pass(spcg_ctx* c, const PassGeom& g, PassArgs a) {
  int grid = c->pb.grid;
  if (grid > g.ntiles) grid = g.ntiles;
  if (grid < 1) grid = 1;
  a.m = g.m;
  a.d = g.d;
  a.nbox = g.nbox;
  a.boxc = g.boxc;
  a.tm = g.tm;
  a.ntiles = g.ntiles;
  a.stages = g.stages;
  a.tx_bytes = (uint32_t)((size_t)g.nbox * g.boxc * g.tm * g.esize);
  a.slot_elems = (uint32_t)(g.stage_bytes / g.nbox / g.esize);
  a.stage_elems = (uint32_t)(g.stage_bytes / g.esize);
  a.region_bytes = (uint32_t)g.region_bytes;
  a.partials = c->pb.partials;
  a.ldp = c->pb.ldp;
  a.scal = c->scal;
  a.spin = c->opts.spin_budget > 0 ? c->opts.spin_budget : (1ll << 31);
  a.inject_stall = c->opts.inject_stall;
  c->pb.last_grid = grid;
  if (g.dtype == DT_F64) return dispatch_ni<double>(c, g, a, grid);
  if (g.dtype == DT_F32) return dispatch_ni<float>(c, g, a, grid);
  return dispatch_ni<__nv_bfloat16>(c, g, a, grid);
}

spcg_status pass_resid(spcg_ctx* c, const PassGeom& g, const double* b, const double* x) {
  PassArgs a{};
  a.mode = PASS_RESID;
  a.vec = x;
  a.b = b;
  return launch_pass(c, g, a);
}

spcg_status pass_gram_plain(spcg_ctx* c, const PassGeom& g, const double* p) {
  PassArgs a{};
  a.mode = PASS_PLAIN;
  a.vec = p;
  return launch_pass(c, g, a);
}

spcg_status pass_gram_iter(spcg_ctx* c, const PassGeom& g, int pp, int gp, int start, int check,
                           double tau) {
  PassArgs a{};
  a.mode = PASS_ITER;
  a.z = c->pb.z;
  a.p_prev = c->pb.p[pp];
  a.p_next = c->pb.p[pp ^ 1];
  a.dots_gz = c->pb.dots_gz;
  a.dots_rb = c->pb.dots_rb;
  a.n_dots = c->pb.n_ds;
  a.gp = gp;
  a.start = start;
  a.check = check;
  a.tau = tau;
  return launch_pass(c, g, a);
}

spcg_status launch_reduce(spcg_ctx* c, double* out, const double* dotvec) {
  const int d = c->d;
  const int nr = (d + 31) / 32;
  k_reduce<<<nr, 256, 0, c->stream>>>(c->pb.partials, c->pb.last_grid, c->pb.ldp, d, out, dotvec,
                                      c->pb.dots_pw, c->scal);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 1;
  return SPCG_OK;
}

// CTAs of k_dspace: spcg_opts.dspace_ctas when set, else about eight columns
// (and rows) per CTA; at most one per SM and one per column.  (One CTA with R
// and R^{-1} staged in shared memory and no grid barrier was slower at every
// d measured, 40 to 200: the spread CTAs overlap more of the loads.)
int dspace_grid(const spcg_ctx* c) {
  int g = c->opts.dspace_ctas > 0 ? c->opts.dspace_ctas : (c->d + 7) / 8;
  if (g > c->num_sms) g = c->num_sms;
  if (g > c->d) g = c->d;
  return g < 1 ? 1 : g;
}

spcg_status launch_dspace(spcg_ctx* c, int iter, int cur, int pp, int gp, double* beta) {
  DspaceArgs a{};
  a.d = c->d;
  a.iter = iter;
  a.partials = c->pb.partials;
  a.nb = c->pb.last_grid;
  a.ldp = c->pb.ldp;
  a.R = c->sk.R;
  a.Rinv = c->sk.Rinv;
  a.RinvT = c->sk.RinvT;
  a.g_cur = c->pb.g[cur];
  a.g_nxt = c->pb.g[cur ^ 1];
  a.w = c->pb.w;
  a.p = c->pb.p[pp];
  a.beta = beta;
  a.u = c->pb.u;
  a.z = c->pb.z;
  a.dots_pw = c->pb.dots_pw;
  a.dots_gz = c->pb.dots_gz;
  a.dots_rb = c->pb.dots_rb;
  a.gp = gp;
  a.scal = c->scal;
  a.bar = c->sk.qr_bar;
  a.spin = c->opts.spin_budget > 0 ? c->opts.spin_budget : (1ll << 31);
  const size_t smem = (size_t)3 * c->d * sizeof(double);
  void* args[] = {&a};
  SPCG_CK(cudaLaunchCooperativeKernel((const void*)k_dspace, dim3(c->pb.n_ds), dim3(kDsThreads),
                                      args, smem, c->stream));
  c->n_launch += 1;
  return SPCG_OK;
}

spcg_status launch_check(spcg_ctx* c, double tau) {
  k_check<<<1, 32, 0, c->stream>>>(c->pb.dots_gz, c->pb.dots_rb, c->pb.n_ds, tau, c->scal);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 1;
  return SPCG_OK;
}

// Before a loop of passes: clear the stopping flag and the iteration count
// but keep a device error of earlier work.
spcg_status launch_reset_loop(spcg_ctx* c) {
  k_reset<<<1, 1, 0, c->stream>>>(c->scal, 0, c->sk.qr_bar);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 1;
  return SPCG_OK;
}

spcg_status launch_reset_flags(spcg_ctx* c) {
  k_reset<<<1, 1, 0, c->stream>>>(c->scal, 1, c->sk.qr_bar);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 1;
  return SPCG_OK;
}

}  // namespace spcg

namespace spcg {

// The fused pass (plain mode) and the partial-sum reduction with scratch
// that the caller provides: `partials` holds grid x ldp doubles and `scal`
// one DevScalars whose status and done words the caller has cleared.
template <int NI>
static spcg_status launch_gram_scratch_ni(const PassGeom& g, const PassArgs& a, int grid,
                                          cudaStream_t st) {
  SPCG_CK(cudaFuncSetAttribute(k_pass<double, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)g.smem_bytes));
  k_pass<double, NI><<<grid, PassCfg<NI>::THREADS, g.smem_bytes, st>>>(g.tmap, a);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

spcg_status launch_gram_with_scratch(const PassGeom& g, const double* p, double* w,
                                     double* partials, int ldp, int grid, DevScalars* scal,
                                     cudaStream_t st) {
  PassArgs a{};
  a.mode = PASS_PLAIN;
  a.vec = p;
  a.m = g.m;
  a.d = g.d;
  a.nbox = g.nbox;
  a.boxc = g.boxc;
  a.tm = g.tm;
  a.ntiles = g.ntiles;
  a.stages = g.stages;
  a.tx_bytes = (uint32_t)((size_t)g.nbox * g.boxc * g.tm * 8);
  a.slot_elems = (uint32_t)(g.stage_bytes / g.nbox / 8);
  a.stage_elems = (uint32_t)(g.stage_bytes / 8);
  a.region_bytes = (uint32_t)g.region_bytes;
  a.partials = partials;
  a.ldp = ldp;
  a.scal = scal;
  a.spin = 1ll << 31;
  spcg_status s;
  switch (ni_for(g.d)) {
    case 1: s = launch_gram_scratch_ni<1>(g, a, grid, st); break;
    case 2: s = launch_gram_scratch_ni<2>(g, a, grid, st); break;
    case 4: s = launch_gram_scratch_ni<4>(g, a, grid, st); break;
    case 8: s = launch_gram_scratch_ni<8>(g, a, grid, st); break;
    case 16: s = launch_gram_scratch_ni<16>(g, a, grid, st); break;
    case 32: s = launch_gram_scratch_ni<32>(g, a, grid, st); break;
    default: return SPCG_E_INVALID_ARG;
  }
  if (s != SPCG_OK) return s;
  k_reduce<<<(g.d + 31) / 32, 256, 0, st>>>(partials, grid, ldp, g.d, w, nullptr, nullptr, scal);
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

}  // namespace spcg

namespace spcg {

// Features of the schedule model after stage 1: the condition estimate
// max R_ii / min R_ii of the preconditioner and the share of b_1 that the
// stage-1 iterate leaves unexplained, ||b_1 - A_1 beta||^2 / ||b_1||^2 (a
// noise estimate: sigma^2 (m_1 - d) / ||b_1||^2 at the sketched solution).
template <typename T>
__global__ void __launch_bounds__(256) k_feat_resid(const T* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ b, int64_t m, int d,
                                                    const double* __restrict__ beta,
                                                    double* __restrict__ part) {
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double r2 = 0.0, b2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < m; i += (int64_t)gridDim.x * 8) {
    double t = 0.0;
    for (int j = lane; j < d; j += 32) t = fma((double)PassElem<T>::load(A[i * lda + j]), beta[j], t);
    t = warp_allsum(t);
    const double r = b[i] - t;
    r2 = fma(r, r, r2);
    b2 = fma(b[i], b[i], b2);
  }
  if (lane == 0) {
    red[0][warp] = r2;
    red[1][warp] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < 8; ++w) {
      x += red[0][w];
      y += red[1][w];
    }
    part[2 * blockIdx.x] = x;
    part[2 * blockIdx.x + 1] = y;
  }
}

__global__ void k_feat_final(const double* __restrict__ part, int nb, const double* __restrict__ R,
                             int d, float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double x = 0.0, y = 0.0;
  for (int i = 0; i < nb; ++i) {
    x += part[2 * i];
    y += part[2 * i + 1];
  }
  double mx = 0.0, mn = INFINITY;
  for (int i = 0; i < d; ++i) {
    const double v = fabs(R[(size_t)i * d + i]);
    mx = fmax(mx, v);
    mn = fmin(mn, v);
  }
  out[0] = (float)log10(mx / mn);
  out[1] = (float)log10(fmax(x, 1e-300) / fmax(y, 1e-300));
}

spcg_status launch_features(spcg_ctx* c, const double* beta, float* dev_out2) {
  const Sketch& s = c->sk;
  const int64_t m1 = s.sched.m[0];
  const int nb = 128;
  if (s.mixed)
    k_feat_resid<__nv_bfloat16><<<nb, 256, 0, c->stream>>>(
        reinterpret_cast<const __nv_bfloat16*>(s.AK16), s.ldak16, s.bK, m1, c->d, beta,
        c->feat_part);
  else
    k_feat_resid<double><<<nb, 256, 0, c->stream>>>(s.AK, s.ldak, s.bK, m1, c->d, beta,
                                                     c->feat_part);
  SPCG_CK(cudaGetLastError());
  k_feat_final<<<1, 32, 0, c->stream>>>(c->feat_part, nb, s.R, c->d, dev_out2);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 2;
  return SPCG_OK;
}

}  // namespace spcg

namespace spcg {

// ---------------------------------------------------------------------------
// The fused pass over the FP32 split X = Xh + Xl (|X - Xh - Xl| <= 2^-48 |X|)
// in double-FP32 arithmetic: products by TwoProd (FMA), sums by TwoSum, the
// direction (or beta) and b split into FP32 pairs.  Every FP64 value of X is
// read as 8 bytes of FP32 pairs, so the pass streams at memory speed instead
// of the FP64 pipe's rate, with an error near 2^-44 relative instead of 2^-53.
// The mixed path takes every trusted gradient X^T (Y - X beta) from it, and,
// when the condition estimate says that FP32 rows would perturb the
// preconditioned operator too much, the Stage II iterations as well.  Modes
// as k_pass (PLAIN, ITER with the same fused prologue, RESID).
// ---------------------------------------------------------------------------
// The error-free transformations use the _rn intrinsics on purpose: they are
// never contracted into an FMA.  A contraction such as s = fma(x, y, a) for
// s = a + x*y would fold the product's rounding error into s while the error
// term still adds it back, counting it twice and leaving FP32-level accuracy.
__device__ __forceinline__ void ts(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Consumer warps of the pair pass: 15 for every width (the dependent TwoSum
// chains need the warps to hide their latency; 15 consumers plus the producer
// make 512 threads, which leaves 128 registers a thread).  Wide rows (NI = 32)
// keep the direction in shared memory instead of registers to fit.  (15
// instead of 12 consumers made rows of 128-512 columns 5-9 % faster.)
template <int NI>
struct DfCfg {
  static constexpr int C = 15;
  static constexpr int THREADS = 32 * (C + 1);
  static constexpr bool PREG = NI <= 16;     // direction pair in registers
  static constexpr bool XCACHE = NI <= 16;   // row kept in registers between the two products
};
constexpr int kDfMaxConsumers = 15;

template <int NI>
__global__ void __launch_bounds__(DfCfg<NI>::THREADS, 1)
    k_pass_df(const __grid_constant__ CUtensorMap tmh, const __grid_constant__ CUtensorMap tml,
              const PassArgs a) {
  constexpr int KC = DfCfg<NI>::C;
  constexpr bool PREG = DfCfg<NI>::PREG;
  // lanes own runs of V = 4 consecutive columns (one float4 of each half)
  constexpr int V = 4;
  constexpr int NG = (NI * 32 + 32 * V - 1) / (32 * V);
  constexpr int RS = NG * 32 * V;
  constexpr bool XCACHE = DfCfg<NI>::XCACHE;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_addr = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((128u - (base_addr & 127u)) & 127u);
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.region_bytes);
  uint64_t* empty = full + kMaxStages;
  float* vh_s = reinterpret_cast<float*>(empty + kMaxStages);
  float* vl_s = vh_s + RS;
  __shared__ int s_abort;
  __shared__ double s_scal[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (a.scal->status != 0 || a.scal->done > (a.mode == PASS_RESID ? 1 : 0)) return;   // as k_pass
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], KC);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  double ratio = 0.0;
  if (a.mode == PASS_ITER && !iter_prologue(a, s_scal, ratio)) return;
  for (int j = tid; j < RS; j += blockDim.x) {
    double v = 0.0;
    if (j < a.d) {
      if (a.mode == PASS_ITER) {
        v = a.z[j] + ratio * a.p_prev[j];
        if (blockIdx.x == 0) a.p_next[j] = v;
      } else {
        v = a.vec[j];
      }
    }
    const float h = (float)v;
    vh_s[j] = h;
    vl_s[j] = (float)(v - (double)h);
  }
  __syncthreads();
  const int my_tiles = (blockIdx.x < a.ntiles) ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  float wh[NG][V], wl[NG][V];   // w = sum of t x over this CTA's rows, as (sum, error)
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int v = 0; v < V; ++v) wh[g][v] = wl[g][v] = 0.f;
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      const uint64_t pol = l2_evict_first_policy();
      for (int k = 0; k < my_tiles; ++k) {
        const int s = k % a.stages;
        if (k >= a.stages && !mbar_wait_bounded(&empty[s], ((k / a.stages) - 1) & 1, a.spin)) {
          atomicExch(&a.scal->status, DEV_TIMEOUT);
          s_abort = 1;
          break;
        }
        if (*(volatile int*)&s_abort) break;
        issued = k + 1;
        const int tile = blockIdx.x + k * gridDim.x;
        mbar_expect_tx(&full[s], a.tx_bytes);
        float* dst = tiles + (size_t)s * a.stage_elems;
        for (int bx = 0; bx < a.nbox; ++bx) {
          tma_load_2d(dst + (size_t)bx * a.slot_elems, &tmh, bx * a.boxc, tile * a.tm, &full[s],
                      pol);
          tma_load_2d(dst + (size_t)(a.nbox + bx) * a.slot_elems, &tml, bx * a.boxc, tile * a.tm,
                      &full[s], pol);
        }
      }
    }
  } else {
    const int cw = warp - 1;
    // Rows up to 512 wide (BF): lanes whose columns lie past d read the row's
    // first columns instead; the direction is zero there, so the row products
    // are unchanged, and their column sums are never written, so the row
    // loops have no branch (6-8 % faster).  Wider rows skip those columns
    // with a branch: without it their 128 registers spill.
    constexpr bool BF = NI <= 16;
    int off[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int c0 = g * 32 * V + lane * V;
      off[g] = (c0 < a.d) ? (c0 / a.boxc) * (int)a.slot_elems + (c0 % a.boxc) : (BF ? 0 : -1);
    }
    float ph[PREG ? NG : 1][V], pl[PREG ? NG : 1][V];
    if constexpr (PREG) {
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          ph[g][v] = vh_s[g * 32 * V + lane * V + v];
          pl[g][v] = vl_s[g * 32 * V + lane * V + v];
        }
    }
    const int lo_off = a.nbox * (int)a.slot_elems;
    for (int k = 0; k < my_tiles; ++k) {
      const int s = k % a.stages;
      if (!mbar_wait_bounded(&full[s], (k / a.stages) & 1, a.spin)) {
        atomicExch(&a.scal->status, DEV_TIMEOUT);
        s_abort = 1;
        break;
      }
      const int tile = blockIdx.x + k * gridDim.x;
      const int64_t row0 = (int64_t)tile * a.tm;
      const float* st = tiles + (size_t)s * a.stage_elems;
      const int r0 = (int)(((int64_t)cw - (int64_t)k * a.tm) % KC + KC) % KC;   // as in k_pass
      for (int rr = r0; rr < a.tm; rr += KC) {
        if (row0 + rr >= a.m) break;
        const float* rh = st + rr * a.boxc;
        const float* rl = rh + lo_off;
        float xh[XCACHE ? NG : 1][V], xl[XCACHE ? NG : 1][V];
        float sh = 0.f, sl = 0.f;   // x . v in double-FP32
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (!BF && off[g] < 0) continue;
          const float4 h4 = *reinterpret_cast<const float4*>(rh + off[g]);
          const float4 l4 = *reinterpret_cast<const float4*>(rl + off[g]);
          const float xa[V] = {h4.x, h4.y, h4.z, h4.w}, xb[V] = {l4.x, l4.y, l4.z, l4.w};
          float qh[V], ql[V];
          if constexpr (PREG) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
              qh[v] = ph[PREG ? g : 0][v];
              ql[v] = pl[PREG ? g : 0][v];
            }
          } else {
            const float4 a4 = *reinterpret_cast<const float4*>(vh_s + g * 32 * V + lane * V);
            const float4 b4 = *reinterpret_cast<const float4*>(vl_s + g * 32 * V + lane * V);
            qh[0] = a4.x; qh[1] = a4.y; qh[2] = a4.z; qh[3] = a4.w;
            ql[0] = b4.x; ql[1] = b4.y; ql[2] = b4.z; ql[3] = b4.w;
          }
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float pr = __fmul_rn(xa[v], qh[v]);
            const float pe = fmaf(xa[v], qh[v], -pr);
            float s2, se;
            ts(sh, pr, s2, se);
            sh = s2;
            sl += pe + se + fmaf(xa[v], ql[v], xb[v] * qh[v]);
            if constexpr (XCACHE) {
              xh[g][v] = xa[v];
              xl[g][v] = xb[v];
            }
          }
        }
        // Butterfly all-reduce of the pair.  Both partners must end with the
        // same bits: sh + oh and sl + ol are commutative, and se is the exact
        // error either way.  (sl += ol + se would round differently in the two
        // lanes; with cancellation sl is not small against sh, and lanes would
        // then scale their columns by slightly different t, an error that the
        // stopping metric amplifies by ||D R^{-1}||.)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
          const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
          float s2, se;
          ts(sh, oh, s2, se);
          sh = s2;
          sl = __fadd_rn(__fadd_rn(sl, ol), se);
        }
        // t = x . v, or b - x . beta, as a normalised pair (th, tl)
        float th, tl;
        if (a.mode == PASS_RESID) {
          const double bv = a.b[row0 + rr];
          const float b_h = (float)bv, b_l = (float)(bv - (double)b_h);
          ts(b_h, -sh, th, tl);
          tl += b_l - sl;
        } else {
          th = sh;
          tl = sl;
        }
        {
          float s2, se;
          ts(th, tl, s2, se);
          th = s2;
          tl = se;
        }
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (!BF && off[g] < 0) continue;
          float xa[V], xb[V];
          if constexpr (XCACHE) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
              xa[v] = xh[g][v];
              xb[v] = xl[g][v];
            }
          } else {
            const float4 h4 = *reinterpret_cast<const float4*>(rh + off[g]);
            const float4 l4 = *reinterpret_cast<const float4*>(rl + off[g]);
            xa[0] = h4.x; xa[1] = h4.y; xa[2] = h4.z; xa[3] = h4.w;
            xb[0] = l4.x; xb[1] = l4.y; xb[2] = l4.z; xb[3] = l4.w;
          }
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float pr = __fmul_rn(th, xa[v]);
            const float pe = fmaf(th, xa[v], -pr);
            float s2, se;
            ts(wh[g][v], pr, s2, se);
            wh[g][v] = s2;
            wl[g][v] += pe + se + fmaf(th, xb[v], tl * xa[v]);
          }
        }
      }
      // Renormalise the pairs every few tiles: wl collects one TwoSum error
      // per row and would otherwise grow with the rows a lane sums, and its
      // own FP32 rounding with it.
      if ((k & 7) == 7) {
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            float s2, se;
            ts(wh[g][v], wl[g][v], s2, se);
            wh[g][v] = s2;
            wl[g][v] = se;
          }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();
  if (s_abort && tid == 0) {
    const int first = issued > a.stages ? issued - a.stages : 0;
    for (int k = first; k < issued; ++k)
      (void)mbar_wait_bounded(&full[k % a.stages], (k / a.stages) & 1, 1ll << 31);
  }
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem);   // KC x RS, reuses the staging region
  if (warp > 0) {
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int v = 0; v < V; ++v)
        red[(size_t)(warp - 1) * RS + g * 32 * V + lane * V + v] =
            (double)wh[g][v] + (double)wl[g][v];
  }
  __syncthreads();
  for (int j = tid; j < a.d; j += blockDim.x) {
    double sum = 0.0;
    for (int w = 0; w < KC; ++w) sum += red[(size_t)w * RS + j];
    a.partials[(size_t)blockIdx.x * a.ldp + j] = sum;
  }
}

// Geometry of the hi/lo pair pass: FP32 boxes for both halves in one stage.
spcg_status make_pass_geom_df(const float* Xh, const float* Xl, int64_t m, int d, int64_t lda,
                              PassGeom* g, CUtensorMap* tml) {
  SPCG_TRY(make_pass_geom_t(Xl, m, d, lda, DT_F32, g));
  *tml = g->tmap;
  PassGeom h;
  // half the rows per tile: each stage carries both halves
  SPCG_TRY(make_pass_geom_t(Xh, m, d, lda, DT_F32, &h));
  int tm = h.tm > 1 ? h.tm / 2 : 1;
  if (tm > 8) tm &= ~7;
  const int bc = h.boxc;
  EncodeTiledFn enc = get_encode();
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)(lda * 4)};
  cuuint32_t box[2] = {(cuuint32_t)bc, (cuuint32_t)tm};
  cuuint32_t es[2] = {1, 1};
  CUresult r1 = enc(&h.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Xh), dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = enc(tml, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Xl), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) return SPCG_E_CUDA;
  h.tm = tm;
  h.ntiles = (int)((m + tm - 1) / tm);
  const size_t slot = (((size_t)tm * bc * 4) + 127) & ~(size_t)127;
  const size_t stage = slot * h.nbox * 2;
  int stages = (int)((192 * 1024) / stage);
  if (stages > kMaxStages) stages = kMaxStages;
  if (stages < 2) stages = 2;
  h.stages = stages;
  h.stage_bytes = stage;
  const size_t ni32 = (size_t)ni_for(d) * 32;
  const size_t cover = ni32 > 256 ? ni32 : 256;   // RS of k_pass_df is at most this
  size_t red = (size_t)kDfMaxConsumers * cover * 8;
  size_t tiles = stage * stages;
  if (tiles < red) tiles = red;
  h.region_bytes = tiles;
  h.smem_bytes = 128 + tiles + 2 * kMaxStages * 8 + 2 * cover * 4;
  h.dtype = DT_F32;
  h.esize = 8;   // algorithmic bytes per element (the pair)
  *g = h;
  return SPCG_OK;
}

template <int NI>
static spcg_status launch_df_ni(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml,
                                const PassArgs& a, int grid) {
  SPCG_CK(cudaFuncSetAttribute(k_pass_df<NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)g.smem_bytes));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->opts.profile) SPCG_TRY(prof_events(c, &e0, &e1, OP_PAIR));
  if (e0) SPCG_CK(cudaEventRecord(e0, c->stream));
  k_pass_df<NI><<<grid, DfCfg<NI>::THREADS, g.smem_bytes, c->stream>>>(g.tmap, tml, a);
  SPCG_CK(cudaGetLastError());
  if (e1) SPCG_CK(cudaEventRecord(e1, c->stream));
  c->n_launch += 1;
  c->n_pass += 1;
  c->pass_bytes += (uint64_t)g.m * g.d * 8;
  c->n_pass_op[OP_PAIR] += 1;
  c->pass_bytes_op[OP_PAIR] += (uint64_t)g.m * g.d * 8;
  return SPCG_OK;
}

static spcg_status launch_pass_df(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml,
                                  PassArgs a) {
  int grid = c->pb.grid;
  if (grid > g.ntiles) grid = g.ntiles;
  if (grid < 1) grid = 1;
  a.m = g.m;
  a.d = g.d;
  a.nbox = g.nbox;
  a.boxc = g.boxc;
  a.tm = g.tm;
  a.ntiles = g.ntiles;
  a.stages = g.stages;
  a.tx_bytes = (uint32_t)((size_t)2 * g.nbox * g.boxc * g.tm * 4);
  a.slot_elems = (uint32_t)(g.stage_bytes / (2 * g.nbox) / 4);
  a.stage_elems = (uint32_t)(g.stage_bytes / 4);
  a.region_bytes = (uint32_t)g.region_bytes;
  a.partials = c->pb.partials;
  a.ldp = c->pb.ldp;
  a.scal = c->scal;
  a.spin = c->opts.spin_budget > 0 ? c->opts.spin_budget : (1ll << 31);
  c->pb.last_grid = grid;
  switch (ni_for(g.d)) {
    case 1: return launch_df_ni<1>(c, g, tml, a, grid);
    case 2: return launch_df_ni<2>(c, g, tml, a, grid);
    case 4: return launch_df_ni<4>(c, g, tml, a, grid);
    case 8: return launch_df_ni<8>(c, g, tml, a, grid);
    case 16: return launch_df_ni<16>(c, g, tml, a, grid);
    case 32: return launch_df_ni<32>(c, g, tml, a, grid);
    default: return SPCG_E_INVALID_ARG;
  }
}

spcg_status pass_resid_df(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml,
                          const double* b, const double* x) {
  PassArgs a{};
  a.mode = PASS_RESID;
  a.vec = x;
  a.b = b;
  return launch_pass_df(c, g, tml, a);
}

spcg_status pass_gram_plain_df(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml,
                               const double* p) {
  PassArgs a{};
  a.mode = PASS_PLAIN;
  a.vec = p;
  return launch_pass_df(c, g, tml, a);
}

spcg_status pass_gram_iter_df(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml, int pp,
                              int gp, int start, int check, double tau) {
  PassArgs a{};
  a.mode = PASS_ITER;
  a.z = c->pb.z;
  a.p_prev = c->pb.p[pp];
  a.p_next = c->pb.p[pp ^ 1];
  a.dots_gz = c->pb.dots_gz;
  a.dots_rb = c->pb.dots_rb;
  a.n_dots = c->pb.n_ds;
  a.gp = gp;
  a.start = start;
  a.check = check;
  a.tau = tau;
  return launch_pass_df(c, g, tml, a);
}

}  // namespace spcg
