// The preconditioner factor (Sec. 2.2; Sec. 4 applies H-hat through a QR):
// H-hat = (S-hat X)^T (S-hat X) = R^T R with R from a Householder QR of the
// r x d sketch S-hat X, then R^{-1} and R^{-T} for the two triangular
// products z = R^{-1} (R^{-T} g) of every PCG iteration.  FP64 throughout:
// at kappa = 1e8 the sketch must be factored well below 1/kappa relative
// error.
//
// Main path, k_qr_coop: blocked Householder QR with the compact WY form
// (H_0 ... H_{b-1} = I - V T V^T) in ONE cooperative launch, one CTA per SM
// (fewer for small r), every CTA owning a contiguous block of rows.
//   Panel of b = 32 columns, factored by the first GP CTAs (about 48 rows
//   each): every panel CTA keeps its rows of the panel in shared memory.
//   Column step j needs one reduction over the panel CTAs of 2b numbers: the
//   column's squared norm below the diagonal, its dot products with the
//   other panel columns below the diagonal, and the panel's values on the
//   diagonal row.  From these sums every CTA derives alpha, the reflector's
//   first entry v_0, v^T a_i for the later columns (so each CTA updates its
//   own rows without a second reduction) and V^T v_j for the column j of T.
//   Trailing matrix C, on all CTAs (rows of V and T read back from global
//   memory): W = V^T C (per-CTA partials over its rows), then W' = T^T W
//   (columns split over CTAs), then C -= V W' (own rows).
//   A grid barrier separates the phases; its wait is bounded (on expiry the
//   device status becomes TIMEOUT and every CTA leaves at its next barrier).
//   Partial sums are added in CTA order, so the result is reproducible.
// Fallback for r too large for the panel rows to fit in shared memory: one
// launch per column (k_householder_cluster / k_householder_step below).
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

// ---------------------------------------------------------------------------
// Cooperative blocked QR
// ---------------------------------------------------------------------------
constexpr int QB = kQrPanel;           // panel width b
constexpr int QSL = 2 * QB;            // reduction slots of a column step
constexpr int QT = 256;                // threads per CTA
constexpr int QLD = QB + 1;            // row stride of the panel slice in shared memory
constexpr int QCOLB = 8;               // columns per batch in the T^T W phase
constexpr int QUNR = 8;                // independent loads in flight per thread in the sums
constexpr int QRED = 16;               // the same in a column step's read-back (one round for
                                       // up to 64 panel CTAs)
constexpr int kQrPanelRows = 48;       // rows per panel CTA (default panel group size)
constexpr int QRR = 4;                 // rows per step of the trailing-update loops
constexpr int kQrLaPanelWork = 30000;  // look-ahead QR: panel CTAs = this / d (default)
constexpr int kQrLaMinD = 256;         // look-ahead QR from this many columns (eight panels)

struct QrCoopArgs {
  double* A;           // r x d column-major (ld = r), reduced in place
  int64_t r;
  int d;
  int gp;              // CTAs that factor the panels (the first gp of the grid)
  int chunk_max;       // rows of the largest row slice a CTA holds in shared memory
  double* Tg;          // QB x QB: T of the current panel, for the trailing update
  double* Rdiag;       // d: alpha_k (R_kk before the sign fix)
  double* vdiag;       // d: v_0 of reflector k
  double* red;         // 2 x G x QSL
  double* Wp;          // G x QB x d
  double* Wt;          // QB x d
  unsigned* bar;       // grid barrier (kBarWords, zero at launch)
  unsigned* bar2;      // barrier of the panel CTAs (kBarWords, zero at launch)
  int* status;
  long long spin;
};

__global__ void __launch_bounds__(QT, 1) k_qr_coop(const QrCoopArgs a) {
  extern __shared__ double qsm[];
  double* P = qsm;                                   // chunk_max x QLD: panel rows, then V
  double* T = P + (size_t)a.chunk_max * QLD;         // QB x QB, T[i * QB + j]
  double* tot = T + QB * QB;                         // QSL summed slots
  double* comb = tot + QSL;                          // 4 x QSL partial slots
  double* pv0 = comb + 4 * QSL;                      // QB: v_0 of the panel's reflectors
  double* wsm = pv0 + QB;                            // QCOLB x QB: W columns of one batch
  __shared__ int s_fail;
  __shared__ double sc[2];   // v_0 and tau of the current reflector
  __shared__ double fcol[QB];  // tau v^T a_i of the later panel columns
  const int tid = threadIdx.x, G = gridDim.x, q = blockIdx.x;
  if (tid == 0) s_fail = 0;
  if (*a.status != 0) return;                        // uniform: set before this launch
  __syncthreads();
  const int64_t r = a.r;
  const int d = a.d;
  int step = 0;
  const int GP = a.gp;
  for (int k0 = 0; k0 < d; k0 += QB) {
    const int bw = d - k0 < QB ? d - k0 : QB;
    const int64_t mp = r - k0;
    if (q < GP) {
      // ---- panel: the first GP CTAs, each a block of rows in shared memory ----
      const int64_t chunk = (mp + GP - 1) / GP;
      const int64_t lo = k0 + (int64_t)q * chunk;
      const int64_t hi = lo + chunk < r ? lo + chunk : r;
      const int nr = hi > lo ? (int)(hi - lo) : 0;
      for (int e = tid; e < nr * QB; e += QT) {
        const int j = e / nr, ri = e % nr;
        P[ri * QLD + j] = j < bw ? a.A[(int64_t)(k0 + j) * r + lo + ri] : 0.0;
      }
      for (int e = tid; e < QB * QB; e += QT) T[e] = 0.0;
      __syncthreads();
      for (int j = 0; j < bw; ++j, ++step) {
        const int64_t diag = k0 + j;
        const int own = (diag >= lo && diag < hi) ? (int)(diag - lo) : -1;
        // slot s < QB: sum over own rows below the diagonal of P[., s] P[., j];
        // slot QB + s: the diagonal row's value of column s (owner only)
        {
          const int sl = tid % QSL, grp = tid / QSL;   // 4 row groups
          double acc = 0.0;
          if (sl < QB) {
            if (sl < bw) {
              int ri0 = (int)(diag + 1 - lo);
              if (ri0 < 0) ri0 = 0;
              for (int ri = ri0 + grp; ri < nr; ri += 4) acc = fma(P[ri * QLD + sl], P[ri * QLD + j], acc);
            }
          } else if (grp == 0 && own >= 0 && sl - QB < bw) {
            acc = P[own * QLD + (sl - QB)];
          }
          comb[grp * QSL + sl] = acc;
        }
        __syncthreads();
        double* red = a.red + (size_t)(step & 1) * G * QSL;
        if (tid < QSL)
          red[(size_t)q * QSL + tid] =
              ((comb[tid] + comb[QSL + tid]) + comb[2 * QSL + tid]) + comb[3 * QSL + tid];
        if (!group_sync_bounded(a.bar2, (unsigned)GP, a.status, a.spin, &s_fail)) return;
        {
          // the same sums in every panel CTA: slot sl over CTAs g, g + 4, ...
          // then the four quarter sums in order
          const int sl = tid % QSL, grp = tid / QSL;
          double acc = 0.0;
          for (int g0 = grp; g0 < GP; g0 += 4 * QRED) {   // loads first, then the sums in order
            double v[QRED];
#pragma unroll
            for (int k = 0; k < QRED; ++k) {
              const int g = g0 + 4 * k;
              v[k] = g < GP ? red[(size_t)g * QSL + sl] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < QRED; ++k) acc += v[k];
          }
          comb[grp * QSL + sl] = acc;
        }
        __syncthreads();
        if (tid < QSL) tot[tid] = ((comb[tid] + comb[QSL + tid]) + comb[2 * QSL + tid]) + comb[3 * QSL + tid];
        __syncthreads();
        if (tid == 0) {   // the reflector's scalars, once per CTA (FP64 sqrt and divide are slow)
          const double s2 = tot[j], x0 = tot[QB + j];
          const double normx = sqrt(fma(x0, x0, s2));
          const double alpha = (x0 >= 0.0) ? -normx : normx;
          const double v0 = x0 - alpha;
          const double vv = fma(v0, v0, s2);
          pv0[j] = v0;
          sc[0] = v0;
          sc[1] = vv > 0.0 ? 2.0 / vv : 0.0;
          if (q == 0) {
            a.Rdiag[diag] = alpha;
            a.vdiag[diag] = v0;
          }
        }
        __syncthreads();
        const double v0 = sc[0], tau = sc[1];
        // T(0:j, j) = -tau T(0:j, 0:j) V(:, 0:j)^T v_j, with
        // v_l^T v_j = (below the diagonal) + v_l(diag) v_0
        if (tid < j) {   // four independent partial sums over l
          double s4[4] = {0.0, 0.0, 0.0, 0.0};
          int l = tid;
          for (; l + 3 < j; l += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              s4[u] = fma(T[tid * QB + l + u], fma(tot[QB + l + u], v0, tot[l + u]), s4[u]);
          }
          for (; l < j; ++l) s4[0] = fma(T[tid * QB + l], fma(tot[QB + l], v0, tot[l]), s4[0]);
          T[tid * QB + j] = -tau * ((s4[0] + s4[1]) + (s4[2] + s4[3]));
        } else if (tid == j) {
          T[j * QB + j] = tau;
        }
        // later panel columns, own rows: a_i -= f_i v with f_i = tau (v^T a_i),
        // formed once per column (FP64 operations are the scarce resource here)
        const int ncl = bw - j - 1;
        if (tid > j && tid < bw) fcol[tid] = tau * fma(v0, tot[QB + tid], tot[tid]);
        __syncthreads();
        for (int e = tid; e < nr * ncl; e += QT) {
          const int i = j + 1 + e / nr, ri = e % nr;
          const int64_t row = lo + ri;
          if (row < diag) continue;
          const double vr = (row == diag) ? v0 : P[ri * QLD + j];
          P[ri * QLD + i] = fma(-fcol[i], vr, P[ri * QLD + i]);
        }
        __syncthreads();
      }
      // write the panel back (R above the diagonal, v below it, x_0 on it);
      // the panel's T goes to global memory for the trailing update
      for (int e = tid; e < nr * bw; e += QT) {
        const int j = e / nr, ri = e % nr;
        a.A[(int64_t)(k0 + j) * r + lo + ri] = P[ri * QLD + j];
      }
      if (q == 0)
        for (int e = tid; e < QB * QB; e += QT) a.Tg[e] = T[e];
    } else {
      step += bw;   // keep the reduction buffers' parity in step with the panel CTAs
    }
    const int nt = d - k0 - bw;   // trailing columns
    if (nt <= 0) break;           // last panel: nothing to update
    if (!grid_sync_bounded(a.bar, a.status, a.spin, &s_fail)) return;
    // ---- trailing update on all CTAs: this CTA's rows of V (0 above the
    // diagonal, v_0 on it) and T from global memory ----
    const int64_t chunk = (mp + G - 1) / G;
    const int64_t lo = k0 + (int64_t)q * chunk;
    const int64_t hi = lo + chunk < r ? lo + chunk : r;
    const int nr = hi > lo ? (int)(hi - lo) : 0;
    for (int e = tid; e < nr * QB; e += QT) {
      const int i = e / nr, ri = e % nr;
      const int64_t row = lo + ri;
      double v = 0.0;
      if (i < bw) v = row > k0 + i ? a.A[(int64_t)(k0 + i) * r + row] : (row == k0 + i ? a.vdiag[k0 + i] : 0.0);
      P[ri * QLD + i] = v;
    }
    for (int e = tid; e < QB * QB; e += QT) T[e] = a.Tg[e];
    __syncthreads();
    // W partial = V_own^T C_own (QRR rows of the column loaded at a time)
    for (int c = tid; c < nt; c += QT) {
      double w[QB];
#pragma unroll
      for (int i = 0; i < QB; ++i) w[i] = 0.0;
      const double* col = a.A + (int64_t)(k0 + bw + c) * r + lo;
      for (int ri0 = 0; ri0 < nr; ri0 += QRR) {
        double cv[QRR];
#pragma unroll
        for (int u = 0; u < QRR; ++u) cv[u] = ri0 + u < nr ? col[ri0 + u] : 0.0;
#pragma unroll
        for (int u = 0; u < QRR; ++u) {
          if (ri0 + u >= nr) break;   // uniform over the CTA
#pragma unroll
          for (int i = 0; i < QB; ++i) w[i] = fma(P[(ri0 + u) * QLD + i], cv[u], w[i]);
        }
      }
      double* dst = a.Wp + (size_t)q * QB * d + c;
#pragma unroll
      for (int i = 0; i < QB; ++i) dst[(size_t)i * d] = w[i];
    }
    if (!grid_sync_bounded(a.bar, a.status, a.spin, &s_fail)) return;
    // W = sum of the partials (CTA order), W' = T^T W for this CTA's columns
    {
      const int cs = (nt + G - 1) / G;
      const int c_lo = q * cs, c_hi = c_lo + cs < nt ? c_lo + cs : nt;
      for (int cb = c_lo; cb < c_hi; cb += QCOLB) {
        const int ncb = c_hi - cb < QCOLB ? c_hi - cb : QCOLB;
        for (int e = tid; e < ncb * QB; e += QT) {
          const int cc = e / QB, i = e % QB;
          double acc = 0.0;
          const double* src = a.Wp + (size_t)i * d + cb + cc;
          for (int g0 = 0; g0 < G; g0 += QUNR) {
            double v[QUNR];
#pragma unroll
            for (int k = 0; k < QUNR; ++k) v[k] = g0 + k < G ? src[(size_t)(g0 + k) * QB * d] : 0.0;
#pragma unroll
            for (int k = 0; k < QUNR; ++k) acc += v[k];
          }
          wsm[cc * QB + i] = acc;
        }
        __syncthreads();
        for (int e = tid; e < ncb * QB; e += QT) {
          const int cc = e / QB, i = e % QB;
          double acc = 0.0;
          for (int l = 0; l <= i; ++l) acc = fma(T[l * QB + i], wsm[cc * QB + l], acc);
          a.Wt[(size_t)i * d + cb + cc] = acc;
        }
        __syncthreads();
      }
    }
    if (!grid_sync_bounded(a.bar, a.status, a.spin, &s_fail)) return;
    // C_own -= V_own W': QRR rows at a time, so that QRR independent chains
    // of multiply-adds keep the FP64 pipe busy
    for (int c = tid; c < nt; c += QT) {
      double wt[QB];
#pragma unroll
      for (int i = 0; i < QB; ++i) wt[i] = a.Wt[(size_t)i * d + c];
      double* col = a.A + (int64_t)(k0 + bw + c) * r + lo;
      for (int ri0 = 0; ri0 < nr; ri0 += QRR) {
        double acc[QRR];
#pragma unroll
        for (int u = 0; u < QRR; ++u) acc[u] = ri0 + u < nr ? col[ri0 + u] : 0.0;
#pragma unroll
        for (int i = 0; i < QB; ++i)
#pragma unroll
          for (int u = 0; u < QRR; ++u)
            acc[u] = fma(-P[(ri0 + u < nr ? ri0 + u : 0) * QLD + i], wt[i], acc[u]);
#pragma unroll
        for (int u = 0; u < QRR; ++u)
          if (ri0 + u < nr) col[ri0 + u] = acc[u];
      }
    }
    if (!grid_sync_bounded(a.bar, a.status, a.spin, &s_fail)) return;
  }
}

// ---------------------------------------------------------------------------
// Blocked QR with look-ahead, one cooperative launch.  The grid is split in
// two groups that work at the same time on every panel p:
//   panel group (CTAs [0, GP), rows of the panel split among them): applies
//     panel p-1's reflectors to panel p's columns (W = V^T C summed over the
//     group, W' = T^T W, C -= V W'; CTA 0 also takes the 32 rows of panel
//     p-1's block, which hold R entries), then factors panel p as k_qr_coop
//     does (one group reduction per column step);
//   update group (CTAs [GP, G), rows split among them): applies panel p-1's
//     reflectors to every column right of panel p, as k_qr_coop's trailing
//     update with a barrier of its own.
// One grid barrier per panel; the latency-bound column steps of panel p run
// while the FP64-bound update of the columns right of it proceeds.  Panel T
// factors alternate between two buffers (the update group reads T_{p-1}
// while the panel group writes T_p).  (An update group that split the columns
// instead, each column's W = V^T c inside one CTA with V staged 128 rows at a
// time, was slower: the staging is latency-bound.)
// ---------------------------------------------------------------------------

struct QrLaArgs {
  double* A;           // r x d column-major (ld = r), reduced in place
  int64_t r;
  int d;
  int gp;              // CTAs of the panel group
  int chunk_max;       // largest row slice of a panel CTA
  double* Tg;          // 2 x QB x QB: T of panel p at Tg + (p & 1) QB QB
  double* Rdiag;       // d: alpha_k
  double* vdiag;       // d: v_0 of reflector k
  double* red;         // 2 x G x QSL: column-step sums of the panel group
  double* Wl;          // (GP + 1) x QB x QB: look-ahead partials, then their sum
  double* Wp;          // GU x QB x d: the update group's W partials
  double* Wt;          // QB x d: W' = T^T W of the update group
  int chunk_u;         // rows of the largest row slice of an update CTA
  unsigned* bar;       // grid barrier (zero at launch)
  unsigned* bar2;      // panel-group barrier (zero at launch)
  unsigned* bar3;      // update-group barrier (zero at launch)
  int* status;
  long long spin;
};

__global__ void __launch_bounds__(QT, 1) k_qr_la(const QrLaArgs a) {
  extern __shared__ double qsm[];
  __shared__ int s_fail;
  __shared__ double sc[2];
  __shared__ double fcol[QB];
  const int tid = threadIdx.x, G = gridDim.x, q = blockIdx.x;
  if (tid == 0) s_fail = 0;
  if (*a.status != 0) return;   // uniform: set before this launch
  __syncthreads();
  const int64_t r = a.r;
  const int d = a.d;
  const int GP = a.gp;
  const bool panel_cta = q < GP;
  // panel group layout
  double* P = qsm;                                   // chunk_max x QLD
  double* Vo = P + (size_t)a.chunk_max * QLD;        // chunk_max x QLD: V_{p-1}, own rows
  double* E = Vo + (size_t)a.chunk_max * QLD;        // QB x QLD: rows of panel p-1's block
  double* VE = E + QB * QLD;                         // QB x QLD: V_{p-1} on those rows
  double* T = VE + QB * QLD;                         // QB x QB
  double* W = T + QB * QB;                           // QB x QB
  double* tot = W + QB * QB;                         // QSL
  double* comb = tot + QSL;                          // 4 x QSL
  double* pv0 = comb + 4 * QSL;                      // QB
  int step = 0;
  for (int k0 = 0; k0 < d; k0 += QB) {
    const int p = k0 / QB;
    const int bw = d - k0 < QB ? d - k0 : QB;
    const int kp = k0 - QB;   // first column (and row) of panel p-1
    if (panel_cta) {
      const int64_t mp = r - k0;
      const int64_t chunk = (mp + GP - 1) / GP;
      const int64_t lo = k0 + (int64_t)q * chunk;
      const int64_t hi = lo + chunk < r ? lo + chunk : r;
      const int nr = hi > lo ? (int)(hi - lo) : 0;
      for (int e = tid; e < nr * QB; e += QT) {
        const int j = e / nr, ri = e % nr;
        P[ri * QLD + j] = j < bw ? a.A[(int64_t)(k0 + j) * r + lo + ri] : 0.0;
      }
      if (p > 0) {
        // ---- look-ahead: panel p-1's reflectors on panel p's columns ----
        for (int e = tid; e < nr * QB; e += QT) {   // own rows lie below panel p-1's block
          const int i = e / nr, ri = e % nr;
          Vo[ri * QLD + i] = a.A[(int64_t)(kp + i) * r + lo + ri];
        }
        if (q == 0)
          for (int e = tid; e < QB * QB; e += QT) {
            const int i = e / QB, ee = e % QB;   // row kp + ee, column i of V / j of C
            const int64_t row = kp + ee;
            VE[ee * QLD + i] = ee > i ? a.A[(int64_t)(kp + i) * r + row]
                                      : (ee == i ? a.vdiag[kp + i] : 0.0);
            E[ee * QLD + i] = i < bw ? a.A[(int64_t)(k0 + i) * r + row] : 0.0;
          }
        for (int e = tid; e < QB * QB; e += QT) T[e] = a.Tg[(size_t)((p - 1) & 1) * QB * QB + e];
        __syncthreads();
        // partial W = V^T C over own rows (thread: row i of W, four columns)
        {
          const int i = tid >> 3, j0 = (tid & 7) * 4;
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
          for (int ri = 0; ri < nr; ++ri) {
            const double v = Vo[ri * QLD + i];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(v, P[ri * QLD + j0 + u], acc[u]);
          }
          if (q == 0)
            for (int ee = 0; ee < QB; ++ee) {
              const double v = VE[ee * QLD + i];
#pragma unroll
              for (int u = 0; u < 4; ++u) acc[u] = fma(v, E[ee * QLD + j0 + u], acc[u]);
            }
          double* dst = a.Wl + (size_t)q * QB * QB + i * QB + j0;
#pragma unroll
          for (int u = 0; u < 4; ++u) dst[u] = acc[u];
        }
        if (!group_sync_bounded(a.bar2, (unsigned)GP, a.status, a.spin, &s_fail)) return;
        // W = sum of the partials in CTA order, each CTA a share of the entries
        {
          double* Wsum = a.Wl + (size_t)GP * QB * QB;
          const int per = (QB * QB + GP - 1) / GP;
          for (int e = q * per + tid; e < (q + 1) * per && e < QB * QB; e += QT) {
            double acc = 0.0;
            for (int g0 = 0; g0 < GP; g0 += QUNR) {
              double v[QUNR];
#pragma unroll
              for (int k = 0; k < QUNR; ++k)
                v[k] = g0 + k < GP ? a.Wl[(size_t)(g0 + k) * QB * QB + e] : 0.0;
#pragma unroll
              for (int k = 0; k < QUNR; ++k) acc += v[k];
            }
            Wsum[e] = acc;
          }
        }
        if (!group_sync_bounded(a.bar2, (unsigned)GP, a.status, a.spin, &s_fail)) return;
        {
          const double* Wsum = a.Wl + (size_t)GP * QB * QB;
          for (int e = tid; e < QB * QB; e += QT) W[e] = Wsum[e];
        }
        __syncthreads();
        // W' = T^T W, formed in registers and written over W
        {
          const int i = tid >> 3, j0 = (tid & 7) * 4;
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
          for (int l = 0; l <= i; ++l) {
            const double t = T[l * QB + i];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(t, W[l * QB + j0 + u], acc[u]);
          }
          __syncthreads();
#pragma unroll
          for (int u = 0; u < 4; ++u) W[i * QB + j0 + u] = acc[u];
        }
        __syncthreads();
        // C -= V W' on own rows (and CTA 0's block rows, written back now)
        for (int e = tid; e < nr * QB; e += QT) {
          const int ri = e / QB, j = e % QB;
          double acc = P[ri * QLD + j];
          for (int i = 0; i < QB; ++i) acc = fma(-Vo[ri * QLD + i], W[i * QB + j], acc);
          P[ri * QLD + j] = acc;
        }
        if (q == 0)
          for (int e = tid; e < QB * bw; e += QT) {
            const int ee = e / bw, j = e % bw;
            double acc = E[ee * QLD + j];
            for (int i = 0; i < QB; ++i) acc = fma(-VE[ee * QLD + i], W[i * QB + j], acc);
            a.A[(int64_t)(k0 + j) * r + kp + ee] = acc;
          }
      }
      for (int e = tid; e < QB * QB; e += QT) T[e] = 0.0;
      __syncthreads();
      // ---- factor panel p (as in k_qr_coop) ----
      for (int j = 0; j < bw; ++j, ++step) {
        const int64_t diag = k0 + j;
        const int own = (diag >= lo && diag < hi) ? (int)(diag - lo) : -1;
        {
          const int sl = tid % QSL, grp = tid / QSL;
          double acc = 0.0;
          if (sl < QB) {
            if (sl < bw) {
              int ri0 = (int)(diag + 1 - lo);
              if (ri0 < 0) ri0 = 0;
              for (int ri = ri0 + grp; ri < nr; ri += 4) acc = fma(P[ri * QLD + sl], P[ri * QLD + j], acc);
            }
          } else if (grp == 0 && own >= 0 && sl - QB < bw) {
            acc = P[own * QLD + (sl - QB)];
          }
          comb[grp * QSL + sl] = acc;
        }
        __syncthreads();
        double* red = a.red + (size_t)(step & 1) * G * QSL;
        if (tid < QSL)
          red[(size_t)q * QSL + tid] =
              ((comb[tid] + comb[QSL + tid]) + comb[2 * QSL + tid]) + comb[3 * QSL + tid];
        if (!group_sync_bounded(a.bar2, (unsigned)GP, a.status, a.spin, &s_fail)) return;
        {
          const int sl = tid % QSL, grp = tid / QSL;
          double acc = 0.0;
          for (int g0 = grp; g0 < GP; g0 += 4 * QRED) {
            double v[QRED];
#pragma unroll
            for (int k = 0; k < QRED; ++k) {
              const int g = g0 + 4 * k;
              v[k] = g < GP ? red[(size_t)g * QSL + sl] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < QRED; ++k) acc += v[k];
          }
          comb[grp * QSL + sl] = acc;
        }
        __syncthreads();
        if (tid < QSL) tot[tid] = ((comb[tid] + comb[QSL + tid]) + comb[2 * QSL + tid]) + comb[3 * QSL + tid];
        __syncthreads();
        if (tid == 0) {
          const double s2 = tot[j], x0 = tot[QB + j];
          const double normx = sqrt(fma(x0, x0, s2));
          const double alpha = (x0 >= 0.0) ? -normx : normx;
          const double v0 = x0 - alpha;
          const double vv = fma(v0, v0, s2);
          pv0[j] = v0;
          sc[0] = v0;
          sc[1] = vv > 0.0 ? 2.0 / vv : 0.0;
          if (q == 0) {
            a.Rdiag[diag] = alpha;
            a.vdiag[diag] = v0;
          }
        }
        __syncthreads();
        const double v0 = sc[0], tau = sc[1];
        if (tid < j) {   // four independent partial sums over l
          double s4[4] = {0.0, 0.0, 0.0, 0.0};
          int l = tid;
          for (; l + 3 < j; l += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              s4[u] = fma(T[tid * QB + l + u], fma(tot[QB + l + u], v0, tot[l + u]), s4[u]);
          }
          for (; l < j; ++l) s4[0] = fma(T[tid * QB + l], fma(tot[QB + l], v0, tot[l]), s4[0]);
          T[tid * QB + j] = -tau * ((s4[0] + s4[1]) + (s4[2] + s4[3]));
        } else if (tid == j) {
          T[j * QB + j] = tau;
        }
        const int ncl = bw - j - 1;
        if (tid > j && tid < bw) fcol[tid] = tau * fma(v0, tot[QB + tid], tot[tid]);
        __syncthreads();
        for (int e = tid; e < nr * ncl; e += QT) {
          const int i = j + 1 + e / nr, ri = e % nr;
          const int64_t row = lo + ri;
          if (row < diag) continue;
          const double vr = (row == diag) ? v0 : P[ri * QLD + j];
          P[ri * QLD + i] = fma(-fcol[i], vr, P[ri * QLD + i]);
        }
        __syncthreads();
      }
      for (int e = tid; e < nr * bw; e += QT) {
        const int j = e / nr, ri = e % nr;
        a.A[(int64_t)(k0 + j) * r + lo + ri] = P[ri * QLD + j];
      }
      if (q == 0)
        for (int e = tid; e < QB * QB; e += QT) a.Tg[(size_t)(p & 1) * QB * QB + e] = T[e];
    } else {
      step += bw;   // keep the reduction buffers' parity with the panel group
      // ---- update group: panel p-1's reflectors on the columns right of panel
      // p, rows kp .. r-1 split among the GU CTAs (as k_qr_coop's trailing
      // update, with the group's own barrier): W partials, their sum and
      // W' = T^T W by columns, then C -= V W' on own rows ----
      const int cstart = k0 + bw;
      const int nt = d - cstart;
      if (p > 0 && nt > 0) {
        const int GU = G - GP, u = q - GP;
        const int64_t mu = r - kp;
        const int64_t chunk = (mu + GU - 1) / GU;
        const int64_t lo = kp + (int64_t)u * chunk;
        const int64_t hi = lo + chunk < r ? lo + chunk : r;
        const int nr = hi > lo ? (int)(hi - lo) : 0;
        double* Pu = qsm;                              // chunk x QLD: V_{p-1}, own rows
        double* Tu = Pu + (size_t)a.chunk_u * QLD;     // QB x QB
        double* wsm = Tu + QB * QB;                    // QCOLB x QB
        for (int e = tid; e < nr * QB; e += QT) {
          const int i = e / nr, ri = e % nr;
          const int64_t row = lo + ri;
          Pu[ri * QLD + i] = row > kp + i ? a.A[(int64_t)(kp + i) * r + row]
                                          : (row == kp + i ? a.vdiag[kp + i] : 0.0);
        }
        for (int e = tid; e < QB * QB; e += QT) Tu[e] = a.Tg[(size_t)((p - 1) & 1) * QB * QB + e];
        __syncthreads();
        for (int c = tid; c < nt; c += QT) {
          double w[QB];
#pragma unroll
          for (int i = 0; i < QB; ++i) w[i] = 0.0;
          const double* col = a.A + (int64_t)(cstart + c) * r + lo;
          for (int ri0 = 0; ri0 < nr; ri0 += QRR) {
            double cv[QRR];
#pragma unroll
            for (int k = 0; k < QRR; ++k) cv[k] = ri0 + k < nr ? col[ri0 + k] : 0.0;
#pragma unroll
            for (int k = 0; k < QRR; ++k) {
              if (ri0 + k >= nr) break;   // uniform over the CTA
#pragma unroll
              for (int i = 0; i < QB; ++i) w[i] = fma(Pu[(ri0 + k) * QLD + i], cv[k], w[i]);
            }
          }
          double* dst = a.Wp + (size_t)u * QB * d + c;
#pragma unroll
          for (int i = 0; i < QB; ++i) dst[(size_t)i * d] = w[i];
        }
        if (!group_sync_bounded(a.bar3, (unsigned)GU, a.status, a.spin, &s_fail)) return;
        {
          const int cs = (nt + GU - 1) / GU;
          const int c_lo = u * cs, c_hi = c_lo + cs < nt ? c_lo + cs : nt;
          for (int cb = c_lo; cb < c_hi; cb += QCOLB) {
            const int ncb = c_hi - cb < QCOLB ? c_hi - cb : QCOLB;
            for (int e = tid; e < ncb * QB; e += QT) {
              const int cc = e / QB, i = e % QB;
              double acc = 0.0;
              const double* src = a.Wp + (size_t)i * d + cb + cc;
              for (int g0 = 0; g0 < GU; g0 += QUNR) {
                double v[QUNR];
#pragma unroll
                for (int k = 0; k < QUNR; ++k) v[k] = g0 + k < GU ? src[(size_t)(g0 + k) * QB * d] : 0.0;
#pragma unroll
                for (int k = 0; k < QUNR; ++k) acc += v[k];
              }
              wsm[cc * QB + i] = acc;
            }
            __syncthreads();
            for (int e = tid; e < ncb * QB; e += QT) {
              const int cc = e / QB, i = e % QB;
              double acc = 0.0;
              for (int l = 0; l <= i; ++l) acc = fma(Tu[l * QB + i], wsm[cc * QB + l], acc);
              a.Wt[(size_t)i * d + cb + cc] = acc;
            }
            __syncthreads();
          }
        }
        if (!group_sync_bounded(a.bar3, (unsigned)GU, a.status, a.spin, &s_fail)) return;
        for (int c = tid; c < nt; c += QT) {
          double wt[QB];
#pragma unroll
          for (int i = 0; i < QB; ++i) wt[i] = a.Wt[(size_t)i * d + c];
          double* col = a.A + (int64_t)(cstart + c) * r + lo;
          for (int ri0 = 0; ri0 < nr; ri0 += QRR) {
            double acc[QRR];
#pragma unroll
            for (int k = 0; k < QRR; ++k) acc[k] = ri0 + k < nr ? col[ri0 + k] : 0.0;
#pragma unroll
            for (int i = 0; i < QB; ++i)
#pragma unroll
              for (int k = 0; k < QRR; ++k)
                acc[k] = fma(-Pu[(ri0 + k < nr ? ri0 + k : 0) * QLD + i], wt[i], acc[k]);
#pragma unroll
            for (int k = 0; k < QRR; ++k)
              if (ri0 + k < nr) col[ri0 + k] = acc[k];
          }
        }
      }
    }
    if (k0 + bw >= d) break;   // last panel factored
    if (!grid_sync_bounded(a.bar, a.status, a.spin, &s_fail)) return;
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

// R^{-1} column by column, one warp per column j, blocked back substitution
// of R x = e_j over blocks of 32 rows, from the bottom block up:
//   - the block's 32 x 32 triangle is solved in registers: lane L holds
//     b_{kb+L} and row kb+L of the triangle; x_t = b_t / R_tt is broadcast
//     with a shuffle and the lanes above it subtract x_t R_{L t};
//   - the rows above the block then take the block's contribution,
//     b_i -= sum_t R_{i, kb+t} x_{kb+t}, with all 32 loads of a row
//     independent (no dependency chain through memory).
// Column j of R^{-1} is written as row j of R^{-T} (contiguous); R^{-1} is
// its transpose.  Columns are dealt to warps so that every CTA mixes short
// and long columns (column j costs about j^2 / 2 multiply-adds).
constexpr int TRI_WARPS = 4;

__global__ void __launch_bounds__(TRI_WARPS * 32) k_trtri_blocked(const double* __restrict__ R, int d,
                                                                 double* __restrict__ RinvT) {
  extern __shared__ double xs[];   // TRI_WARPS x d
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x + gridDim.x * warp;
  if (j >= d) return;
  double* b = xs + (size_t)warp * d;
  for (int i = lane; i <= j; i += 32) b[i] = (i == j) ? 1.0 : 0.0;
  __syncwarp();
  for (int kb = (j / 32) * 32; kb >= 0; kb -= 32) {
    const int nb = j - kb + 1 < 32 ? j - kb + 1 : 32;   // rows kb .. kb+nb-1 (<= j < d)
    double tri[32];
    const double* Rrow = R + (size_t)(kb + (lane < nb ? lane : 0)) * d + kb;
#pragma unroll
    for (int t = 0; t < 32; ++t) tri[t] = (lane < nb && t > lane && t < nb) ? Rrow[t] : 0.0;
    const double rin = lane < nb ? 1.0 / Rrow[lane] : 0.0;
    double bl = lane < nb ? b[kb + lane] : 0.0;
#pragma unroll
    for (int t = 31; t >= 0; --t) {
      if (t < nb) {   // warp-uniform
        const double xt = __shfl_sync(0xffffffffu, bl * rin, t);
        if (lane == t) bl = xt;
        else if (lane < t) bl = fma(-xt, tri[t], bl);
      }
    }
    if (lane < nb) b[kb + lane] = bl;
    __syncwarp();
    for (int i = lane; i < kb; i += 32) {
      const double* Ri = R + (size_t)i * d + kb;
      double acc = b[i];
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < nb) acc = fma(-Ri[t], b[kb + t], acc);
      b[i] = acc;
    }
    __syncwarp();
  }
  for (int i = lane; i < d; i += 32) RinvT[(size_t)j * d + i] = i <= j ? b[i] : 0.0;
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

// The grid of the cooperative QR: at least about 8 rows per CTA, at most one
// CTA per SM (the trailing updates are FP64-bound: every SM helps).
static int qr_coop_grid(int64_t r, int sms) {
  int64_t g = (r + 7) / 8;
  if (g > sms) g = sms;
  if (g < 1) g = 1;
  return (int)g;
}

static size_t qr_coop_smem(int64_t chunk_max) {
  return ((size_t)chunk_max * QLD + QB * QB + QSL + 4 * QSL + QB + QCOLB * QB) * sizeof(double);
}

static size_t qr_la_smem(int64_t chunk_max, int64_t chunk_u) {
  const size_t panel = (size_t)2 * chunk_max * QLD + 2 * QB * QLD + 2 * QB * QB + QSL + 4 * QSL + QB;
  const size_t update = (size_t)chunk_u * QLD + QB * QB + QCOLB * QB;
  return (panel > update ? panel : update) * sizeof(double);
}

// The per-column fallback (one launch per Householder step).
static spcg_status householder_by_column(spcg_ctx* c) {
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
  c->n_launch += d;
  SPCG_CK(cudaGetLastError());
  return SPCG_OK;
}

static spcg_status finish_precond(spcg_ctx* c);

// The look-ahead QR when it applies (more than one panel, an update group of
// at least one CTA, the panel rows in shared memory); false: use k_qr_coop.
static bool launch_qr_la(spcg_ctx* c, bool* launched) {
  *launched = false;
  Sketch& s = c->sk;
  const int d = c->d;
  const int64_t r = s.sched.r;
  // with fewer than eight panels there is little to overlap: k_qr_coop
  if (c->opts.qr_by_column != 0 || d < kQrLaMinD) return true;
  const int G = qr_coop_grid(r, c->num_sms);
  // panel group: about kQrLaPanelWork / d CTAs, at most half the grid (the
  // panel path shortens with more CTAs, the trailing update with fewer;
  // measured best near 63 at d = 500 and 24-37 at d = 1000, r = 6d)
  int GP = c->opts.qr_panel_ctas > 0 ? c->opts.qr_panel_ctas : kQrLaPanelWork / d;
  if (c->opts.qr_panel_ctas <= 0 && GP > G / 2) GP = G / 2;
  if (GP > G - 1) GP = G - 1;
  if (GP < 1) return true;
  const int64_t chunk_max = (r + GP - 1) / GP;
  const int64_t chunk_u = (r + (G - GP) - 1) / (G - GP);
  const size_t smem = qr_la_smem(chunk_max, chunk_u);
  if (smem > (size_t)200 * 1024) return true;
  if (cudaFuncSetAttribute(k_qr_la, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return false;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_la, QT, smem) != cudaSuccess)
    return false;
  if (per_sm < 1) return true;
  if (cudaMemsetAsync(s.qr_bar, 0, 3 * kBarWords * sizeof(unsigned), c->stream) != cudaSuccess)
    return false;
  QrLaArgs a{};
  a.A = s.Ahat;
  a.r = r;
  a.d = d;
  a.gp = GP;
  a.chunk_max = (int)chunk_max;
  a.Tg = s.qr_tg;
  a.Rdiag = s.Rdiag;
  a.vdiag = s.qr_vdiag;
  a.red = s.qr_red;
  a.Wl = s.qr_wl;
  a.Wp = s.qr_wp;
  a.Wt = s.qr_wt;
  a.chunk_u = (int)chunk_u;
  a.bar = s.qr_bar;
  a.bar2 = s.qr_bar + kBarWords;
  a.bar3 = s.qr_bar + 2 * kBarWords;
  a.status = &c->scal->status;
  a.spin = c->opts.spin_budget > 0 ? c->opts.spin_budget : (1ll << 31);
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)k_qr_la, dim3(G), dim3(QT), args, smem,
                                  c->stream) != cudaSuccess)
    return false;
  c->n_launch += 1;
  *launched = true;
  return true;
}

spcg_status launch_precond_factor(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int d = c->d;
  const int64_t r = s.sched.r;
  bool la = false;
  if (!launch_qr_la(c, &la)) return SPCG_E_CUDA;
  if (la) return finish_precond(c);
  int G = qr_coop_grid(r, c->num_sms);
  // the panels are factored by the first GP CTAs, about kQrPanelRows rows each:
  // fewer CTAs in each column step's reduction and barrier (latency), more rows
  // each (the step's FP64 work); the trailing updates use all G CTAs
  int GP = c->opts.qr_panel_ctas > 0 ? c->opts.qr_panel_ctas
                                     : (int)((r + kQrPanelRows - 1) / kQrPanelRows);
  if (GP > G) GP = G;
  if (GP < 1) GP = 1;
  const int64_t chunk_max = (r + GP - 1) / GP;
  const size_t smem = qr_coop_smem(chunk_max);
  bool coop = smem <= (size_t)200 * 1024 && c->opts.qr_by_column != 1;
  if (coop) {
    SPCG_CK(cudaFuncSetAttribute(k_qr_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SPCG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_coop, QT, smem));
    if (per_sm < 1) coop = false;   // cannot be co-resident: use the per-column steps
  }
  if (coop) {
    SPCG_CK(cudaMemsetAsync(s.qr_bar, 0, 2 * kBarWords * sizeof(unsigned), c->stream));
    QrCoopArgs a{};
    a.A = s.Ahat;
    a.r = r;
    a.d = d;
    a.gp = GP;
    a.chunk_max = (int)chunk_max;
    a.Tg = s.qr_tg;
    a.bar2 = s.qr_bar + kBarWords;
    a.Rdiag = s.Rdiag;
    a.vdiag = s.qr_vdiag;
    a.red = s.qr_red;
    a.Wp = s.qr_wp;
    a.Wt = s.qr_wt;
    a.bar = s.qr_bar;
    a.status = &c->scal->status;
    a.spin = c->opts.spin_budget > 0 ? c->opts.spin_budget : (1ll << 31);
    void* args[] = {&a};
    SPCG_CK(cudaLaunchCooperativeKernel((const void*)k_qr_coop, dim3(G), dim3(QT), args, smem,
                                        c->stream));
    c->n_launch += 1;
  } else {
    SPCG_TRY(householder_by_column(c));
  }
  return finish_precond(c);
}

// R from the reduced sketch, R^{-1} and R^{-T}.
static spcg_status finish_precond(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int d = c->d;
  const int64_t r = s.sched.r;
  const int64_t dd = (int64_t)d * d;
  int g = (int)((dd + 255) / 256);
  if (g > 4096) g = 4096;
  k_extract_R<<<g, 256, 0, c->stream>>>(s.Ahat, r, d, s.Rdiag, s.R, &c->scal->status);
  SPCG_CK(cudaGetLastError());
  const size_t tsm = (size_t)TRI_WARPS * d * sizeof(double);
  SPCG_CK(cudaFuncSetAttribute(k_trtri_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tsm));
  k_trtri_blocked<<<(d + TRI_WARPS - 1) / TRI_WARPS, TRI_WARPS * 32, tsm, c->stream>>>(s.R, d,
                                                                                   s.RinvT);
  SPCG_CK(cudaGetLastError());
  dim3 tg((d + 31) / 32, (d + 31) / 32);
  k_transpose<<<tg, dim3(32, 8), 0, c->stream>>>(s.RinvT, d, s.Rinv);
  SPCG_CK(cudaGetLastError());
  c->n_launch += 3;
  return SPCG_OK;
}

}  // namespace spcg
