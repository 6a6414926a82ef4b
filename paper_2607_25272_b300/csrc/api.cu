// The C ABI of include/spcg.h: context, Algorithm 1 orchestration, exports.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.hpp"

namespace spcg {

// NVTX ranges around the phases of a solve (sketch, transform, preconditioner,
// each stage, Stage II) when the environment has SPCG_NVTX=1, read once per
// process, so that a profiler can group launches by phase (e.g. ncu --nvtx
// --nvtx-include "spcg_refine/").  The ranges are host-side and enclose the
// launches issued; with no profiler attached the NVTX calls do nothing.
static bool nvtx_on() {
  static const bool on = [] {
    const char* e = getenv("SPCG_NVTX");
    return e && e[0] == '1' && e[1] == 0;
  }();
  return on;
}

struct NvtxRange {
  bool on;
  explicit NvtxRange(const char* name) : on(nvtx_on()) {
    if (on) nvtxRangePushA(name);
  }
  NvtxRange(const char* name, int index) : on(nvtx_on()) {
    if (on) {
      char buf[48];
      snprintf(buf, sizeof(buf), "%s %d", name, index);
      nvtxRangePushA(buf);
    }
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

spcg_status from_cuda(cudaError_t e) {
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SPCG_E_OOM : SPCG_E_CUDA;
}

// Device allocations of a context go through dalloc/dfree, which keep the
// context's workspace total; with spcg_opts.max_workspace_bytes > 0 an
// allocation that would take the total past the cap fails with SPCG_E_OOM
// before cudaMalloc is called.
template <typename T>
static spcg_status dalloc(spcg_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  const size_t bytes = count * sizeof(T);
  if (c->opts.max_workspace_bytes > 0 &&
      c->ws_bytes + bytes > (size_t)c->opts.max_workspace_bytes)
    return SPCG_E_OOM;
  if (c->pool) SPCG_CK(cudaMallocFromPoolAsync((void**)p, bytes, c->pool, c->stream));
  else SPCG_CK(cudaMalloc((void**)p, bytes));
  c->ws_sizes[(const void*)*p] = bytes;
  c->ws_bytes += bytes;
  return SPCG_OK;
}

template <typename T>
static void dfree(spcg_ctx* c, T*& p) {
  if (p) {
    auto it = c->ws_sizes.find((const void*)p);
    if (it != c->ws_sizes.end()) {
      c->ws_bytes -= it->second;
      c->ws_sizes.erase(it);
    }
    if (c->pool) cudaFreeAsync((void*)p, c->stream);
    else cudaFree((void*)p);
  }
  p = nullptr;
}

// Scratch of the cooperative QR (launch_precond_factor): one CTA per SM at
// most, panels of kQrPanel columns.
static spcg_status qr_alloc(spcg_ctx* c) {
  Sketch& s = c->sk;
  const int d = c->d, G = c->num_sms;
  SPCG_TRY(dalloc(c, &s.qr_vdiag, (size_t)d));
  SPCG_TRY(dalloc(c, &s.qr_red, (size_t)2 * G * 2 * kQrPanel));
  SPCG_TRY(dalloc(c, &s.qr_wp, (size_t)G * kQrPanel * d));
  SPCG_TRY(dalloc(c, &s.qr_wt, (size_t)kQrPanel * d));
  SPCG_TRY(dalloc(c, &s.qr_tg, (size_t)2 * kQrPanel * kQrPanel));
  SPCG_TRY(dalloc(c, &s.qr_wl, (size_t)(G + 1) * kQrPanel * kQrPanel));
  SPCG_TRY(dalloc(c, &s.qr_bar, (size_t)3 * kBarWords));
  return SPCG_OK;
}

static int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

static int ilog2(int64_t p) {
  int k = 0;
  while ((int64_t(1) << k) < p) ++k;
  return k;
}

static spcg_status validate_schedule(const spcg_schedule& s, int64_t N, int d) {
  const int64_t n_pad = next_pow2(N);
  if (s.K < 0 || s.K > SPCG_MAX_STAGES) return SPCG_E_INVALID_ARG;
  if (s.r < d || s.r > n_pad) return SPCG_E_INVALID_ARG;
  for (int i = 0; i < s.K; ++i) {
    if (s.m[i] < d || s.m[i] > n_pad || s.a[i] < 0) return SPCG_E_INVALID_ARG;
    if (i > 0 && s.m[i] <= s.m[i - 1]) return SPCG_E_INVALID_ARG;
  }
  if (!(s.tol > 0.0) || s.max_iters < 0 || s.max_restarts < 0) return SPCG_E_INVALID_ARG;
  if (s.sketch != SPCG_SKETCH_SRHT && s.sketch != SPCG_SKETCH_COUNT) return SPCG_E_INVALID_ARG;
  if (s.sketch == SPCG_SKETCH_COUNT) {
    if (s.K < 1) return SPCG_E_INVALID_ARG;
    for (int i = 0; i < s.K; ++i)   // buckets fold modulo m_i: powers of two
      if (s.m[i] & (s.m[i] - 1)) return SPCG_E_INVALID_ARG;
    if (s.r > (int64_t(1) << 31)) return SPCG_E_INVALID_ARG;
  }
  return SPCG_OK;
}

spcg_status prof_events(spcg_ctx* c, cudaEvent_t* e0, cudaEvent_t* e1, int op) {
  if (c->prof_used + 2 > c->prof_cap) {
    // the stream is idle only after a sync; collect what is pending first
    SPCG_CK(cudaStreamSynchronize(c->stream));
    SPCG_TRY(prof_collect(c));
    if (c->prof_cap == 0) {
      c->prof_cap = 512;
      c->prof_ev = (cudaEvent_t*)calloc(c->prof_cap, sizeof(cudaEvent_t));
      c->prof_op = (int*)calloc(c->prof_cap / 2, sizeof(int));
      if (!c->prof_ev || !c->prof_op) return SPCG_E_OOM;
      for (int i = 0; i < c->prof_cap; ++i) SPCG_CK(cudaEventCreate(&c->prof_ev[i]));
    }
  }
  c->prof_op[c->prof_used / 2] = op;
  *e0 = c->prof_ev[c->prof_used++];
  *e1 = c->prof_ev[c->prof_used++];
  return SPCG_OK;
}

spcg_status prof_collect(spcg_ctx* c) {
  for (int i = 0; i + 1 < c->prof_used; i += 2) {
    float ms = 0.f;
    SPCG_CK(cudaEventElapsedTime(&ms, c->prof_ev[i], c->prof_ev[i + 1]));
    c->prof_ms += ms;
    c->prof_ms_op[c->prof_op[i / 2] & 3] += ms;
  }
  c->prof_used = 0;
  return SPCG_OK;
}

// Launch and pass accounting of one solve (spcg_info).
static void reset_accounting(spcg_ctx* c) {
  c->n_launch = c->n_pass = 0;
  c->pass_bytes = 0;
  c->prof_ms = 0.0;
  for (int k = 0; k < 4; ++k) {
    c->n_pass_op[k] = 0;
    c->pass_bytes_op[k] = 0;
    c->prof_ms_op[k] = 0.0;
  }
}

// Read the device scalars (synchronises the stream) and map the device
// status to the ABI status.
static spcg_status sync_scalars(spcg_ctx* c) {
  SPCG_CK(cudaMemcpyAsync(&c->host_scal, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                          c->stream));
  SPCG_CK(cudaStreamSynchronize(c->stream));
  SPCG_TRY(prof_collect(c));
  switch (c->host_scal.status) {
    case DEV_OK: return SPCG_OK;
    case DEV_BREAKDOWN: return SPCG_E_BREAKDOWN;
    case DEV_TIMEOUT: return SPCG_E_TIMEOUT;
    default: return SPCG_E_CUDA;
  }
}

// g = A^T (b - A beta), u = R^{-T} g, z = R^{-1} u, dots: the PCG start.
// df: the gradient comes from the double-FP32 pass over the split of X.
static spcg_status start_sequence(spcg_ctx* c, const PassGeom& g, const double* b,
                                  double* beta, int& cur, bool df = false) {
  if (df) SPCG_TRY(pass_resid_df(c, c->gxdf, c->tml, b, beta));
  else SPCG_TRY(pass_resid(c, g, b, beta));
  SPCG_TRY(launch_dspace(c, 0, cur, 0, 0, beta));   // g, u = R^{-T} g, z, dots
  cur ^= 1;
  return SPCG_OK;
}

// Operand of the fused pass: one array (FP64, FP32 or BF16 rows), or the
// double-FP32 pair Xh + Xl when tml is set.
struct Operand {
  const PassGeom* g;
  const CUtensorMap* tml;
};

// One PCG iteration (two launches: the fused pass and the d-space kernel)
// after start_sequence or a previous one.
static spcg_status iteration(spcg_ctx* c, const Operand& op, double* beta, int& cur, int& pp,
                             int& gp, int start, int check, double tau) {
  if (op.tml) SPCG_TRY(pass_gram_iter_df(c, *op.g, *op.tml, pp, gp, start, check, tau));
  else SPCG_TRY(pass_gram_iter(c, *op.g, pp, gp, start, check, tau));
  pp ^= 1;
  gp ^= 1;
  SPCG_TRY(launch_dspace(c, 1, cur, pp, gp, beta));
  cur ^= 1;
  return SPCG_OK;
}

static spcg_status run_stage(spcg_ctx* c, int i, int a_i, double* beta) {
  const NvtxRange range("spcg_stage", i);
  const PassGeom& g = c->sk.geom[i];
  SPCG_TRY(launch_reset_loop(c));
  int cur = 0, pp = 0, gp = 0;
  SPCG_TRY(start_sequence(c, g, c->sk.bK + c->sk.stage_off[i], beta, cur));
  const Operand op{&g, nullptr};
  for (int k = 0; k < a_i; ++k) SPCG_TRY(iteration(c, op, beta, cur, pp, gp, k == 0, 0, 0.0));
  return SPCG_OK;
}

// A stage on the first m rows of the sketched prefix (SRHT only).
static spcg_status run_stage_m(spcg_ctx* c, int64_t m, int a_i, double* beta) {
  PassGeom g;
  if (c->sk.mixed)
    SPCG_TRY(make_pass_geom_t(c->sk.AK16, m, c->d, c->sk.ldak16, DT_BF16, &g));
  else
    SPCG_TRY(make_pass_geom(c->sk.AK, m, c->d, c->sk.ldak, &g));
  SPCG_TRY(launch_reset_loop(c));
  int cur = 0, pp = 0, gp = 0;
  SPCG_TRY(start_sequence(c, g, c->sk.bK, beta, cur));
  const Operand op{&g, nullptr};
  for (int k = 0; k < a_i; ++k) SPCG_TRY(iteration(c, op, beta, cur, pp, gp, k == 0, 0, 0.0));
  return SPCG_OK;
}

struct RefineResult {
  int iters = 0, restarts = 0, converged = 0;
};

// Stage II operand of the mixed path: FP32 rows while 2^-24 nu <= 1/32 (nu
// the ||D R^{-1}||_2 estimate of the sketch), else the double-FP32 pair.
constexpr double kInnerF32MaxPerturbation = 1.0 / 32.0;

// True gradients of the mixed path: double-FP32 while 2^-48 nu <= tol/64.
// The double-FP32 error per term is near 2^-48 relative; reaching the
// stopping metric it is amplified by up to nu, and the test compares it with
// (tol/2) ||R beta||.
constexpr double kGradDfMaxPerturbationPerTol = 1.0 / 64.0;

static int choose_grad(const spcg_ctx* c, double tol) {
  if (c->opts.precision != SPCG_PREC_MIXED) return SPCG_GRAD_F64;
  if (c->opts.grad_prec == SPCG_GRAD_F64 || c->opts.grad_prec == SPCG_GRAD_DF)
    return c->opts.grad_prec;
  return ldexp(c->cond_est, -48) <= kGradDfMaxPerturbationPerTol * tol ? SPCG_GRAD_DF
                                                                       : SPCG_GRAD_F64;
}

static int choose_inner(const spcg_ctx* c) {
  if (c->opts.inner_prec == SPCG_INNER_F32 || c->opts.inner_prec == SPCG_INNER_DF)
    return c->opts.inner_prec;
  return ldexp(c->cond_est, -24) <= kInnerF32MaxPerturbation ? SPCG_INNER_F32 : SPCG_INNER_DF;
}

static spcg_status run_refine(spcg_ctx* c, double tol, int max_iters, int max_restarts,
                              double* beta, RefineResult* res) {
  const NvtxRange range("spcg_refine");
  const double tau = tol / 2.0;
  const bool mixed = c->opts.precision == SPCG_PREC_MIXED;
  const PassGeom& g = c->gx;                                  // true gradients: FP64 X
  Operand gi{&c->gx, nullptr};                                // iterations
  c->inner_used = 0;
  c->grad_used = choose_grad(c, tol);
  const bool df_grad = c->grad_used == SPCG_GRAD_DF;
  if (mixed) {
    c->inner_used = choose_inner(c);
    gi = c->inner_used == SPCG_INNER_DF ? Operand{&c->gxdf, &c->tml} : Operand{&c->gxf, nullptr};
  }
  int total = 0, restarts = 0;
  SPCG_TRY(launch_reset_loop(c));
  for (;;) {
    // true gradient and the stopping test on it
    int cur = 0, pp = 0, gp = 0;
    SPCG_TRY(start_sequence(c, g, c->Y, beta, cur, df_grad));
    SPCG_TRY(launch_check(c, tau));
    SPCG_TRY(sync_scalars(c));
    if (c->host_scal.done == 2) {
      res->iters = total;
      res->restarts = restarts;
      res->converged = 1;
      return SPCG_OK;
    }
    if (total >= max_iters || restarts > max_restarts) break;
    int start = 1;
    bool hit = false;
    while (total < max_iters) {
      const int remaining = max_iters - total;
      const int chunk = remaining < 4 ? remaining : 4;
      for (int k = 0; k < chunk; ++k) {
        SPCG_TRY(iteration(c, gi, beta, cur, pp, gp, start, 1, tau));
        start = 0;
      }
      SPCG_TRY(sync_scalars(c));
      total += c->host_scal.iters;
      SPCG_TRY(launch_reset_loop(c));   // clears done and the iteration count
      if (c->host_scal.done == 1) {
        hit = true;
        break;
      }
    }
    if (!hit) break;
    ++restarts;
  }
  res->iters = total;
  res->restarts = restarts;
  res->converged = 0;
  return SPCG_E_NOT_CONVERGED;
}

static void free_sketch(spcg_ctx* c) {
  Sketch& s = c->sk;
  dfree(c, s.AK16);
  dfree(c, s.gather);
  dfree(c, s.dest);
  dfree(c, s.hdest);
  dfree(c, s.work);
  dfree(c, s.AK);
  dfree(c, s.bK);
  dfree(c, s.Ahat);
  s.ready = false;
  s.rows_alloc = s.r_alloc = 0;
  s.work_bytes = 0;
  s.n_pad = 0;
}

}  // namespace spcg

using namespace spcg;

extern "C" const char* spcg_status_str(spcg_status s) {
  switch (s) {
    case SPCG_OK: return "SPCG_OK";
    case SPCG_E_INVALID_ARG: return "SPCG_E_INVALID_ARG";
    case SPCG_E_OOM: return "SPCG_E_OOM";
    case SPCG_E_CUDA: return "SPCG_E_CUDA";
    case SPCG_E_BREAKDOWN: return "SPCG_E_BREAKDOWN";
    case SPCG_E_NOT_CONVERGED: return "SPCG_E_NOT_CONVERGED";
    case SPCG_E_TIMEOUT: return "SPCG_E_TIMEOUT";
    case SPCG_E_STATE: return "SPCG_E_STATE";
  }
  return "SPCG_E_UNKNOWN";
}

extern "C" spcg_status spcg_default_schedule(int64_t N, int32_t d, spcg_schedule* out) {
  if (!out || d < 1 || N <= d) return SPCG_E_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  const int64_t n_pad = next_pow2(N);
  int64_t m = next_pow2(8 * (int64_t)d);
  int K = 0;
  while (m <= n_pad / 2 && K < SPCG_MAX_STAGES) {
    out->m[K] = m;
    out->a[K] = 3;
    ++K;
    m *= 2;
  }
  out->K = K;
  out->r = 6 * (int64_t)d < n_pad ? 6 * (int64_t)d : n_pad;
  out->tol = 1e-6;
  out->max_iters = 100;
  out->max_restarts = 5;
  return SPCG_OK;
}

extern "C" spcg_status spcg_tuned_schedule(int64_t N, int32_t d, spcg_schedule* out) {
  SPCG_TRY(spcg_default_schedule(N, d, out));
  const int64_t n_pad = next_pow2(N);
  int64_t m = next_pow2(16 * (int64_t)d);
  int K = 0;
  while (K < 7 && m < n_pad / 4) {
    out->m[K] = m;
    out->a[K] = 4;
    ++K;
    m *= 2;
  }
  const int64_t last = K > 0 ? out->m[K - 1] : 0;
  if (n_pad / 4 > last && n_pad / 4 > 6 * (int64_t)d) {
    out->m[K] = n_pad / 4;
    out->a[K] = 4;
    ++K;
  }
  for (int i = K; i < SPCG_MAX_STAGES; ++i) {
    out->m[i] = 0;
    out->a[i] = 0;
  }
  out->K = K;
  out->r = 6 * (int64_t)d < n_pad ? 6 * (int64_t)d : n_pad;
  return SPCG_OK;
}

// The stream-ordered memory pool of spcg_solve_host, one per device, created
// on first use with a release threshold of "never": memory freed at the end
// of a call stays in the pool for the next call (spcg_host_pool_trim
// returns it to the device).
namespace {
struct HostPool {
  std::mutex mu;
  cudaMemPool_t pool = nullptr;
};
HostPool g_host_pools[64];

spcg_status host_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 64) return SPCG_E_INVALID_ARG;
  HostPool& hp = g_host_pools[dev];
  std::lock_guard<std::mutex> lock(hp.mu);
  if (!hp.pool) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    SPCG_CK(cudaMemPoolCreate(&p, &props));
    uint64_t keep = ~0ull;
    if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return from_cuda(cudaGetLastError());
    }
    hp.pool = p;
  }
  *out = hp.pool;
  return SPCG_OK;
}
}  // namespace

// Options out of their documented ranges (checked before any CUDA call).
static bool opts_valid(const spcg_opts& o) {
  return (o.precision == SPCG_PREC_FP64 || o.precision == SPCG_PREC_MIXED) &&
         o.fwht_tile >= 0 && o.fwht_tile <= 3 && o.fwht_first_levels >= 0 &&
         o.fwht_first_levels <= 12 && o.max_workspace_bytes >= 0 && o.qr_panel_ctas >= 0 &&
         o.dspace_ctas >= 0 && o.qr_by_column >= 0 && o.qr_by_column <= 2;
}

static spcg_status create_impl(const double* X, const double* Y, int64_t N, int32_t d,
                               int64_t ldx, void* stream, const spcg_opts* opts,
                               cudaMemPool_t pool, spcg_ctx** out) {
  if (!out) return SPCG_E_INVALID_ARG;
  *out = nullptr;
  if (!X || !Y || d < 1 || d > SPCG_MAX_D || N <= d || N > (int64_t(1) << 30) || ldx < d)
    return SPCG_E_INVALID_ARG;
  if (opts && !opts_valid(*opts)) return SPCG_E_INVALID_ARG;
  spcg_ctx* c = new spcg_ctx();
  c->pool = pool;
  c->stream = (cudaStream_t)stream;
  if (opts) c->opts = *opts;
  c->N = N;
  c->d = d;
  c->Y = Y;
  spcg_status st = SPCG_OK;
  auto fail = [&](spcg_status s) {
    spcg_destroy(c);
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(SPCG_E_CUDA);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
      cudaSuccess)
    return fail(SPCG_E_CUDA);
  // X: borrowed, or a padded copy when the row stride breaks the TMA rule
  if ((ldx * 8) % 16 != 0 || ((uintptr_t)X & 15u) != 0) {
    const int64_t ld2 = (d + 1) & ~int64_t(1);
    if ((st = dalloc(c, &c->X_own, (size_t)N * ld2)) != SPCG_OK) return fail(st);
    if (cudaMemcpy2DAsync(c->X_own, ld2 * 8, X, ldx * 8, (size_t)d * 8, N,
                          cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
      return fail(SPCG_E_CUDA);
    c->X = c->X_own;
    c->ldx = ld2;
  } else {
    c->X = X;
    c->ldx = ldx;
  }
  if ((st = dalloc(c, &c->scal, 1)) != SPCG_OK) return fail(st);
  if (cudaMemsetAsync(c->scal, 0, sizeof(DevScalars), c->stream) != cudaSuccess)
    return fail(SPCG_E_CUDA);
  PcgBuffers& pb = c->pb;
  pb.grid = c->opts.grid_ctas > 0 ? c->opts.grid_ctas : c->num_sms;
  int ni = 1;
  while (ni * 32 < d) ni <<= 1;
  pb.ldp = ni * 32;
  pb.n_red = (d + 31) / 32;
  pb.n_pre = (d + 3) / 4;
  pb.n_ds = dspace_grid(c);
  if ((st = dalloc(c, &pb.partials, (size_t)pb.grid * pb.ldp)) != SPCG_OK) return fail(st);
  double** vecs[] = {&pb.w, &pb.u, &pb.z, &pb.g[0], &pb.g[1], &pb.p[0], &pb.p[1], &c->beta_work};
  for (double** v : vecs) {
    if ((st = dalloc(c, v, (size_t)d)) != SPCG_OK) return fail(st);
    if (cudaMemsetAsync(*v, 0, (size_t)d * 8, c->stream) != cudaSuccess) return fail(SPCG_E_CUDA);
  }
  const int n_dots = std::max(std::max(pb.n_pre, pb.n_red), pb.n_ds);
  if ((st = dalloc(c, &pb.dots_pw, (size_t)n_dots)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &pb.dots_gz, (size_t)n_dots)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &pb.dots_rb, (size_t)n_dots)) != SPCG_OK) return fail(st);
  Sketch& s = c->sk;
  if ((st = dalloc(c, &s.Rdiag, (size_t)d)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &s.R, (size_t)d * d)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &s.Rinv, (size_t)d * d)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &s.RinvT, (size_t)d * d)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &s.colmax, (size_t)d + 1)) != SPCG_OK) return fail(st);
  if ((st = qr_alloc(c)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &c->mlp_x, 16)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &c->mlp_y, 64)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &c->feat_part, 2 * 128)) != SPCG_OK) return fail(st);
  if ((st = dalloc(c, &s.colshift, (size_t)d + 1)) != SPCG_OK) return fail(st);
  if ((st = make_pass_geom(c->X, N, d, c->ldx, &c->gx)) != SPCG_OK) return fail(st);
  if (c->opts.precision == SPCG_PREC_MIXED) {
    c->ldxf = (d + 3) & ~int64_t(3);
    if ((st = dalloc(c, &c->Xf, (size_t)N * c->ldxf)) != SPCG_OK) return fail(st);
    if ((st = dalloc(c, &c->Xl, (size_t)N * c->ldxf)) != SPCG_OK) return fail(st);
    if (c->ldxf > d && (cudaMemsetAsync(c->Xf, 0, (size_t)N * c->ldxf * 4, c->stream) != cudaSuccess ||
                        cudaMemsetAsync(c->Xl, 0, (size_t)N * c->ldxf * 4, c->stream) != cudaSuccess))
      return fail(SPCG_E_CUDA);
    if ((st = make_pass_geom_t(c->Xf, N, d, c->ldxf, DT_F32, &c->gxf)) != SPCG_OK) return fail(st);
    if ((st = make_pass_geom_df(c->Xf, c->Xl, N, d, c->ldxf, &c->gxdf, &c->tml)) != SPCG_OK)
      return fail(st);
  }
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(SPCG_E_CUDA);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(SPCG_E_CUDA);
  *out = c;
  return SPCG_OK;
}

extern "C" spcg_status spcg_create(const double* X, const double* Y, int64_t N, int32_t d,
                                   int64_t ldx, void* stream, const spcg_opts* opts,
                                   spcg_ctx** out) {
  return create_impl(X, Y, N, d, ldx, stream, opts, nullptr, out);
}

extern "C" void spcg_destroy(spcg_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_sketch(c);
  dfree(c, c->sk.Rdiag);
  dfree(c, c->sk.R);
  dfree(c, c->sk.Rinv);
  dfree(c, c->sk.RinvT);
  dfree(c, c->sk.colmax);
  dfree(c, c->sk.qr_vdiag);
  dfree(c, c->sk.qr_red);
  dfree(c, c->sk.qr_wp);
  dfree(c, c->sk.qr_wl);
  dfree(c, c->sk.qr_wt);
  dfree(c, c->sk.qr_bar);
  dfree(c, c->sk.qr_tg);
  dfree(c, c->mlp_x);
  dfree(c, c->mlp_y);
  dfree(c, c->feat_part);
  dfree(c, c->sk.colshift);
  PcgBuffers& pb = c->pb;
  dfree(c, pb.partials);
  dfree(c, pb.w);
  dfree(c, pb.u);
  dfree(c, pb.z);
  dfree(c, pb.g[0]);
  dfree(c, pb.g[1]);
  dfree(c, pb.p[0]);
  dfree(c, pb.p[1]);
  dfree(c, pb.dots_pw);
  dfree(c, pb.dots_gz);
  dfree(c, pb.dots_rb);
  dfree(c, c->beta_work);
  dfree(c, c->scal);
  dfree(c, c->X_own);
  dfree(c, c->Xf);
  dfree(c, c->Xl);
  dfree(c, c->sk.AK16);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < c->prof_cap; ++i)
    if (c->prof_ev[i]) cudaEventDestroy(c->prof_ev[i]);
  free(c->prof_ev);
  free(c->prof_op);
  delete c;
}

extern "C" spcg_status spcg_sketch(spcg_ctx* c, uint64_t seed, const spcg_schedule* sched) {
  if (!c) return SPCG_E_INVALID_ARG;
  const NvtxRange range("spcg_sketch");
  spcg_schedule sc;
  if (sched) sc = *sched;
  else SPCG_TRY(spcg_default_schedule(c->N, c->d, &sc));
  SPCG_TRY(validate_schedule(sc, c->N, c->d));
  Sketch& s = c->sk;
  s.ready = false;
  const int d = c->d;
  const int64_t n_pad = next_pow2(c->N);
  const int nbits = ilog2(n_pad);
  const int64_t mK = sc.K > 0 ? sc.m[sc.K - 1] : 0;
  if (s.n_pad != n_pad) {
    dfree(c, s.gather);
    dfree(c, s.dest);
    dfree(c, s.hdest);
    SPCG_TRY(dalloc(c, &s.gather, (size_t)n_pad));
    SPCG_TRY(dalloc(c, &s.dest, (size_t)n_pad));
    SPCG_TRY(dalloc(c, &s.hdest, (size_t)n_pad));
    s.n_pad = n_pad;
  }
  s.nbits = nbits;
  const bool cs = sc.sketch == SPCG_SKETCH_COUNT;
  // stage storage: SRHT stages share one prefix; CountSketch stages are separate
  int64_t rows = 0;
  for (int i = 0; i < sc.K; ++i) {
    s.stage_off[i] = cs ? rows : 0;
    rows = cs ? rows + sc.m[i] : mK;
  }
  const bool multipass = nbits > 12;
  size_t work_bytes = multipass ? (size_t)n_pad * (d + 1) * 8 : 0;
  if (cs) work_bytes = (size_t)(mK + sc.r) * (d + 1) * 8;   // int64 buckets of S_K and S-hat
  if (work_bytes > s.work_bytes) {
    dfree(c, s.work);
    SPCG_TRY(dalloc(c, (unsigned char**)&s.work, work_bytes));
    s.work_bytes = work_bytes;
  }
  s.ldw = d + 1;
  s.ldak = (d + 1) & ~int64_t(1);
  s.ldak16 = (d + 7) & ~int64_t(7);
  const bool mixed = (c->opts.precision == SPCG_PREC_MIXED);
  if (rows > s.rows_alloc || mixed != s.mixed) {
    dfree(c, s.AK);
    dfree(c, s.AK16);
    dfree(c, s.bK);
    s.rows_alloc = 0;
    SPCG_TRY(dalloc(c, &s.bK, (size_t)rows));
    if (mixed) SPCG_TRY(dalloc(c, &s.AK16, (size_t)rows * s.ldak16));
    else SPCG_TRY(dalloc(c, &s.AK, (size_t)rows * s.ldak));
    s.rows_alloc = rows;
  }
  s.mixed = mixed;
  if (sc.r > s.r_alloc) {
    dfree(c, s.Ahat);
    SPCG_TRY(dalloc(c, &s.Ahat, (size_t)sc.r * d));
    s.r_alloc = sc.r;
  }
  s.seed = seed;
  s.sched = sc;
  if (!s.mixed && s.ldak > d && rows > 0)   // padding columns of the stage rows stay zero
    SPCG_CK(cudaMemsetAsync(s.AK, 0, (size_t)rows * s.ldak * 8, c->stream));
  if (s.mixed && s.ldak16 > d && rows > 0)
    SPCG_CK(cudaMemsetAsync(s.AK16, 0, (size_t)rows * s.ldak16 * 2, c->stream));
  for (int i = 0; i < sc.K; ++i) {
    if (s.mixed)
      SPCG_TRY(make_pass_geom_t(reinterpret_cast<uint16_t*>(s.AK16) + s.stage_off[i] * s.ldak16,
                                sc.m[i], d, s.ldak16, DT_BF16, &s.geom[i]));
    else
      SPCG_TRY(make_pass_geom(s.AK + s.stage_off[i] * s.ldak, sc.m[i], d, s.ldak, &s.geom[i]));
  }
  SPCG_TRY(launch_reset_flags(c));
  {
    const NvtxRange range(cs ? "spcg_countsketch" : "spcg_transform");
    if (cs) {
      SPCG_TRY(launch_countsketch(c));
    } else {
      SPCG_TRY(launch_sketch_maps(c));
      SPCG_TRY(launch_transform(c));
    }
  }
  {
    const NvtxRange range("spcg_precond");
    SPCG_TRY(launch_precond_factor(c));
    if (s.mixed) SPCG_TRY(launch_condest(c));
  }
  SPCG_TRY(sync_scalars(c));
  c->cond_est = s.mixed ? c->host_scal.cond : 0.0;
  s.ready = true;
  return SPCG_OK;
}

extern "C" spcg_status spcg_pcg_stage(spcg_ctx* c, int32_t i, int32_t a_i, double* beta) {
  if (!c || !beta) return SPCG_E_INVALID_ARG;
  if (!c->sk.ready) return SPCG_E_STATE;
  if (i < 0 || i >= c->sk.sched.K || a_i < 0) return SPCG_E_INVALID_ARG;
  SPCG_TRY(launch_reset_flags(c));   // a new call starts without an earlier error
  SPCG_TRY(run_stage(c, i, a_i, beta));
  return sync_scalars(c);
}

extern "C" spcg_status spcg_refine(spcg_ctx* c, double tol, int32_t max_iters, double* beta,
                                   int32_t* iters_out) {
  if (!c || !beta || !(tol > 0.0) || max_iters < 0) return SPCG_E_INVALID_ARG;
  if (!c->sk.ready) return SPCG_E_STATE;
  if (c->opts.precision == SPCG_PREC_MIXED) SPCG_TRY(launch_to_f32(c));
  SPCG_TRY(launch_reset_flags(c));   // a new call starts without an earlier error
  RefineResult rr;
  spcg_status st = run_refine(c, tol, max_iters, c->sk.sched.max_restarts, beta, &rr);
  if (iters_out) *iters_out = rr.iters;
  return st;
}

// The sketch of a solve; in the mixed form the FP32 split of X runs first and
// hands the sketch its column maxima (one read of X fewer).
static spcg_status sketch_after_split(spcg_ctx* c, uint64_t seed, const spcg_schedule* sched) {
  if (c->opts.precision != SPCG_PREC_MIXED) return spcg_sketch(c, seed, sched);
  SPCG_TRY(launch_to_f32_colmax(c));
  const spcg_status st = spcg_sketch(c, seed, sched);
  c->sk.colmax_pre = false;   // only that sketch may use them
  return st;
}

extern "C" spcg_status spcg_solve(spcg_ctx* c, uint64_t seed, const spcg_schedule* sched,
                                  double* beta, spcg_info* info) {
  if (!c || !beta) return SPCG_E_INVALID_ARG;
  const NvtxRange range("spcg_solve");
  if (info) memset(info, 0, sizeof(*info));
  reset_accounting(c);
  SPCG_CK(cudaEventRecord(c->ev[0], c->stream));
  SPCG_TRY(sketch_after_split(c, seed, sched));
  SPCG_CK(cudaEventRecord(c->ev[1], c->stream));
  const spcg_schedule& sc = c->sk.sched;
  SPCG_CK(cudaMemsetAsync(c->beta_work, 0, (size_t)c->d * 8, c->stream));
  for (int i = 0; i < sc.K; ++i) SPCG_TRY(run_stage(c, i, sc.a[i], c->beta_work));
  SPCG_TRY(sync_scalars(c));
  SPCG_CK(cudaEventRecord(c->ev[2], c->stream));
  RefineResult rr;
  spcg_status st = run_refine(c, sc.tol, sc.max_iters, sc.max_restarts, c->beta_work, &rr);
  SPCG_CK(cudaEventRecord(c->ev[3], c->stream));
  SPCG_CK(cudaMemcpyAsync(beta, c->beta_work, (size_t)c->d * 8, cudaMemcpyDeviceToDevice,
                          c->stream));
  SPCG_CK(cudaStreamSynchronize(c->stream));
  SPCG_TRY(prof_collect(c));
  if (info) {
    info->K = sc.K;
    info->pass_launches = (int32_t)c->n_pass;
    info->launches = (int32_t)c->n_launch;
    info->pass_ms = c->prof_ms;
    for (int k = 0; k < 4; ++k) {
      info->pass_ms_by_op[k] = c->prof_ms_op[k];
      info->bytes_by_op[k] = c->pass_bytes_op[k];
      info->launches_by_op[k] = (int32_t)c->n_pass_op[k];
    }
    for (int i = 0; i < sc.K; ++i) info->stage_iters[i] = sc.a[i];
    info->refine_iters = rr.iters;
    info->restarts = rr.restarts;
    info->converged = rr.converged;
    info->sqrt_gamma = c->host_scal.sqrt_gamma;
    info->norm_R_beta = c->host_scal.norm_rb;
    info->bytes_pass = c->pass_bytes;
    info->cond_est = c->cond_est;
    info->inner_prec = c->inner_used;
    info->grad_prec = c->grad_used;
    float ms;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    info->ms_sketch = ms;
    cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]);
    info->ms_stages = ms;
    cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
    info->ms_refine = ms;
  }
  return st;
}

extern "C" spcg_status spcg_solve_enqueue(spcg_ctx* c, double* beta, int32_t rounds,
                                          int32_t iters_per_round) {
  if (!c || !beta || rounds < 1 || iters_per_round < 1) return SPCG_E_INVALID_ARG;
  if (!c->sk.ready) return SPCG_E_STATE;
  if (c->opts.profile) return SPCG_E_INVALID_ARG;   // event timing reads the host between launches
  const spcg_schedule& sc = c->sk.sched;
  const bool mixed = c->opts.precision == SPCG_PREC_MIXED;
  reset_accounting(c);
  if (mixed) SPCG_TRY(launch_to_f32(c));
  SPCG_TRY(launch_reset_flags(c));
  SPCG_CK(cudaMemsetAsync(beta, 0, (size_t)c->d * 8, c->stream));
  for (int i = 0; i < sc.K; ++i) SPCG_TRY(run_stage(c, i, sc.a[i], beta));
  // Stage II on a fixed schedule: every round is a true gradient with its
  // test, then iters_per_round iterations with the recursive test.  Once the
  // test passes, the rest of the round does nothing (done 1) until the next
  // round's true gradient confirms it (done 2: everything after does nothing)
  // or sends the iterations on from that gradient (done 0).
  const double tau = sc.tol / 2.0;
  c->inner_used = 0;
  c->grad_used = choose_grad(c, sc.tol);
  Operand gi{&c->gx, nullptr};
  if (mixed) {
    c->inner_used = choose_inner(c);
    gi = c->inner_used == SPCG_INNER_DF ? Operand{&c->gxdf, &c->tml} : Operand{&c->gxf, nullptr};
  }
  SPCG_TRY(launch_reset_loop(c));
  for (int rd = 0; rd < rounds; ++rd) {
    int cur = 0, pp = 0, gp = 0;
    SPCG_TRY(start_sequence(c, c->gx, c->Y, beta, cur, c->grad_used == SPCG_GRAD_DF));
    SPCG_TRY(launch_check(c, tau));
    for (int k = 0; k < iters_per_round; ++k)
      SPCG_TRY(iteration(c, gi, beta, cur, pp, gp, k == 0, 1, tau));
  }
  // a last true gradient and test, so that an iterate reached in the last
  // round can still be confirmed
  int cur = 0;
  SPCG_TRY(start_sequence(c, c->gx, c->Y, beta, cur, c->grad_used == SPCG_GRAD_DF));
  SPCG_TRY(launch_check(c, tau));
  return SPCG_OK;
}

extern "C" spcg_status spcg_solve_result(spcg_ctx* c, spcg_info* info) {
  if (!c) return SPCG_E_INVALID_ARG;
  const spcg_status st = sync_scalars(c);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->K = c->sk.sched.K;
    for (int i = 0; i < c->sk.sched.K; ++i) info->stage_iters[i] = c->sk.sched.a[i];
    info->refine_iters = c->host_scal.iters;
    info->converged = c->host_scal.done == 2 ? 1 : 0;
    info->sqrt_gamma = c->host_scal.sqrt_gamma;
    info->norm_R_beta = c->host_scal.norm_rb;
    info->cond_est = c->cond_est;
    info->inner_prec = c->inner_used;
    info->grad_prec = c->grad_used;
    info->pass_launches = (int32_t)c->n_pass;
    info->launches = (int32_t)c->n_launch;
    info->bytes_pass = c->pass_bytes;
  }
  if (st != SPCG_OK) return st;
  return c->host_scal.done == 2 ? SPCG_OK : SPCG_E_NOT_CONVERGED;
}

extern "C" spcg_status spcg_solve_host(const double* X, const double* Y, int64_t N, int32_t d,
                                       int64_t ldx, uint64_t seed, const spcg_schedule* sched,
                                       const spcg_opts* opts, void* stream, double* beta,
                                       spcg_info* info) {
  if (!X || !Y || !beta || d < 1 || d > SPCG_MAX_D || N <= d || N > (int64_t(1) << 30) ||
      ldx < d || (opts && !opts_valid(*opts)))
    return SPCG_E_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  SPCG_CK(cudaGetDevice(&dev));
  cudaMemPool_t pool = nullptr;
  SPCG_TRY(host_pool(dev, &pool));
  const int64_t ld = (d + 1) & ~int64_t(1);   // device rows 16-byte aligned (TMA stride rule)
  double *Xd = nullptr, *Yd = nullptr, *bd = nullptr;
  spcg_ctx* c = nullptr;
  spcg_status res = SPCG_OK;
  cudaError_t e = cudaMallocFromPoolAsync((void**)&Xd, (size_t)N * ld * sizeof(double), pool, st);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&Yd, (size_t)N * sizeof(double), pool, st);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&bd, (size_t)d * sizeof(double), pool, st);
  if (e == cudaSuccess) {
    if (ldx == ld)
      e = cudaMemcpyAsync(Xd, X, (size_t)N * ld * sizeof(double), cudaMemcpyHostToDevice, st);
    else
      e = cudaMemcpy2DAsync(Xd, ld * sizeof(double), X, ldx * sizeof(double), d * sizeof(double),
                            N, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Yd, Y, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) res = from_cuda(e);
  if (res == SPCG_OK) res = create_impl(Xd, Yd, N, d, ld, stream, opts, pool, &c);
  spcg_status solve_st = SPCG_OK;
  if (res == SPCG_OK) {
    solve_st = spcg_solve(c, seed, sched, bd, info);
    // beta is copied back also when the solve did not converge (last iterate)
    if (solve_st == SPCG_OK || solve_st == SPCG_E_NOT_CONVERGED) {
      e = cudaMemcpyAsync(beta, bd, (size_t)d * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) res = from_cuda(e);
    }
  }
  if (c) spcg_destroy(c);   // synchronises the stream, then returns its workspace to the pool
  if (Xd) cudaFreeAsync(Xd, st);
  if (Yd) cudaFreeAsync(Yd, st);
  if (bd) cudaFreeAsync(bd, st);
  cudaStreamSynchronize(st);
  return res != SPCG_OK ? res : solve_st;
}

extern "C" spcg_status spcg_host_pool_trim(void) {
  for (int dev = 0; dev < 64; ++dev) {
    HostPool& hp = g_host_pools[dev];
    std::lock_guard<std::mutex> lock(hp.mu);
    if (hp.pool) SPCG_CK(cudaMemPoolTrimTo(hp.pool, 0));
  }
  return SPCG_OK;
}

extern "C" spcg_status spcg_export_sketch(spcg_ctx* c, int64_t row0, int64_t nrows, double* A,
                                          double* b) {
  if (!c || nrows < 0 || row0 < 0) return SPCG_E_INVALID_ARG;
  if (!c->sk.ready) return SPCG_E_STATE;
  const Sketch& s = c->sk;
  const int64_t mK = s.sched.K > 0 ? s.sched.m[s.sched.K - 1] : 0;
  if (row0 + nrows > mK) return SPCG_E_INVALID_ARG;
  if (nrows == 0) return SPCG_OK;
  SPCG_TRY(launch_export_rows(c, row0, nrows, A, b));
  SPCG_CK(cudaStreamSynchronize(c->stream));
  return SPCG_OK;
}

__global__ void k_colmajor_to_rowmajor(const double* __restrict__ src, int64_t r, int d,
                                       double* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d, j = e % d;
    dst[e] = src[j * r + i];
  }
}

extern "C" spcg_status spcg_export_precond(spcg_ctx* c, double* R, double* Rinv, double* Ahat) {
  if (!c) return SPCG_E_INVALID_ARG;
  if (!c->sk.ready) return SPCG_E_STATE;
  const size_t dd = (size_t)c->d * c->d * 8;
  if (R) SPCG_CK(cudaMemcpyAsync(R, c->sk.R, dd, cudaMemcpyDeviceToDevice, c->stream));
  if (Rinv) SPCG_CK(cudaMemcpyAsync(Rinv, c->sk.Rinv, dd, cudaMemcpyDeviceToDevice, c->stream));
  if (Ahat) {
    // Ahat is reduced in place by the QR; only R survives.  Re-run the
    // sketch into it when an export is asked for.
    if (c->sk.sched.sketch == SPCG_SKETCH_COUNT) SPCG_TRY(launch_countsketch(c));
    else SPCG_TRY(launch_transform(c));
    k_colmajor_to_rowmajor<<<256, 256, 0, c->stream>>>(c->sk.Ahat, c->sk.sched.r, c->d, Ahat);
    SPCG_CK(cudaGetLastError());
    // restore the factorised state expected by later calls
    SPCG_TRY(launch_precond_factor(c));
  }
  return sync_scalars(c);
}

extern "C" spcg_status spcg_gram_apply(spcg_ctx* c, const double* A, int64_t m, int64_t lda,
                                       const double* p, double* w) {
  if (!c || !p || !w || m < 0) return SPCG_E_INVALID_ARG;
  if (m == 0) {
    SPCG_CK(cudaMemsetAsync(w, 0, (size_t)c->d * 8, c->stream));
    SPCG_CK(cudaStreamSynchronize(c->stream));
    return SPCG_OK;
  }
  if (!A) return SPCG_E_INVALID_ARG;
  PassGeom g;
  SPCG_TRY(make_pass_geom(A, m, c->d, lda, &g));
  SPCG_TRY(launch_reset_flags(c));
  SPCG_TRY(pass_gram_plain(c, g, p));
  SPCG_TRY(launch_reduce(c, w, nullptr));
  return sync_scalars(c);
}

extern "C" spcg_status spcg_gram_apply_typed(spcg_ctx* c, const void* A, int32_t dtype, int64_t m,
                                             int64_t lda, const double* p, double* w) {
  if (!c || !p || !w || m < 0 || dtype < 0 || dtype > 3) return SPCG_E_INVALID_ARG;
  if (m == 0) {
    SPCG_CK(cudaMemsetAsync(w, 0, (size_t)c->d * 8, c->stream));
    SPCG_CK(cudaStreamSynchronize(c->stream));
    return SPCG_OK;
  }
  if (!A) return SPCG_E_INVALID_ARG;
  PassGeom g;
  SPCG_TRY(launch_reset_flags(c));
  if (dtype == 3) {   // double-FP32 pair: hi block, then lo block
    if (m > (int64_t(1) << 40) / (lda > 0 ? lda : 1)) return SPCG_E_INVALID_ARG;
    const float* hi = static_cast<const float*>(A);
    CUtensorMap tml;
    SPCG_TRY(make_pass_geom_df(hi, hi + m * lda, m, c->d, lda, &g, &tml));
    SPCG_TRY(pass_gram_plain_df(c, g, tml, p));
  } else {
    SPCG_TRY(make_pass_geom_t(A, m, c->d, lda, dtype, &g));
    SPCG_TRY(pass_gram_plain(c, g, p));
  }
  SPCG_TRY(launch_reduce(c, w, nullptr));
  return sync_scalars(c);
}

extern "C" spcg_status spcg_resid_apply_typed(spcg_ctx* c, const void* A, int32_t dtype,
                                              int64_t m, int64_t lda, const double* b,
                                              const double* x, double* g) {
  if (!c || !x || !g || m < 0 || dtype < 0 || dtype > 3) return SPCG_E_INVALID_ARG;
  if (m == 0) {
    SPCG_CK(cudaMemsetAsync(g, 0, (size_t)c->d * 8, c->stream));
    SPCG_CK(cudaStreamSynchronize(c->stream));
    return SPCG_OK;
  }
  if (!A || !b) return SPCG_E_INVALID_ARG;
  PassGeom geo;
  SPCG_TRY(launch_reset_flags(c));
  if (dtype == 3) {
    if (m > (int64_t(1) << 40) / (lda > 0 ? lda : 1)) return SPCG_E_INVALID_ARG;
    const float* hi = static_cast<const float*>(A);
    CUtensorMap tml;
    SPCG_TRY(make_pass_geom_df(hi, hi + m * lda, m, c->d, lda, &geo, &tml));
    SPCG_TRY(pass_resid_df(c, geo, tml, b, x));
  } else {
    SPCG_TRY(make_pass_geom_t(A, m, c->d, lda, dtype, &geo));
    SPCG_TRY(pass_resid(c, geo, b, x));
  }
  SPCG_TRY(launch_reduce(c, g, nullptr));
  return sync_scalars(c);
}

// ---------------------------------------------------------------------------
// Learned schedule: candidates, features, and the solve that uses the model.
// ---------------------------------------------------------------------------
namespace spcg {
spcg_status mlp_forward_launch(const void* Wb, int nout, const float* x, int64_t B, float* y,
                               cudaStream_t st);
spcg_status launch_features(spcg_ctx* c, const double* beta, float* dev_out2);
}

extern "C" int32_t spcg_num_candidates(void) { return 25; }

extern "C" spcg_status spcg_candidate_schedule(int64_t N, int32_t d, int32_t idx,
                                               spcg_schedule* out) {
  if (idx < 0 || idx >= 25) return SPCG_E_INVALID_ARG;
  SPCG_TRY(spcg_default_schedule(N, d, out));
  if (out->K == 0) return SPCG_OK;
  const int64_t n_pad = next_pow2(N);
  const int64_t m1 = out->m[0];
  int K = 1;
  out->a[0] = 3;
  if (idx > 0) {
    const int g = 1 + (idx - 1) / 6, rem = (idx - 1) % 6, sgrow = 1 + rem / 3, a = 2 + rem % 3;
    const int64_t top = n_pad >> g;
    for (int64_t m = m1 << sgrow; m <= top && K < SPCG_MAX_STAGES; m <<= sgrow) {
      out->m[K] = m;
      out->a[K] = a;
      ++K;
    }
  }
  for (int i = K; i < SPCG_MAX_STAGES; ++i) {
    out->m[i] = 0;
    out->a[i] = 0;
  }
  out->K = K;
  return SPCG_OK;
}

extern "C" spcg_status spcg_features(spcg_ctx* c, const double* beta, float* out4) {
  if (!c || !beta || !out4) return SPCG_E_INVALID_ARG;
  if (!c->sk.ready || c->sk.sched.sketch != SPCG_SKETCH_SRHT || c->sk.sched.K < 1)
    return SPCG_E_STATE;
  SPCG_TRY(launch_features(c, beta, c->mlp_x + 2));
  float f2[2];
  SPCG_CK(cudaMemcpyAsync(f2, c->mlp_x + 2, sizeof(f2), cudaMemcpyDeviceToHost, c->stream));
  SPCG_CK(cudaStreamSynchronize(c->stream));
  out4[0] = (float)log2((double)c->N);
  out4[1] = (float)log2((double)c->d);
  out4[2] = f2[0];
  out4[3] = f2[1];
  return SPCG_OK;
}

// Sketch (or reuse the context's sketch of the same seed), stage 1, then the
// candidate `force_idx` (>= 0) or the one the model scores cheapest.
static spcg_status solve_choice(spcg_ctx* c, uint64_t seed, const uint16_t* Wb, int32_t n_out,
                                const float* norm, double tol, int force_idx, int reuse,
                                double* beta, spcg_info* info, int32_t* choice) {
  if (!c || !beta || !(tol > 0.0)) return SPCG_E_INVALID_ARG;
  if (info) memset(info, 0, sizeof(*info));
  const int paper = 2;   // candidate index of the paper's schedule
  spcg_schedule sc;
  SPCG_TRY(spcg_default_schedule(c->N, c->d, &sc));
  sc.tol = tol;
  reset_accounting(c);
  SPCG_CK(cudaEventRecord(c->ev[0], c->stream));
  const bool have = reuse && c->sk.ready && c->sk.seed == seed &&
                    c->sk.sched.sketch == SPCG_SKETCH_SRHT && c->sk.sched.K == sc.K &&
                    (sc.K == 0 || c->sk.sched.m[sc.K - 1] == sc.m[sc.K - 1]);
  if (!have) {
    SPCG_TRY(sketch_after_split(c, seed, &sc));   // the prefix holds N'/2 rows: every candidate fits
  }
  SPCG_CK(cudaEventRecord(c->ev[1], c->stream));
  SPCG_CK(cudaMemsetAsync(c->beta_work, 0, (size_t)c->d * 8, c->stream));
  SPCG_TRY(launch_reset_flags(c));   // the reused sketch may follow a failed call
  int idx = paper;
  spcg_schedule cand = sc;
  if (sc.K > 0) {
    SPCG_TRY(run_stage(c, 0, 3, c->beta_work));
    if (force_idx >= 0) {
      idx = force_idx;
    } else if (Wb && norm && n_out == 25) {
      float f[4];
      SPCG_TRY(spcg_features(c, c->beta_work, f));
      float xn[4];
      for (int k = 0; k < 4; ++k) xn[k] = (f[k] - norm[k]) / norm[4 + k];
      SPCG_CK(cudaMemcpyAsync(c->mlp_x, xn, sizeof(xn), cudaMemcpyHostToDevice, c->stream));
      SPCG_TRY(mlp_forward_launch(Wb, n_out, c->mlp_x, 1, c->mlp_y, c->stream));
      c->n_launch += 1;
      float y[25];
      SPCG_CK(cudaMemcpyAsync(y, c->mlp_y, sizeof(y), cudaMemcpyDeviceToHost, c->stream));
      SPCG_CK(cudaStreamSynchronize(c->stream));
      bool ok = true;
      int best = 0;
      for (int k = 0; k < 25; ++k) {
        if (!isfinite(y[k])) ok = false;
        if (y[k] < y[best]) best = k;
      }
      if (ok) idx = best;
    }
    SPCG_TRY(spcg_candidate_schedule(c->N, c->d, idx, &cand));
    for (int i = 1; i < cand.K; ++i) SPCG_TRY(run_stage_m(c, cand.m[i], cand.a[i], c->beta_work));
  }
  SPCG_TRY(sync_scalars(c));
  SPCG_CK(cudaEventRecord(c->ev[2], c->stream));
  RefineResult rr;
  spcg_status st = run_refine(c, tol, sc.max_iters, sc.max_restarts, c->beta_work, &rr);
  SPCG_CK(cudaEventRecord(c->ev[3], c->stream));
  SPCG_CK(cudaMemcpyAsync(beta, c->beta_work, (size_t)c->d * 8, cudaMemcpyDeviceToDevice,
                          c->stream));
  SPCG_CK(cudaStreamSynchronize(c->stream));
  SPCG_TRY(prof_collect(c));
  if (choice) *choice = idx;
  if (info) {
    info->K = cand.K;
    for (int i = 0; i < cand.K; ++i) info->stage_iters[i] = cand.a[i];
    info->refine_iters = rr.iters;
    info->restarts = rr.restarts;
    info->converged = rr.converged;
    info->sqrt_gamma = c->host_scal.sqrt_gamma;
    info->norm_R_beta = c->host_scal.norm_rb;
    info->bytes_pass = c->pass_bytes;
    info->cond_est = c->cond_est;
    info->inner_prec = c->inner_used;
    info->grad_prec = c->grad_used;
    info->pass_launches = (int32_t)c->n_pass;
    info->launches = (int32_t)c->n_launch;
    info->pass_ms = c->prof_ms;
    for (int k = 0; k < 4; ++k) {
      info->pass_ms_by_op[k] = c->prof_ms_op[k];
      info->bytes_by_op[k] = c->pass_bytes_op[k];
      info->launches_by_op[k] = (int32_t)c->n_pass_op[k];
    }
    float ms;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    info->ms_sketch = ms;
    cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]);
    info->ms_stages = ms;
    cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
    info->ms_refine = ms;
  }
  return st;
}

extern "C" spcg_status spcg_solve_learned(spcg_ctx* c, uint64_t seed, const uint16_t* Wb,
                                          int32_t n_out, const float* norm, double tol,
                                          double* beta, spcg_info* info, int32_t* choice) {
  return solve_choice(c, seed, Wb, n_out, norm, tol, -1, 0, beta, info, choice);
}

extern "C" spcg_status spcg_solve_candidate(spcg_ctx* c, uint64_t seed, int32_t idx, double tol,
                                            int32_t reuse_sketch, double* beta, spcg_info* info) {
  if (idx < 0 || idx >= 25) return SPCG_E_INVALID_ARG;
  return solve_choice(c, seed, nullptr, 0, nullptr, tol, idx, reuse_sketch, beta, info, nullptr);
}
