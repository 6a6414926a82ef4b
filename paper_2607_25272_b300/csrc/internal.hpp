// Host-side internals shared by the translation units of the SPCG library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <unordered_map>

#include "../../include/spcg.h"

namespace spcg {

// Device scalars of one context (one allocation, zeroed at create).
struct DevScalars {
  int status;        // DEV_* error code, sticky until the next spcg_* call
  int done;          // 0 iterating; 1 the recursive stopping test passed (pass
                     // prologue); 2 confirmed on a true gradient (k_check)
  int iters;         // PCG iterations that ran a pass since the last reset
  int pad;
  double gam[2];     // gamma ping-pong
  double sqrt_gamma; // last check: sqrt(gamma)
  double norm_rb;    // last check: ||R beta||
  double cond;       // estimate of ||D R^{-1}||_2 (condest.cu)
};

// Element types of a fused-pass operand.
enum : int { DT_F64 = 0, DT_F32 = 1, DT_BF16 = 2 };
// Operand kinds of the pass accounting (spcg_info.*_by_op): the three
// element types and the double-FP32 pair.
enum : int { OP_F64 = 0, OP_F32 = 1, OP_BF16 = 2, OP_PAIR = 3 };

// Geometry of the fused pass over one operand.
struct PassGeom {
  int64_t m;     // rows
  int d;         // columns
  int dtype;     // DT_*
  int esize;     // bytes per element
  int nbox;      // TMA boxes across a row
  int boxc;      // columns per box (even)
  int tm;        // rows per tile (box height)
  int ntiles;
  int stages;
  size_t stage_bytes;
  size_t region_bytes;  // staging region (>= stages * stage_bytes and the reduction scratch)
  size_t smem_bytes;
  CUtensorMap tmap;
};

struct PcgBuffers {
  double* partials;  // grid x ldp
  int ldp;
  int grid;          // CTAs of the fused pass
  double* w;
  double* u;
  double* z;
  double* g[2];
  double* p[2];
  double* dots_pw;   // per reduce CTA
  double* dots_gz;   // per precond CTA
  double* dots_rb;
  int n_red;         // CTAs of the reduce kernel
  int n_pre;         // (d + 3) / 4: sizes the per-CTA dot arrays
  int n_ds;          // CTAs of k_dspace (= shares in dots_pw, dots_gz, dots_rb)
  int last_grid;     // CTAs of the last fused pass (= partials to reduce)
};

struct Sketch {
  bool ready = false;
  bool colmax_pre = false;   // colmax already holds this call's maxima (fused split)
  uint64_t seed = 0;
  spcg_schedule sched{};
  int64_t n_pad = 0;
  int nbits = 0;
  // random maps (N' entries)
  uint32_t* gather = nullptr;   // P(j) | sign bit
  int32_t* dest = nullptr;      // pi^{-1}(j) if < m_K else -1
  int32_t* hdest = nullptr;     // sigma_hat^{-1}(j) if < r else -1
  double* work = nullptr;       // N' x ldw int64 transform buffer (multi-pass only)
  int64_t ldw = 0;
  size_t work_bytes = 0;
  double* AK = nullptr;         // m_K x ldak sketched prefix (pi order), FP64 mode
  int64_t ldak = 0;
  uint16_t* AK16 = nullptr;     // m_K x ldak16 BF16 prefix, mixed mode
  int64_t ldak16 = 0;
  int64_t mK16_alloc = 0;
  double* bK = nullptr;         // m_K
  int64_t mK_alloc = 0;
  double* Ahat = nullptr;       // r x d column-major (ld = r), QR in place
  int64_t r_alloc = 0;
  double* Rdiag = nullptr;      // d
  double* R = nullptr;          // d x d row-major upper
  double* Rinv = nullptr;       // d x d row-major upper
  double* RinvT = nullptr;      // d x d row-major lower (R^{-T})
  // scratch of the cooperative blocked QR (qr.cu), sized at create for one CTA per SM
  double* qr_vdiag = nullptr;   // d: first entry v_0 of each Householder vector
  double* qr_red = nullptr;     // 2 x SMs x (2 x panel width): per-CTA partial sums
  double* qr_wp = nullptr;      // SMs x panel width x d: per-CTA partials of V^T C
  double* qr_wt = nullptr;      // panel width x d: T^T V^T C
  double* qr_tg = nullptr;      // 2 x panel width^2: T of the current (and previous) panel
  double* qr_wl = nullptr;      // (SMs + 1) x panel width^2: look-ahead partials of V^T C
  unsigned* qr_bar = nullptr;   // 3 barriers of kBarWords (grid, panel group, update group)
  unsigned long long* colmax = nullptr;  // d + 1: largest |x| per column (bit pattern)
  int* colshift = nullptr;      // d + 1: fixed-point scale exponent per column
  PassGeom geom[SPCG_MAX_STAGES];  // fused-pass geometry of stage i
  int64_t stage_off[SPCG_MAX_STAGES];  // first row of stage i in AK/AK16/bK (SRHT: 0)
  int64_t rows_alloc = 0;              // rows of AK/AK16/bK
  bool mixed = false;             // prefix stored as BF16 (SPCG_PREC_MIXED)
};

}  // namespace spcg

struct spcg_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  spcg_opts opts{};
  int64_t N = 0;
  int d = 0;
  const double* X = nullptr;   // caller's (or our padded copy)
  int64_t ldx = 0;
  double* X_own = nullptr;
  const double* Y = nullptr;
  spcg::DevScalars* scal = nullptr;
  spcg::DevScalars host_scal{};
  spcg::PcgBuffers pb{};
  double* beta_work = nullptr;   // d
  spcg::Sketch sk;
  spcg::PassGeom gx{};           // pass geometry over X
  bool gx_ready = false;
  float* Xf = nullptr;           // FP32 copy of X (mixed precision): Xh = fl32(X)
  float* Xl = nullptr;           // FP32 remainder: Xl = fl32(X - Xh)
  spcg::PassGeom gxdf{};         // pass geometry over the pair (Xh, Xl)
  CUtensorMap tml{};             // tensor map of Xl for that pass
  float* mlp_x = nullptr;        // schedule-model input (4) and two feature scalars
  float* mlp_y = nullptr;        // schedule-model output (up to 64)
  double* feat_part = nullptr;   // feature partial sums
  int64_t ldxf = 0;
  spcg::PassGeom gxf{};          // pass geometry over Xf
  double cond_est = 0.0;         // mixed path: ||D R^{-1}||_2 estimate of the last sketch
  int inner_used = 0;            // mixed path: SPCG_INNER_* of the last Stage II
  int grad_used = 0;             // SPCG_GRAD_* of the last Stage II
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // launch accounting and optional per-pass event timing
  int64_t n_launch = 0;
  int64_t n_pass = 0;
  uint64_t pass_bytes = 0;
  // the same per operand kind (OP_*: FP64, FP32, BF16 rows, double-FP32 pair)
  int64_t n_pass_op[4] = {0, 0, 0, 0};
  uint64_t pass_bytes_op[4] = {0, 0, 0, 0};
  double prof_ms_op[4] = {0.0, 0.0, 0.0, 0.0};
  int* prof_op = nullptr;           // operand kind of each event pair
  cudaEvent_t* prof_ev = nullptr;   // pairs around fused-pass launches
  int prof_cap = 0;
  int prof_used = 0;
  double prof_ms = 0.0;
  // device workspace of this context (dalloc/dfree in api.cu); contexts made
  // by spcg_solve_host draw it from the library's stream-ordered pool
  cudaMemPool_t pool = nullptr;
  size_t ws_bytes = 0;
  std::unordered_map<const void*, size_t> ws_sizes;
};

namespace spcg {

// Error helpers --------------------------------------------------------------
spcg_status from_cuda(cudaError_t e);
#define SPCG_CK(call)                                         \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) return spcg::from_cuda(e__);      \
  } while (0)
#define SPCG_TRY(call)                                        \
  do {                                                        \
    spcg_status s__ = (call);                                 \
    if (s__ != SPCG_OK) return s__;                           \
  } while (0)

// rng.cu
spcg_status launch_sketch_maps(spcg_ctx* c);
// fwht.cu
spcg_status launch_transform(spcg_ctx* c);
// Split n index bits into transform passes of at most 12 bits; returns the
// number of passes and their levels in logl[] (first_levels > 0 fixes the
// first of a two-pass plan).
int fwht_pass_plan(int n, int* logl, int first_levels);
spcg_status launch_colscales(spcg_ctx* c);
// countsketch.cu
spcg_status launch_countsketch(spcg_ctx* c);
spcg_status launch_export_rows(spcg_ctx* c, int64_t row0, int64_t n, double* A, double* b);
spcg_status launch_to_f32(spcg_ctx* c);   // X -> Xf
spcg_status launch_to_f32_colmax(spcg_ctx* c);   // X -> Xf and the sketch's column maxima
// qr.cu
constexpr int kQrPanel = 32;   // panel width of the blocked QR
spcg_status launch_precond_factor(spcg_ctx* c);
// pcg.cu
spcg_status make_pass_geom(const double* A, int64_t m, int d, int64_t lda, PassGeom* g);
spcg_status make_pass_geom_t(const void* A, int64_t m, int d, int64_t lda, int dtype,
                             PassGeom* g);
spcg_status pass_resid(spcg_ctx* c, const PassGeom& g, const double* b, const double* x);
spcg_status pass_gram_iter(spcg_ctx* c, const PassGeom& g, int pp, int gp, int start,
                           int check, double tau);
spcg_status launch_reduce(spcg_ctx* c, double* out, const double* dotvec);
spcg_status launch_check(spcg_ctx* c, double tau);
int dspace_grid(const spcg_ctx* c);
spcg_status launch_dspace(spcg_ctx* c, int iter, int cur, int pp, int gp, double* beta);
spcg_status launch_reset_flags(spcg_ctx* c);   // also clears the device status
spcg_status launch_reset_loop(spcg_ctx* c);    // keeps the device status
spcg_status prof_events(spcg_ctx* c, cudaEvent_t* e0, cudaEvent_t* e1, int op);
spcg_status prof_collect(spcg_ctx* c);   // after a stream sync
spcg_status pass_gram_plain(spcg_ctx* c, const PassGeom& g, const double* p);
spcg_status make_pass_geom_df(const float* Xh, const float* Xl, int64_t m, int d, int64_t lda,
                              PassGeom* g, CUtensorMap* tml);
spcg_status pass_resid_df(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml,
                          const double* b, const double* x);
spcg_status pass_gram_plain_df(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml,
                               const double* p);
spcg_status pass_gram_iter_df(spcg_ctx* c, const PassGeom& g, const CUtensorMap& tml, int pp,
                              int gp, int start, int check, double tau);
// condest.cu
spcg_status launch_condest(spcg_ctx* c);   // -> DevScalars::cond

}  // namespace spcg
