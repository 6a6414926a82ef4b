/*
 * spcg.h - C ABI of the SPCG hot path on one NVIDIA B300 (sm_103a).
 *
 * SPCG (Sequential Preconditioned Conjugate Gradient) estimates the OLS
 * solution beta-hat = argmin_u ||Y - X u|| (Sec. 1, Eq. (ols)) of a tall
 * dense X (N x d, N >> d, full column rank) by Algorithm 1:
 *   - one nested SRHT of (X, Y) gives K sketched pairs (S_i X, S_i Y) with
 *     doubling sizes m_1 < ... < m_K (Sec. 2.1, Sec. 2.2);
 *   - an independent r-row sketch gives H-hat = R^T R, R from a Householder
 *     QR of S-hat X (Sec. 2.2; Sec. 4 applies H-hat "through a QR");
 *   - Stage I runs a_i PCG iterations on each sketched pair, warm-started;
 *   - Stage II runs PCG on (X, Y) until a stopping rule holds.
 *
 * Conventions for every call:
 *   - Pointers named "device" are CUDA device pointers on the current device;
 *     "host" pointers are ordinary host memory.
 *   - Matrices are row-major with a leading dimension (elements between the
 *     starts of consecutive rows), unless stated otherwise.
 *   - Work is ordered on the CUDA stream given to spcg_create (NULL = legacy
 *     default stream).  Calls that return a status depending on device results
 *     synchronise that stream before returning.
 *   - Every call returns a status and never aborts, throws or exits.
 *   - Device memory is allocated only by spcg_create and spcg_sketch (the
 *     context's workspace) and freed by spcg_destroy.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef SPCG_H
#define SPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spcg_ctx spcg_ctx;   /* opaque, owned by the library */

typedef enum {
  SPCG_OK = 0,
  SPCG_E_INVALID_ARG = 1,   /* bad size, null pointer, invalid schedule       */
  SPCG_E_OOM = 2,           /* a device allocation failed                     */
  SPCG_E_CUDA = 3,          /* a CUDA runtime/driver call failed              */
  SPCG_E_BREAKDOWN = 4,     /* p^T A^T A p <= 0, a non-finite value, or R
                               singular (X not of full column rank, Sec. 1)   */
  SPCG_E_NOT_CONVERGED = 5, /* Stage II hit its iteration or restart limit;
                               beta holds the last iterate                    */
  SPCG_E_TIMEOUT = 6,       /* a bounded device-side wait expired             */
  SPCG_E_STATE = 7          /* call out of order (e.g. a stage before a sketch) */
} spcg_status;

#define SPCG_MAX_STAGES 40
#define SPCG_MAX_D 1024

/* Arithmetic of the X^T(Xp) passes (spcg_opts.precision). */
enum {
  SPCG_PREC_FP64 = 0        /* plain FP64 everywhere (the comparator path)    */
};

/*
 * The sketch-size schedule of Algorithm 1.
 *   K        number of sketched subproblems (0 = plain full-data PCG)
 *   m[i]     sketch sizes with r < m[0] < m[1] < ... < m[K-1] <= N'/2, where
 *            N' = 2^ceil(log2 N) (rows are zero-padded to N', Sec. 2.1)
 *   a[i]     PCG iterations on subproblem i (a_i >= 1)
 *   r        rows of the preconditioner sketch S-hat (d <= r <= N')
 *   tol      Stage II target for the relative prediction error
 *            ||X(beta - beta-hat)|| / ||X beta-hat||.  Stopping rule:
 *            sqrt(g^T H-hat^{-1} g) <= (tol/2) ||R beta||, first on the
 *            recursively updated gradient, then confirmed on the true
 *            gradient X^T (Y - X beta)
 *   max_iters     Stage II iteration limit (the paper's budget is T = 100)
 *   max_restarts  how often Stage II may restart PCG from a recomputed true
 *                 gradient after the recursive test passed but the true one
 *                 did not
 */
typedef struct {
  int32_t K;
  int64_t m[SPCG_MAX_STAGES];
  int32_t a[SPCG_MAX_STAGES];
  int64_t r;
  double tol;
  int32_t max_iters;
  int32_t max_restarts;
} spcg_schedule;

typedef struct {
  int32_t precision;        /* SPCG_PREC_*                                     */
  int32_t grid_ctas;        /* CTAs of the fused pass; 0 = one per SM          */
  int64_t spin_budget;      /* clock cycles a device-side wait may spin before
                               it gives up with SPCG_E_TIMEOUT; 0 = 2^31       */
  int32_t inject_stall;     /* test hook: 1 = the first CTA of every fused pass
                               never issues its first row tile, so its wait
                               runs out (SPCG_E_TIMEOUT) without any fault      */
  int32_t profile;          /* 1 = time every fused pass with CUDA events      */
  int32_t reserved[2];
} spcg_opts;

typedef struct {
  int32_t K;
  int32_t stage_iters[SPCG_MAX_STAGES];
  int32_t refine_iters;     /* Stage II PCG iterations                         */
  int32_t restarts;         /* true-gradient recomputations after the first    */
  int32_t converged;        /* 1 if the stopping rule held on the true gradient */
  double sqrt_gamma;        /* sqrt(g^T H-hat^{-1} g) at exit (true gradient)  */
  double norm_R_beta;       /* ||R beta|| at exit                               */
  double ms_sketch, ms_stages, ms_refine;   /* device time per phase           */
  uint64_t bytes_pass;      /* algorithmic bytes of X/sketch read by the fused
                               passes (m_i d b per pass, b = element size)      */
  int32_t pass_launches;    /* fused-pass launches of this solve               */
  int32_t launches;         /* all kernel launches of this solve               */
  double pass_ms;           /* summed device time of the fused passes (CUDA
                               events around each launch; only when
                               spcg_opts.profile = 1, else 0)                  */
} spcg_info;

/* Human-readable name of a status code (static string, never NULL). */
const char* spcg_status_str(spcg_status s);

/*
 * The experimental schedule of Sec. 4 for an N x d problem: m_1 = 8d rounded
 * up to a power of two (Theorem 3.1 takes m_1 a power of two), m_{i+1} = 2 m_i,
 * m_K = N'/2, r = 6d, a_i = 3 (Sec. 4.1), tol = 1e-6, max_iters = 100,
 * max_restarts = 5.  K = 0 when m_1 > N'/2.  Host-only; makes no CUDA call.
 * Errors: SPCG_E_INVALID_ARG for out == NULL, d < 1, N <= d.
 */
spcg_status spcg_default_schedule(int64_t N, int32_t d, spcg_schedule* out);

/*
 * Create a solver context for the problem (X, Y) of Eq. (model).
 *   X      device, N x d row-major FP64 with leading dimension ldx >= d.
 *          Borrowed: must stay valid and unchanged until spcg_destroy.  If
 *          ldx*8 is not a multiple of 16 bytes (the TMA stride rule) the
 *          context keeps its own padded copy.
 *   Y      device, N FP64, borrowed likewise.
 *   N, d   1 <= d <= SPCG_MAX_D, d < N <= 2^30.
 *   stream cudaStream_t for all work of this context (NULL = default stream).
 *   opts   NULL for defaults.
 *   out    receives the context (set to NULL on failure).
 * Errors: SPCG_E_INVALID_ARG, SPCG_E_OOM, SPCG_E_CUDA.
 */
spcg_status spcg_create(const double* X, const double* Y, int64_t N, int32_t d,
                        int64_t ldx, void* stream, const spcg_opts* opts,
                        spcg_ctx** out);

/* Release the context and all its device memory (NULL is a no-op). */
void spcg_destroy(spcg_ctx* ctx);

/*
 * Build the nested sketches and the preconditioner (Sec. 2.2):
 *   Z = H D P [X Y; 0] (N' rows, H the normalised Sylvester Walsh-Hadamard
 *   matrix, D Rademacher signs, P a permutation), the nested rows
 *   I_K = {pi(t): t < m_K} stored contiguously in pi order so that stage i
 *   reads rows [0, m_i), and S-hat X = sqrt(N'/r) Z[I-hat] with its
 *   Householder factor R (diag(R) > 0), R^{-1} and R^{-T}.
 * The random draws (D, P, pi, I-hat) are Philox4x32-10 / Feistel
 * permutations keyed by seed, identical to spcg_feistel / spcg_signs.
 * sched NULL = spcg_default_schedule(N, d).  The schedule is copied.
 * Errors: SPCG_E_INVALID_ARG (schedule), SPCG_E_OOM, SPCG_E_CUDA,
 * SPCG_E_BREAKDOWN (R has a zero or non-finite diagonal entry).
 */
spcg_status spcg_sketch(spcg_ctx* ctx, uint64_t seed, const spcg_schedule* sched);

/*
 * Stage I step: a_i PCG iterations (Sec. 2.2) on subproblem i (0-based)
 * starting from beta, i.e. beta <- PCG(S_i X, S_i Y, H-hat, beta, a_i).
 *   beta  device, d FP64, in/out (caller-owned).
 * Errors: SPCG_E_STATE (no sketch yet), SPCG_E_INVALID_ARG (i out of range,
 * a_i < 0), SPCG_E_BREAKDOWN, SPCG_E_TIMEOUT, SPCG_E_CUDA.
 */
spcg_status spcg_pcg_stage(spcg_ctx* ctx, int32_t i, int32_t a_i, double* beta);

/*
 * Stage II: PCG on (X, Y) from beta until the stopping rule of spcg_schedule
 * holds for tol, or max_iters iterations.
 *   beta      device, d FP64, in/out.
 *   iters_out host, may be NULL: Stage II iterations used.
 * Errors: SPCG_E_STATE (no sketch), SPCG_E_NOT_CONVERGED, SPCG_E_BREAKDOWN,
 * SPCG_E_TIMEOUT, SPCG_E_CUDA.
 */
spcg_status spcg_refine(spcg_ctx* ctx, double tol, int32_t max_iters,
                        double* beta, int32_t* iters_out);

/*
 * Algorithm 1 end to end: spcg_sketch(seed, sched), beta <- 0, Stage I over
 * all K subproblems, Stage II to sched->tol.
 *   beta  device, d FP64, output.
 *   info  host, may be NULL.
 * Errors: as spcg_sketch, spcg_pcg_stage and spcg_refine.
 */
spcg_status spcg_solve(spcg_ctx* ctx, uint64_t seed, const spcg_schedule* sched,
                       double* beta, spcg_info* info);

/* ----- Lower-level entry points (same kernels; for parity checks) ----- */

/*
 * Philox4x32-10 (Salmon et al., SC'11) on n counters.
 *   ctr  device, 4*n uint32: counter j is ctr[4j .. 4j+3]
 *   out  device, 4*n uint32
 * key = (seed mod 2^32, seed >> 32).  Errors: SPCG_E_INVALID_ARG, SPCG_E_CUDA.
 */
spcg_status spcg_philox(const uint32_t* ctr, uint64_t seed, int64_t n,
                        uint32_t* out, void* stream);

/*
 * The Feistel permutation sigma_tag of [0, 2^nbits) keyed by seed (the draws
 * of P, pi and I-hat; tag 0 = P, 2 = pi, 3 = I-hat):
 *   out[t] = sigma_tag(t) (inverse = 0) or sigma_tag^{-1}(t) (inverse = 1)
 *   for t < count.  out: device int64.  0 <= nbits <= 30, count <= 2^nbits.
 */
spcg_status spcg_feistel(uint64_t seed, int32_t nbits, int32_t tag, int64_t count,
                         int32_t inverse, int64_t* out, void* stream);

/* Rademacher signs D_k (+1.0 / -1.0, FP64) for k < n: device out. */
spcg_status spcg_signs(uint64_t seed, int64_t n, double* out, void* stream);

/*
 * Copy rows [row0, row0 + nrows) of the sketched prefix after spcg_sketch:
 *   A  device, nrows x d row-major (leading dimension d): Z[pi(t), :]
 *   b  device, nrows (may be NULL): Z_Y[pi(t)]
 * (Z normalised by 1/sqrt(N'); stage i's pair is sqrt(N'/m_i) times rows
 * [0, m_i), a scale that leaves the PCG iterates unchanged.)
 */
spcg_status spcg_export_sketch(spcg_ctx* ctx, int64_t row0, int64_t nrows,
                               double* A, double* b);

/*
 * Copy the preconditioner after spcg_sketch: device outputs, each d x d
 * row-major, any may be NULL: R (upper, diag > 0), Rinv = R^{-1}, and
 * Ahat (r x d row-major, leading dimension d) = sqrt(N'/r) Z[I-hat, :].
 */
spcg_status spcg_export_precond(spcg_ctx* ctx, double* R, double* Rinv, double* Ahat);

/*
 * One fused pass of the hot loop on caller data: w = A^T (A p), reading A
 * once.  A: device m x d row-major FP64, lda >= d with lda*8 % 16 == 0 and A
 * 16-byte aligned; p, w: device d.  1 <= d <= SPCG_MAX_D, m >= 0 (m = 0 gives
 * w = 0).  Uses a context only for its workspace and stream.
 */
spcg_status spcg_gram_apply(spcg_ctx* ctx, const double* A, int64_t m, int64_t lda,
                            const double* p, double* w);

/*
 * Allocation-free form of spcg_gram_apply: w = A^T (A p) in one read of A,
 * with no context and no device allocation of any kind.  (The paper has no
 * counterpart; this entry point serves callers that cannot allocate device
 * memory, e.g. code running under a caching allocator that owns the device
 * pool, in a memory-capped sandbox, or where an allocation would force a
 * device-wide synchronisation.)
 *   A       device, m x d row-major FP64, lda >= d, lda*8 % 16 == 0, A 16-byte
 *           aligned (the TMA rules); m >= 0 (m = 0 gives w = 0)
 *   p, w    device, d FP64
 *   d       1 <= d <= SPCG_MAX_D (1024): the scratch holds partial sums for at
 *           most 1024 columns; larger d returns SPCG_E_INVALID_ARG
 *   stream  cudaStream_t; the call synchronises it before returning
 * Scratch: a fixed 1,310,976-byte __device__ array inside the library (per-CTA
 * partial sums for up to 160 CTAs x 1024 columns plus a status word), held by
 * every GPU that loads the library until the process exits.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current, so make the first call on each device outside any stream
 * capture.  All calls share the array: calls that overlap on the GPU race and
 * may return wrong results.
 * Errors: SPCG_E_INVALID_ARG, SPCG_E_CUDA, SPCG_E_TIMEOUT.
 */
spcg_status spcg_gram_apply_noalloc(const double* A, int64_t m, int32_t d, int64_t lda,
                                    const double* p, double* w, void* stream);

#ifdef __cplusplus
}
#endif
#endif
