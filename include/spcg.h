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
 *   - With SPCG_NVTX=1 in the environment (read once per process) the
 *     library marks the phases of a solve with NVTX ranges named
 *     spcg_solve, spcg_sketch, spcg_transform (or spcg_countsketch),
 *     spcg_precond, "spcg_stage i" and spcg_refine, for a profiler to group
 *     kernel launches by; without an attached tool the ranges cost nothing.
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
  SPCG_PREC_FP64 = 0,       /* plain FP64 everywhere (the comparator path)    */
  SPCG_PREC_MIXED = 1       /* Stage I reads a BF16 copy of the sketched rows
                               with FP32 accumulation; Stage II iterates on an
                               FP32 copy Xh of X (FP32 row dot products, row
                               sums folded into TwoSum-compensated accumulators)
                               or, when the condition estimate
                               says FP32 rows are too coarse (see
                               spcg_opts.inner_prec), on the double-FP32 split
                               X = Xh + Xl (|X - Xh - Xl| <= 2^-48 |X|); every
                               true gradient X^T (Y - X beta) that the stopping
                               rule trusts is computed in double-FP32 from that
                               split or, for ill-conditioned X, by an FP64 pass
                               (spcg_opts.grad_prec); the sketch, the QR giving
                               R, R^{-1} and the CG scalars stay FP64          */
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
  int32_t sketch;           /* SPCG_SKETCH_SRHT or SPCG_SKETCH_COUNT          */
} spcg_schedule;

/* Sketching operator of the initialisation (spcg_schedule.sketch). */
enum {
  SPCG_SKETCH_SRHT = 0,     /* nested SRHT (Sec. 2.1, Sec. 2.2)               */
  SPCG_SKETCH_COUNT = 1     /* CountSketch, SPCG-CS (Sec. 4.3): one hash into
                               m_K buckets folded modulo m_i for stage i (all
                               m_i powers of two), an independent r-bucket
                               CountSketch for the preconditioner              */
};

typedef struct {
  int32_t precision;        /* SPCG_PREC_*                                     */
  int32_t grid_ctas;        /* CTAs of the fused pass; 0 = one per SM          */
  int64_t spin_budget;      /* clock cycles a device-side wait may spin before
                               it gives up with SPCG_E_TIMEOUT; 0 = 2^31       */
  int32_t inject_stall;     /* test hook: 1 = the first CTA of every fused pass
                               never issues its first row tile, so its wait
                               runs out (SPCG_E_TIMEOUT) without any fault      */
  int32_t profile;          /* 1 = time every fused pass with CUDA events      */
  int32_t inner_prec;       /* SPCG_PREC_MIXED only: operand of the Stage II
                               iterations, SPCG_INNER_*; 0 = automatic        */
  int32_t grad_prec;        /* SPCG_PREC_MIXED only: arithmetic of the true
                               gradients, SPCG_GRAD_*; 0 = automatic          */
  int64_t max_workspace_bytes; /* cap on the device memory the context may hold
                               (its workspace, without the caller's X, Y and
                               beta); an allocation by spcg_create or
                               spcg_sketch that would pass it fails with
                               SPCG_E_OOM before any cudaMalloc; 0 = no cap   */
  int32_t qr_by_column;     /* preconditioner QR: 0 = blocked, with look-ahead
                               from d = 256 on (a panel group factors panel p
                               while the other CTAs apply panel p-1 to the
                               later columns), 1 = one launch per Householder
                               step, 2 = blocked without look-ahead (same
                               factorisation; 1 and 2 for comparison)          */
  int32_t fwht_tile;        /* transform passes of 9..12 levels: 0 = default
                               (the per-round pass kernel, as 3), 1 = 128 KB
                               tiles, one CTA per SM, 2 = 64 KB tiles, two CTAs
                               per SM (9 or 10 levels; others as 1), 3 = the
                               per-round pass kernel; all give the same bits  */
  int32_t fwht_first_levels; /* levels of the first of two transform passes;
                               0 = split evenly, except that the last pass
                               gets 9 levels where the first then has at
                               most 11 (N' = 2^20: 11 + 9)                    */
  int32_t qr_panel_ctas;    /* CTAs that factor each 32-column panel of the
                               preconditioner QR; 0 = about 30000 / d, at most
                               half the grid (with look-ahead), or one per 48
                               rows of the sketch (without)                    */
  int32_t dspace_ctas;      /* CTAs of the per-iteration d-space step (alpha,
                               g, beta, z = R^{-1} R^{-T} g and its dots, one
                               cooperative launch); 0 = about one per 8
                               columns; at most one per SM and one per column */
} spcg_opts;

/* Stage II operand of the mixed path (spcg_opts.inner_prec, spcg_info.inner_prec).
 * Automatic choice: with nu the power-iteration estimate of ||D R^{-1}||_2,
 * D = diag(||R e_j||) (spcg_info.cond_est), FP32 rows when 2^-24 nu <= 1/32,
 * else the double-FP32 pair.  FP32 rounding perturbs the preconditioned
 * operator by about 2^-24 nu; refinement on true gradients contracts only
 * while that stays well below one. */
enum {
  SPCG_INNER_AUTO = 0,
  SPCG_INNER_F32 = 1,       /* Xh, compensated FP32 (4 bytes per element)     */
  SPCG_INNER_DF = 2         /* Xh + Xl in double-FP32 (8 bytes per element)   */
};

/* True gradients X^T (Y - X beta) of the mixed path (spcg_opts.grad_prec,
 * spcg_info.grad_prec).  The stopping rule compares sqrt(g^T H-hat^{-1} g)
 * with (tol/2) ||R beta||, and an error in g reaches that metric amplified by
 * up to nu.  Automatic choice: the double-FP32 pass (about 2^-48 relative per
 * term, read at memory speed) while 2^-48 nu <= tol/64, else the FP64 pass. */
enum {
  SPCG_GRAD_AUTO = 0,
  SPCG_GRAD_F64 = 1,        /* FP64 pass over X                                */
  SPCG_GRAD_DF = 2          /* double-FP32 pass over Xh + Xl                   */
};

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
  double cond_est;          /* mixed path: estimate of ||D R^{-1}||_2 (above);
                               0 on the FP64 path                              */
  int32_t inner_prec;       /* mixed path: SPCG_INNER_F32 or SPCG_INNER_DF as
                               used by Stage II; 0 on the FP64 path            */
  int32_t grad_prec;        /* SPCG_GRAD_F64 or SPCG_GRAD_DF: the arithmetic of
                               the true gradients of Stage II                  */
  /* The fused passes split by operand: [0] FP64 rows, [1] FP32 rows, [2] BF16
   * rows, [3] the double-FP32 pair (8 bytes per element).  Times only when
   * spcg_opts.profile = 1, else 0. */
  double pass_ms_by_op[4];
  uint64_t bytes_by_op[4];
  int32_t launches_by_op[4];
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
 * The tuned schedule of Sec. 4.3: for N = 2^22, d = 2^6 the paper uses
 * m_i = 2^10, ..., 2^16 followed by a single 2^20 subproblem and a_i = 4.
 * Generalised: m_1 = 2^ceil(log2 16d), at most seven doublings below N'/4,
 * then one transition stage of N'/4 rows; r = 6d; tol, limits as the default.
 * Host-only.  Errors: SPCG_E_INVALID_ARG as spcg_default_schedule.
 */
spcg_status spcg_tuned_schedule(int64_t N, int32_t d, spcg_schedule* out);

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
 * Errors: SPCG_E_INVALID_ARG (a pointer, size or option out of its
 * documented range; found before any CUDA call), SPCG_E_OOM (a device
 * allocation failed, or the workspace would pass opts->max_workspace_bytes),
 * SPCG_E_CUDA.
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
 * Errors: SPCG_E_INVALID_ARG (schedule), SPCG_E_OOM (a device allocation
 * failed or would pass spcg_opts.max_workspace_bytes), SPCG_E_CUDA,
 * SPCG_E_BREAKDOWN (X or Y holds an Inf or a NaN, found by the column maxima
 * of the fixed-point scales; or R has a zero or non-finite diagonal entry).
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

/*
 * Capture-safe Stage I + Stage II: enqueue every launch of the solve on the
 * context's stream without reading anything back, so that the sequence can be
 * captured into a CUDA graph and replayed.  Requires a prior spcg_sketch
 * (which synchronises; call it outside the capture).  beta (device, d, output)
 * is set to 0 and run through all K stages; Stage II then runs `rounds`
 * rounds of [true gradient X^T (Y - X beta) and the stopping test; at most
 * iters_per_round PCG iterations with the recursive test], then one more
 * true-gradient test.  The stopping state lives on the device: once the
 * recursive test holds, the rest of a round does nothing; the next true
 * gradient either confirms it (every later launch then does nothing) or the
 * iterations go on from it.  The schedule is sized by the caller: rounds
 * bounds the restarts, rounds x iters_per_round the Stage II iterations.
 * spcg_opts.profile must be 0.  Nothing is allocated.
 * Errors: SPCG_E_INVALID_ARG, SPCG_E_STATE (no sketch), SPCG_E_CUDA.
 */
spcg_status spcg_solve_enqueue(spcg_ctx* ctx, double* beta, int32_t rounds,
                               int32_t iters_per_round);

/*
 * The outcome of the last spcg_solve_enqueue sequence (synchronises the
 * stream): SPCG_OK when the stopping rule was confirmed on a true gradient,
 * SPCG_E_NOT_CONVERGED when the schedule ran out first, or the device error
 * (SPCG_E_BREAKDOWN, SPCG_E_TIMEOUT).  info (host, may be NULL):
 * refine_iters = Stage II iterations that ran, converged, sqrt_gamma,
 * norm_R_beta, the precision choices; launch counts are those enqueued.
 */
spcg_status spcg_solve_result(spcg_ctx* ctx, spcg_info* info);

/*
 * Algorithm 1 end to end from HOST memory: copies X and Y to the device,
 * solves as spcg_solve, copies beta back.  For callers that hold the problem
 * in host memory and want one call; the copies are part of the call.
 *   X      host, N x d row-major FP64, leading dimension ldx >= d (page-locked
 *          memory, e.g. cudaHostAlloc, makes the copy run at full link speed)
 *   Y      host, N FP64
 *   sched  NULL = spcg_default_schedule(N, d); opts NULL = defaults
 *   stream cudaStream_t for the copies and the solve (NULL = default stream)
 *   beta   host, d FP64 output (the last iterate when SPCG_E_NOT_CONVERGED)
 *   info   host, may be NULL
 * The device copies of X (N x d, rows padded to an even count), Y and beta
 * and the context's workspace come from a stream-ordered memory pool that the
 * library keeps per device: freed at the end of the call, the memory stays in
 * the pool for the next call (of any size) instead of going back to the
 * device, so repeated calls skip the allocation cost.  spcg_host_pool_trim
 * hands it back.  Synchronises `stream`.  Errors: SPCG_E_INVALID_ARG (as
 * spcg_create, found before any CUDA call), SPCG_E_OOM, SPCG_E_CUDA and those
 * of spcg_solve.
 */
spcg_status spcg_solve_host(const double* X, const double* Y, int64_t N, int32_t d, int64_t ldx,
                            uint64_t seed, const spcg_schedule* sched, const spcg_opts* opts,
                            void* stream, double* beta, spcg_info* info);

/* Return the memory kept by spcg_solve_host's pools to the devices (every
 * device that has one).  Call when no spcg_solve_host is running.  Errors:
 * SPCG_E_CUDA. */
spcg_status spcg_host_pool_trim(void);

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
 * Copy rows [row0, row0 + nrows) of the last (largest) stage's sketched pair
 * after spcg_sketch:
 *   A  device, nrows x d row-major (leading dimension d)
 *   b  device, nrows (may be NULL)
 * SRHT: row t is Z[pi(t), :] with Z = H D P [X; 0] normalised by 1/sqrt(N');
 * stage i's pair is sqrt(N'/m_i) times rows [0, m_i), a scale that leaves the
 * PCG iterates unchanged.  CountSketch: row t is bucket t of S_K [X Y].
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
 * The same pass on an FP32 (dtype 1) or BF16 (dtype 2) operand, the element
 * types the mixed-precision path streams (dtype 0 = FP64 as above).  FP32 rows
 * form each row's dot product in FP32 and fold the row sums into a
 * TwoSum-compensated accumulator; BF16 rows use plain FP32; the products with p use p rounded to FP32.  dtype 3 is the
 * double-FP32 pair A = Ah + Al: the m x lda FP32 block Ah followed directly
 * by the m x lda FP32 block Al (so Al starts at (float*)A + m * lda), with p
 * split into an FP32 pair and every product and sum in double-FP32
 * (TwoProd/TwoSum).  lda * element size (4 for dtype 3) must be a multiple
 * of 16 bytes.  p, w: device FP64.
 */
spcg_status spcg_gram_apply_typed(spcg_ctx* ctx, const void* A, int32_t dtype, int64_t m,
                                  int64_t lda, const double* p, double* w);

/*
 * The residual-mode pass, the true gradient of Sec. 2.2's stopping rule on
 * caller data: g = A^T (b - A x), reading A once.  A and dtype as for
 * spcg_gram_apply_typed (0 FP64, 1 FP32, 2 BF16, 3 double-FP32 pair); b:
 * device m (FP64), x, g: device d (FP64).  FP64 rows compute in FP64; FP32
 * and BF16 rows form b - a.x and accumulate in FP32 (FP32 rows with the
 * compensated sums of spcg_gram_apply_typed); the pair in double-FP32 with b
 * and x split into FP32 pairs.  m = 0 gives g = 0.
 */
spcg_status spcg_resid_apply_typed(spcg_ctx* ctx, const void* A, int32_t dtype, int64_t m,
                                   int64_t lda, const double* b, const double* x, double* g);

/*
 * The double-FP32 split the mixed form streams: Xh = fl32(X) and
 * Xl = fl32(X - Xh), both rounded to nearest even, so |X - Xh - Xl| <= 2^-48 |X|
 * for |X| in [2^-74, 2^127).  X: device N x d FP64, row-major, leading
 * dimension ldx (even, X 16-byte aligned); Xh, Xl: device N x d FP32 outputs
 * with leading dimension ldxf (even, 8-byte aligned), columns d.. untouched.
 * Runs on `stream` and synchronises it.  SPCG_E_INVALID_ARG on a bad size,
 * stride or alignment; N = 0 does nothing.
 */
spcg_status spcg_split_f32(const double* X, int64_t N, int32_t d, int64_t ldx, float* Xh,
                           float* Xl, int64_t ldxf, void* stream);

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
 * device current; a failed lookup is retried by the next call.  All calls share
 * the array: calls that overlap on the GPU race and may return wrong results.
 * Errors: SPCG_E_INVALID_ARG, SPCG_E_CUDA, SPCG_E_TIMEOUT.
 */
spcg_status spcg_gram_apply_noalloc(const double* A, int64_t m, int32_t d, int64_t lda,
                                    const double* p, double* w, void* stream);

/*
 * Measurement helper (the paper has no counterpart): the fused multiply-add
 * rate of this GPU for one arithmetic type, measured by a kernel that does
 * nothing but independent FMA chains on every SM, timed with CUDA events on
 * `stream` after a warm-up launch.  The plain FP64 fused pass is bound by FP64
 * FMA issue, so this measured rate is its roofline denominator.
 *   dtype       0 = FP64, 1 = FP32
 *   iters       FMA steps per chain (about 2^16 takes a few milliseconds)
 *   tflops_out  host: 2 x FMAs / elapsed seconds / 1e12
 * Synchronises `stream`.  Errors: SPCG_E_INVALID_ARG (dtype, iters < 1, NULL
 * output), SPCG_E_CUDA.
 */
spcg_status spcg_probe_fma_tflops(int32_t dtype, int32_t iters, double* tflops_out, void* stream);

/* ----- Batched solver: many independent FP32 problems, one persistent kernel ----- */

/* One problem of a batch (all pointers device, caller-owned). */
typedef struct {
  const float* X;           /* N x d row-major FP32 in an allocation of N * ldx
                               floats (rows are read whole), ldx*4 % 16 == 0,
                               16-byte aligned                                    */
  const float* Y;           /* N FP32                                              */
  int64_t N;                /* d < N <= 2^24                                       */
  int32_t d;                /* 1 <= d <= 256                                       */
  int64_t ldx;
  double* beta;             /* output, d FP64                                      */
} spcg_problem_f32;

typedef struct spcg_batch spcg_batch;

/*
 * Prepare a batch of n problems (the array is copied; the buffers it points
 * to are borrowed until spcg_batch_destroy).  Each problem is solved by SPCG
 * with the CountSketch initialisation (SPCG-CS, Sec. 4.3), the paper's
 * default sizes (m_1 = 2^ceil(log2 8d) doubling to N'/2, r = 6d, a_i = 3) and
 * the Stage II stopping rule.  One persistent kernel solves the whole batch:
 * each CTA runs complete solves, taking problems largest first from a work
 * queue.  Allocates the per-CTA scratch (sized by the largest problem).
 * The problem's sketch draws use key seed + (index in the array).
 */
spcg_status spcg_batch_create(const spcg_problem_f32* probs, int32_t n, void* stream,
                              spcg_batch** out);
void spcg_batch_destroy(spcg_batch* b);

/*
 * Solve the batch (a captured CUDA graph: queue reset + the persistent
 * kernel, re-captured when seed, tol or the tiles change).  status_out,
 * iters_out: host arrays of n (may be NULL), in the order of the problems
 * given to spcg_batch_create (0 ok, 4 breakdown, 5 not converged, 6 timeout);
 * ms_out: host, device time of the graph.  Returns the first non-zero status.
 */
spcg_status spcg_batch_solve(spcg_batch* b, uint64_t seed, double tol, int32_t* status_out,
                             int32_t* iters_out, double* ms_out);

/* The whole batch in one call: spcg_batch_create, spcg_batch_solve,
 * spcg_batch_destroy (the per-CTA scratch is allocated and freed inside).
 * status_out, iters_out: host arrays of n, may be NULL.  Returns the first
 * non-zero per-problem status, or the error of a failed create. */
spcg_status spcg_solve_batched(const spcg_problem_f32* probs, int32_t n, uint64_t seed,
                               double tol, void* stream, int32_t* status_out,
                               int32_t* iters_out);

/* Clock cycles (of the SM that solved it) spent by each problem of the last
 * spcg_batch_solve in its phases: [0] column maxima, [1] CountSketch row maps
 * (bucket sizes, offsets, row lists), [2] CountSketch bucket sums, [3] stage
 * matrices, [4] preconditioner QR and R^{-1}, [5] Stage I, [6] Stage II; [7]
 * zero.  cycles_out: host, 8 n int64 in the order of the problems given to
 * spcg_batch_create. */
spcg_status spcg_batch_phase_cycles(spcg_batch* b, int64_t* cycles_out);

/* Rows per streamed chunk, as chunk bytes per width class (d <= 32, <= 64,
 * <= 128, <= 256): 0 = 16 KB, else a multiple of 16 in [1024, 16384]. */
spcg_status spcg_batch_set_tiles(spcg_batch* b, const int32_t* chunk_bytes4);

/* The autotuner: times the batch with 4, 8 and 16 KB chunks per width class
 * and keeps the fastest; chosen4 (host, may be NULL) receives the choice. */
spcg_status spcg_batch_autotune(spcg_batch* b, uint64_t seed, double tol, int32_t* chosen4);

/* ----- Learned schedule (Sec. 4.3 leaves the
 * automatic choice of the sketch-size schedule open) ----- */

/* Number of candidate schedules the model scores (25). */
int32_t spcg_num_candidates(void);

/*
 * Candidate schedule idx (0 <= idx < 25) for an N x d problem.  Stage 1 is
 * always the paper's (m_1 = 2^ceil(log2 8d), a_1 = 3), so that its noise
 * estimate is available before the choice.  idx 0: no further stage.
 * idx = 1 + 6 (g - 1) + 3 (s - 1) + (a - 2) for g in 1..4, s in 1..2,
 * a in 2..4: stages m_1 2^s, m_1 2^{2s}, ... up to N'/2^g with a iterations
 * each.  idx 2 (g = 1, s = 1, a = 3) is the paper's schedule.  r, tol and the
 * limits are those of spcg_default_schedule.  Host-only.
 */
spcg_status spcg_candidate_schedule(int64_t N, int32_t d, int32_t idx, spcg_schedule* out);

/*
 * The model's four features after spcg_sketch (SRHT) and stage 1 (beta =
 * the stage-1 iterate, device): log2 N, log2 d, log10(max R_ii / min R_ii),
 * log10(||b_1 - A_1 beta||^2 / ||b_1||^2).  out4: host.
 */
spcg_status spcg_features(spcg_ctx* ctx, const double* beta, float* out4);

/*
 * Algorithm 1 with the schedule chosen by the model: sketch, stage 1 (paper
 * default), features, the network's predicted log-cost of every candidate,
 * the remaining stages of the cheapest candidate, Stage II to tol.
 *   Wb     device, BF16 weights (layout of spcg_mlp_forward), n_out = 25;
 *          NULL falls back to the paper's schedule, as do non-finite outputs
 *   norm   host, 8 floats: feature means (4) then standard deviations (4)
 *   beta   device output; choice (host, may be NULL): the candidate used
 */
spcg_status spcg_solve_learned(spcg_ctx* ctx, uint64_t seed, const uint16_t* Wb, int32_t n_out,
                               const float* norm, double tol, double* beta, spcg_info* info,
                               int32_t* choice);

/*
 * The same solve with a fixed candidate idx (0 <= idx < 25), for measuring
 * candidate costs.  reuse_sketch = 1 keeps the context's sketch when it was
 * made with the same seed by a previous call (X must be unchanged), so that
 * spcg_info's stage and Stage II times are measured without a new sketch.
 */
spcg_status spcg_solve_candidate(spcg_ctx* ctx, uint64_t seed, int32_t idx, double tol,
                                 int32_t reuse_sketch, double* beta, spcg_info* info);

/*
 * The MLP 4 -> 64 -> 64 -> n_out (ReLU) with BF16 weights and FP32 arithmetic.
 * Parameter layout (n_params = 4480 + 65 n_out): W1 (64 x 4 row-major), b1
 * (64), W2 (64 x 64), b2 (64), W3 (n_out x 64), b3 (n_out).  1 <= n_out <= 64.
 */
int64_t spcg_mlp_params(int32_t n_out);
/* Floats of workspace spcg_mlp_grad needs for a batch of B samples. */
int64_t spcg_mlp_workspace_floats(int32_t n_out, int64_t B);
/* y (device, B x n_out) = MLP(x) for x (device, B x 4); Wb device BF16. */
spcg_status spcg_mlp_forward(const uint16_t* Wb, int32_t n_out, const float* x, int64_t B,
                             float* y, void* stream);
/*
 * Loss = mean over the batch and outputs of (MLP(x) - t)^2 and its gradient
 * with respect to the (BF16) weights: grad (device, n_params FP32), loss
 * (device, 1 FP32, may be NULL); workspace: device, spcg_mlp_workspace_floats.
 * Per-block sums are added in a fixed order (reproducible).
 */
spcg_status spcg_mlp_grad(const uint16_t* Wb, int32_t n_out, const float* x, const float* t,
                          int64_t B, float* grad, float* loss, float* workspace, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master theta;
 * writes the BF16 copy Wb.  step counts from 1. */
spcg_status spcg_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t P,
                          float lr, int32_t step, uint16_t* Wb, void* stream);
/* Wb = BF16(theta), round to nearest even. */
spcg_status spcg_mlp_to_bf16(const float* theta, int64_t P, uint16_t* Wb, void* stream);

#ifdef __cplusplus
}
#endif
#endif
