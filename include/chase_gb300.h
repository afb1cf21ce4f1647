/*
 * chase_gb300.h -- C ABI of the GB300 (sm_103a) Chebyshev-filtered subspace
 * iteration library.
 *
 * The library computes the nev lowest eigenpairs of a dense Hermitian (or real
 * symmetric) matrix A of order n by the method of Di Napoli & Wu, "Estimating
 * the condition number of Chebyshev filtered vectors with application to the
 * ChASE library" (Algorithm 1): Chebyshev filter (Algorithm 4, per-column
 * degrees, Section 2.3), orthonormalisation of [Y V] by CholeskyQR1 /
 * CholeskyQR2 / shifted CholeskyQR2 chosen by the condition-number estimate of
 * Eq. full-est (Algorithm 3), Householder QR as the fallback, Rayleigh-Ritz,
 * residuals (eq. res) and locking.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with a leading dimension (LAPACK layout):
 *     element (i, j) of X lives at X[i + j*ldx].
 *   - CHASE_R64 data are `double`; CHASE_C128 data are interleaved complex
 *     doubles (`double _Complex` / `cuDoubleComplex`, 16 bytes, real first).
 *   - Pointers named d* are DEVICE pointers (on the handle's device);
 *     everything else is host memory.  The caller owns every buffer it passes
 *     and keeps it alive for the duration of the call.  The handle owns its
 *     workspace (device memory it allocates and grows on demand).
 *   - A is read in full (both triangles); the caller guarantees A = A^H.
 *   - All device work is ordered on the handle's CUDA stream; every entry point
 *     returns after that work has completed (it synchronises the stream).
 *   - Return value: CHASE_OK (0); a negative value -i means argument i (1-based,
 *     in the order of the C prototype) is invalid and nothing was done;
 *     positive values are the chase_status codes below.
 *   - No entry point traps or aborts: device-side failures (a non-positive
 *     Cholesky pivot, a non-finite value) are reported through status codes.
 *
 * Minimal use (dA: n x n Hermitian, dV: n x (nev + nex) start block, both on
 * device 0; error checks left out):
 *
 *   chase_handle h;
 *   chase_create(&h, 0, NULL);                  // the handle makes its own stream
 *   chase_config cfg;
 *   chase_config_default(&cfg);
 *   cfg.opt_degree = 1;                         // per-column degrees
 *   cfg.prec = CHASE_FP64_EMU;                  // FP64-accurate tensor-core products
 *   chase_stats st;
 *   int rc = chase_solve(h, CHASE_C128, n, dA, n, nev, nex, &cfg, NULL, dV, n,
 *                        evals, resid, &st, NULL, 0);   // bounds by Lanczos
 *   // rc == CHASE_OK: evals[0..nev) ascending, dV's first nev columns the vectors
 *   chase_destroy(h);
 */
#ifndef CHASE_GB300_H
#define CHASE_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chase_ctx* chase_handle;

typedef enum { CHASE_R64 = 0, CHASE_C128 = 1 } chase_dtype;

/* Arithmetic of the block products.
 *   CHASE_FP64      native FP64 (DFMA) everywhere.
 *   CHASE_FP64_EMU  every block product (filter A*V, Rayleigh-Ritz A*Q, Q^H(AQ), QW,
 *                   (AQ)W, and the QR's Gram X^H X and X R^{-1}) by the Ozaki scheme II
 *                   on the BF16 tensor cores: operands rounded to 57-bit integers (one
 *                   power-of-two scale per row / column), their product formed exactly
 *                   from 17 modular BF16 products (moduli <= 256) and the Chinese
 *                   remainder theorem, then rounded once to FP64; accurate to
 *                   ~2^-57 K max|A_m.| max|V_.c| per entry, the class of an FP64 product
 *                   (inner dimension up to 2^17: complex n <= 65536, real n <= 131072).
 *                   Complex A*V and A*Q run as three real products (A_r V_r, A_i V_i,
 *                   (A_r + A_i)(V_r + V_i)) of the same integers: the same results as one
 *                   product of the stacked real operator, for 3/4 of its work.
 *   CHASE_BF16X3    mixed: BF16x3 filter products (three BF16 tensor-core
 *                   products of hi/lo splits, FP32 accumulation) while the
 *                   residuals are large, then as CHASE_FP64_EMU.
 * The Cholesky factor, its inverse, Householder QR, the Jacobi eigensolver and the
 * residual norms are FP64 in every mode. */
typedef enum { CHASE_FP64 = 0, CHASE_TF32 = 1, CHASE_BF16X3 = 2, CHASE_FP64_EMU = 3 } chase_precision;

typedef enum {
  CHASE_OK = 0,
  CHASE_NOT_CONVERGED = 1,  /* max_iter reached; partial results returned */
  CHASE_CHOL_FAILED = 2,    /* a forced Cholesky variant failed (chase_qr only) */
  CHASE_ERR_CUDA = 3,       /* a CUDA runtime call failed */
  CHASE_ERR_OOM = 4,        /* workspace allocation failed */
  CHASE_ERR_TIMEOUT = 5,    /* a bounded device wait gave up */
  CHASE_ERR_NONFINITE = 6,  /* NaN/Inf met in the data */
  CHASE_ERR_UNSUPPORTED = 7, /* option not available in this build */
  CHASE_ERR_TOO_LARGE = 8    /* problem exceeds chase_filter_noalloc's fixed scratch */
} chase_status;

/* Variant codes of Algorithm 3 (also used by qr_force). */
enum { CHASE_QR_AUTO = 0, CHASE_QR_CHOL1 = 1, CHASE_QR_CHOL2 = 2, CHASE_QR_SHIFTED = 3,
       CHASE_QR_HOUSEHOLDER = 4 };

typedef struct {
  double tol;        /* residual threshold of eq. res (Section 2.4), default 1e-10 */
  int max_iter;      /* outer iterations of Algorithm 1, default 25 */
  int deg_init;      /* degree of every column in the first filter (Section 4.3: 20) */
  int deg_min;       /* lower clamp of the optimised degrees, default 10 */
  int deg_max;       /* upper clamp (Section 4.3: 36) */
  int opt_degree;    /* 1: per-column degrees from the convergence ratio; 0: deg_init always */
  double eta;        /* constant of Proposition th:2-2; 1 per Remark obs:2-1 */
  double cond_hi;    /* Algorithm 3: shifted CholeskyQR2 above this estimate (1e8) */
  double cond_lo;    /* Algorithm 3: CholeskyQR1 below this estimate (20) */
  int qr_force;      /* CHASE_QR_AUTO or a forced variant */
  chase_precision prec; /* arithmetic of the A*V products (see chase_precision) */
  double mp_switch;  /* mixed mode: the filter runs in BF16x3 until the largest residual of the
                        unlocked wanted pairs drops to mp_switch * max(|lambda1|, |b_sup|),
                        then in FP64 for the remaining iterations (default 1e-3) */
  /* Observability (the per-iteration data of Figure 2): if set, called after
   * every filter, before the QR, with the device block [Y V] that Algorithm 3
   * is about to factor (n x ell, ld n, the solve's dtype) and the iteration
   * number (1-based).  The block must not be modified; the call is synchronous
   * with the solve's stream.  NULL (default): no call. */
  void (*filtered_hook)(void* ctx, const void* dX, int n, int ell, int ldx, int iteration);
  void* filtered_hook_ctx;
  /* 0 (default): the estimate of Eq. full-est as printed.  1: the larger of it and
   * eta |rho_1|^{m_ell}.  Once pairs are locked, [Y V] has the unit singular values
   * of Y while the filter's gains are <= 1, so kappa_2([Y V]) can exceed Eq. full-est
   * (measured: up to ~10x); |rho_1|^{m_ell} bounds 1 / (smallest gain). */
  int cond_est_mode;
  /* 1: each FP64_EMU filter call of chase_solve is recorded into a CUDA graph (stream
     capture, thread-local mode) and launched as one unit; the handle's stream must not be
     a default stream (NULL, cudaStreamLegacy, cudaStreamPerThread), otherwise the launches
     are issued directly.  Same kernels in the same order: results are identical.  Default 0. */
  int graph_filter;
  /* 1: the emulated-FP64 products tune their launch plans (column-tile width, K splits) the
     first time the process meets a shape bucket: every candidate plan is timed on that
     product (the plans give bit-identical results) and the fastest is kept for the process
     (chase_autotune_table lists the picks).  0 (default): the picks already in the table,
     else the built-in heuristic. */
  int autotune;
  int reserved[3];
} chase_config;

/* Spectral information the filter needs (Algorithm 1, step "estimate lambda_1,
 * lambda_ell and lambda_n"): lambda1 ~ lowest eigenvalue, lambda_ell ~ the
 * ell-th eigenvalue, b_sup >= largest eigenvalue (must bound it from above). */
typedef struct {
  double lambda1, lambda_ell, b_sup;
} chase_bounds;

typedef struct {
  int iterations;
  int locked;
  long long matvecs;       /* sum over iterations of the unlocked columns' degrees */
  int n_chol1, n_chol2, n_shifted, n_hhqr; /* QR variant used per iteration */
  int n_chol_failures;     /* Cholesky failures that triggered an escalation */
  double t_total, t_filter, t_qr, t_rr, t_resid; /* seconds, CUDA-event timed */
  double filter_flops;     /* algorithmic flops of the filter products (2n^2 / 8n^2 per MatVec) */
  int kernel_launches;     /* CUDA kernels this call launched */
  int filter_launches;     /* of which filter product launches (one per filter step) */
  int n_lowprec_iters;     /* iterations whose filter ran in BF16x3 */
  double t_filter_lowprec; /* seconds of those filters */
  double filter_flops_lowprec; /* their algorithmic flops (counted as for FP64) */
  double t_rr_eig;         /* part of t_rr spent in the Jacobi eigensolver */
  int jacobi_sweeps;       /* Jacobi sweeps summed over iterations */
  double t_filter_product; /* part of t_filter spent in the product kernels alone (CUDA events
                              around each launch; filters launched as graphs add nothing) */
  double t_graph_build;    /* graph_filter = 1: host seconds spent recording and instantiating
                              the filter graphs (inside t_filter) */
  int graph_launches;      /* graph_filter = 1: filter calls that ran as one graph launch */
  int autotune_trials;     /* autotune = 1: candidate product plans timed during this solve */
} chase_stats;

/* Per-iteration record (the kind of data Figure 2 plots). */
typedef struct {
  int iteration, locked_before, locked_after, variant, chol_fail_info, deg_min, deg_max;
  long long matvecs;
  double log_cond_est, c, e, mu1, mu_ell;     /* log_cond_est: the estimate that chose the QR */
  double log_cond_est_paper, log_cond_est_locked; /* both forms (see cond_est_mode) */
} chase_iter_log;

/* Creates a handle bound to CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to order work on (cudaStreamLegacy or cudaStreamPerThread for
 * the default streams), or NULL for a new stream owned by the handle; that
 * stream is a blocking one, so it is ordered with work on the legacy default
 * stream.  Returns CHASE_ERR_CUDA if the device cannot be used. */
int chase_create(chase_handle* h, int device, void* cuda_stream);

/* Frees the handle's workspace and stream (if it owns one). */
int chase_destroy(chase_handle h);

/* Fills *cfg with the defaults listed above. */
int chase_config_default(chase_config* cfg);

/* Device workspace chase_solve needs for this problem shape (bytes). */
int chase_workspace_bytes(chase_dtype dtype, int n, int nev, int nex, chase_precision prec,
                          size_t* bytes);

/* Grows the handle's workspace to at least `bytes` now, so that later calls of
 * that size allocate nothing (a service sizes its handles once at start-up). */
int chase_reserve_workspace(chase_handle h, size_t bytes);

/*
 * chase_solve -- Algorithm 1.
 *   n         matrix order (>= 1);  dA: n x n device matrix, lda >= n.
 *   nev, nex  wanted pairs and extra search vectors; ell = nev + nex <= n.
 *   cfg       options (NULL: defaults).
 *   bounds    spectral estimates, or NULL: then chase_lanczos_bounds runs first
 *             with 4 runs (fewer if ell < 4) of min(25, n - 1) steps started at
 *             the first columns of dV (the start block's random vectors).
 *   dV        device n x ell block, ldv >= n.  On entry: the start block V0 of
 *             Algorithm 1 (random or a warm start; need not be orthonormal).
 *             On exit: columns 0..nev-1 hold the eigenvectors Y in ascending
 *             eigenvalue order, the other columns the remaining search block.
 *   evals     host, nev doubles: eigenvalues ascending.
 *   resid     host, nev doubles: residual norms ||A y - lambda y||_2 (eq. res).
 *   stats     host, optional (may be NULL).
 *   log, log_cap  host array of per-iteration records (may be NULL / 0).
 * Returns CHASE_OK when all nev pairs met tol, CHASE_NOT_CONVERGED after
 * max_iter iterations (results are the current approximations), or an error.
 */
int chase_solve(chase_handle h, chase_dtype dtype, int n, const void* dA, int lda, int nev,
                int nex, const chase_config* cfg, const chase_bounds* bounds, void* dV, int ldv,
                double* evals, double* resid, chase_stats* stats, chase_iter_log* log,
                int log_cap);

/*
 * chase_filter -- Algorithm 4 with per-column degrees (Section 2.3):
 *   dVout[:, a] = p_{m_a}(A) dV[:, a],  p_m(x) = C_m((x - c)/e) / C_m((lambda1 - c)/e),
 * computed by the scaled three-term recurrence.  The damped interval is
 * [c - e, c + e] (e > 0) and lambda1 < c - e.
 *   degrees   host, ncols ints, ascending, each >= 0 (0 copies the column).
 *   dV        device n x ncols input (not modified); dVout device n x ncols
 *             output: either dV itself with ldvout == ldv (filtered in place) or a
 *             block that overlaps neither dV nor dA (otherwise -14, nothing done).
 *   prec      CHASE_FP64, CHASE_FP64_EMU (Ozaki-scheme FP64 products on the
 *             tensor cores) or CHASE_BF16X3 (each A*V product as three BF16
 *             tensor-core products of hi/lo splits, FP32 accumulation); the
 *             recurrence itself is FP64 (CHASE_TF32: CHASE_ERR_UNSUPPORTED).
 */
int chase_filter(chase_handle h, chase_dtype dtype, int n, const void* dA, int lda, int ncols,
                 const void* dV, int ldv, const int* degrees, double c, double e, double lambda1,
                 chase_precision prec, void* dVout, int ldvout);

/*
 * chase_qr -- Algorithm 3 on the device block dX (n x ncols, in place):
 *   qr_force = CHASE_QR_AUTO picks by est_cond (shifted CholeskyQR2 if
 *   est_cond > 1e8, CholeskyQR1 if < 20, else CholeskyQR2; a failing
 *   Cholesky escalates to the shifted branch and then to Householder QR);
 *   a forced Cholesky variant that fails returns CHASE_CHOL_FAILED with dX
 *   unchanged.  On success dX holds an orthonormal basis Q of its column
 *   space with X = Q R.
 *   variant_used, chol_info: host outputs (may be NULL).
 */
int chase_qr(chase_handle h, chase_dtype dtype, int n, int ncols, void* dX, int ldx,
             double est_cond, int qr_force, int* variant_used, int* chol_info);

/*
 * chase_qr_prec -- chase_qr with a choice of arithmetic for its two block
 * products (the Gram matrix X^H X and X R^{-1}; Algorithm 2):
 *   CHASE_FP64      FP64 CUDA-core products (chase_qr);
 *   CHASE_FP64_EMU  Ozaki-scheme products on the BF16 tensor cores, accurate
 *                   to the FP64 error class (the products chase_solve uses in
 *                   that precision).
 * The Cholesky factor, its inverse and the Householder fallback stay FP64.
 * Other precisions return -9.  In the emulated mode the workspace grows by the
 * products' residue planes, residues and FP64 staging: about 450 n ncols bytes
 * (complex) or 150 n ncols bytes (real).
 */
int chase_qr_prec(chase_handle h, chase_dtype dtype, int n, int ncols, void* dX, int ldx,
                  double est_cond, int qr_force, chase_precision prec, int* variant_used,
                  int* chol_info);

/*
 * chase_cond_est -- the estimate of Eq. full-est (Corollary cr:3-1):
 *   kappa_est = eta |rho_{k+1}|^{m_{k+1}} |rho_1|^{m_ell - m_{k+1}},
 * |rho(x)| = |t| + sqrt(t^2 - 1), t = (x - c)/e (1 inside the damped interval).
 *   ell, nlocked    block width and k;  ritz: host, ell Ritz values (the one at
 *   index nlocked belongs to the first unlocked column);  degrees: host, ell
 *   degrees (degrees[nlocked] = m_{k+1}, degrees[ell-1] = m_ell);
 *   lambda1: lowest-eigenvalue estimate (gives rho_1).
 *   est: host output kappa_est;  log_est (may be NULL): its natural log, finite
 *   even when kappa_est overflows.
 * Host arithmetic only; no handle needed.
 */
int chase_cond_est(int ell, int nlocked, const double* ritz, const int* degrees, double lambda1,
                   double c, double e, double eta, double* est, double* log_est);

/*
 * chase_lanczos_bounds -- the spectral estimates Algorithm 1 takes before its
 * loop ("estimate lambda_1, lambda_ell and lambda_n" by a few Lanczos runs).
 *   nruns     runs, started at the columns of dV0 (device, n x nruns, ldv >= n;
 *             random vectors supplied by the caller); steps: Lanczos steps per
 *             run (1 <= steps < n), with full re-orthogonalisation.
 *   ell       nev + nex, the index whose eigenvalue lambda_ell estimates.
 *   out       host: lambda1 = smallest Ritz value of all runs; b_sup = largest
 *             (Ritz value + |last beta|) of a run, an upper bound of lambda_n;
 *             lambda_ell = the smallest Ritz value at which the spectral-density
 *             estimate (n / nruns) sum_runs sum_{theta_i <= x} tau_i reaches ell
 *             (tau_i: squared first component of the tridiagonal's eigenvector).
 * The reading of how the three numbers are formed is this library's (the paper
 * names the Lanczos step without its formulas).
 */
int chase_lanczos_bounds(chase_handle h, chase_dtype dtype, int n, const void* dA, int lda,
                         int nruns, const void* dV0, int ldv, int steps, int ell,
                         chase_bounds* out);

/*
 * Batches: many eigenproblems advanced together (the batched and serving workloads).
 *
 * A batch session keeps any number of problems in flight on one handle.  Each problem has a
 * stream of its own; its QR, Rayleigh-Ritz, residual and locking phase (Algorithm 1 after the
 * filter) runs on a worker thread, and as soon as it ends the problem is ready for its next
 * filter.  The emulated-FP64 filters (Algorithm 4) of all problems ready at that moment run as
 * shared launches: per step of the three-term recurrence one slicing, one modular-product and
 * one reconstruction launch over every problem still filtering (up to 64 problems per launch),
 * so that many small or uneven problems fill the GPU together, and fast problems do not wait
 * for slow ones.
 * Each problem's arithmetic is the one chase_solve performs (the grouped products are exact
 * integer products like the single ones), so results are identical to chase_solve's.  Problems
 * with other precisions, with graph_filter = 1 or with n > 65536, filter one by one inside the
 * same step.
 * Problems may be added between steps (a service admits requests as earlier ones finish).
 * Device workspace comes from a caching pool owned by the session.
 */
typedef struct chase_batch_ctx* chase_batch;

/* Creates an empty batch session on handle h (its device and stream). */
int chase_batch_create(chase_batch* b, chase_handle h);

/* Frees the session; problems still in flight are abandoned (their outputs are not written). */
int chase_batch_destroy(chase_batch b);

/*
 * chase_batch_add -- arguments as chase_solve; the problem is validated, its workspace taken
 * from the session's pool, its start block copied, checked and orthonormalised (Algorithm 1's
 * step 0) before the call returns.  The caller keeps dA, dV and the host outputs (evals, resid,
 * stats, log) alive until the problem is reported finished by chase_batch_step, which then has
 * written them as chase_solve would.  *id receives the problem's id in this session.
 * Returns CHASE_OK, a negative argument index, or an error (nothing added).
 */
int chase_batch_add(chase_batch b, chase_dtype dtype, int n, const void* dA, int lda, int nev,
                    int nex, const chase_config* cfg, const chase_bounds* bounds, void* dV, int ldv,
                    double* evals, double* resid, chase_stats* stats, chase_iter_log* log,
                    int log_cap, int* id);

/*
 * chase_batch_step -- advances the problems in flight (if no finished problem is still waiting
 * to be reported) until every one of them has completed at least one more outer iteration or
 * ended; faster problems may complete several.  No work of the session runs when it returns.
 * Calls on one session must not overlap.  Problems that ended -- all nev pairs converged (CHASE_OK),
 * max_iter reached (CHASE_NOT_CONVERGED) or an error -- are reported in done_ids / done_status
 * (host arrays of cap entries; *ndone receives the count; more than cap finished problems are
 * reported by the next calls).
 */
int chase_batch_step(chase_batch b, int* done_ids, int* done_status, int cap, int* ndone);

/* Problems in flight plus finished ones not yet reported. */
int chase_batch_pending(chase_batch b);

/* One problem of chase_solve_batch (arguments as chase_solve's; bounds may be NULL). */
typedef struct {
  chase_dtype dtype;
  int n;
  const void* dA;
  int lda;
  int nev, nex;
  const chase_bounds* bounds;
  void* dV;
  int ldv;
  double* evals;
  double* resid;
  chase_stats* stats; /* may be NULL */
} chase_problem;

/*
 * chase_solve_batch -- solves `count` problems through one batch session (every problem added,
 * then steps until all have ended).  status[i] receives problem i's result (as chase_solve's
 * return value, or the error its addition met).  Returns CHASE_OK or a session-level error.
 */
int chase_solve_batch(chase_handle h, int count, const chase_problem* problems,
                      const chase_config* cfg, int* status);

/*
 * chase_autotune_table -- the autotuner's picks so far (one text line per shape bucket:
 * shape, bucket, tile-width cap, K splits, measured seconds), NUL-terminated into buf (cap
 * bytes; truncated if short).  *needed (may be NULL) receives the bytes the full table needs.
 * chase_autotune_clear -- forgets every pick.  The table is shared by the whole process.
 * No counterpart in the paper: the launch plans are this implementation's.
 */
int chase_autotune_table(char* buf, size_t cap, size_t* needed);
int chase_autotune_clear(void);

/* Static description of a status code. */
const char* chase_status_string(int status);

/*
 * chase_selftest_wait_timeout -- checks the failure path of the library's
 * bounded device waits without causing a fault (the paper has no counterpart;
 * it is a diagnostic of this implementation).  One device thread waits, for at
 * most `seconds` (0 < seconds <= 10), on a barrier that nothing completes,
 * gives up and records the timeout in the handle's device status word, the way
 * the tensor-core kernels do when a copy or an MMA never completes.  Returns
 * CHASE_ERR_TIMEOUT when the wait ran out and was reported (the expected
 * result), CHASE_OK if it was not, CHASE_ERR_CUDA on a CUDA failure; the
 * status word is cleared again and the handle stays usable.
 */
int chase_selftest_wait_timeout(chase_handle h, double seconds);

/* Size of the fixed device scratch array behind chase_filter_noalloc (32 MiB). */
#define CHASE_FILTER_NOALLOC_MAX_BYTES ((size_t)32 << 20)

/*
 * chase_filter_noalloc -- the same filter as chase_filter, for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is a
 * deployment variant of the library's filter, not a step of the method.
 *
 * chase_filter (like every handle-based call) grows a device workspace with
 * cudaMalloc on demand.  Some callers cannot let a library do that: code that
 * runs while a CUDA graph is being captured (cudaMalloc cannot be recorded),
 * serving processes that reserve all of HBM in their own pool up front, and
 * latency-critical loops where cudaMalloc / cudaFree would synchronise the
 * device.  This entry point calls no allocating routine: its scratch (the
 * recurrence's second n x ncols buffer and the split-K partial sums) lives in
 * one file-scope device array of CHASE_FILTER_NOALLOC_MAX_BYTES that every GPU
 * loading the library holds until the process exits.
 *
 * Arguments as chase_filter (FP64 only), without a handle (dVout: dV itself with
 * ldvout == ldv, or clear of dV and dA; otherwise -12): the work is ordered
 * on `cuda_stream` (a cudaStream_t, NULL = legacy default stream) of the
 * current device, and the call returns after it completes; while `cuda_stream`
 * is being captured into a CUDA graph the work is recorded and the call returns
 * at once (replaying the graph runs the filter on the captured pointers; a capture
 * that was already invalidated gives CHASE_ERR_CUDA).  The
 * caller passes and owns dV and dVout as before.
 * Limits and behaviour:
 *   - sizeof(element) * n * ncols must be <= CHASE_FILTER_NOALLOC_MAX_BYTES,
 *     otherwise CHASE_ERR_TOO_LARGE is returned and nothing is done.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture.
 *   - All calls on a device share the array, which keeps the last call's
 *     contents (nothing in it needs to start at zero).  Calls that overlap on
 *     the GPU race on it: order them on one stream.
 */
int chase_filter_noalloc(chase_dtype dtype, int n, const void* dA, int lda, int ncols,
                         const void* dV, int ldv, const int* degrees, double c, double e,
                         double lambda1, void* dVout, int ldvout, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CHASE_GB300_H */
