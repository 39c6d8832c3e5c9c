/*
 * uoi.h -- C ABI of the GB300 (sm_103a) UoI_LASSO / UoI_VAR(d) hot path.
 *
 * Method: Balasubramanian et al., "Optimizing the Union of Intersections LASSO
 * (UoI_LASSO) and Vector Autoregressive (UoI_VAR) Algorithms for Improved
 * Statistical Estimation at Scale", arXiv 1808.06992:
 *   Alg. 1          UoI_LASSO: B1 bootstraps x q lambdas of LASSO (selection),
 *                   support intersection (Eq. 3), B2 bootstraps of OLS on each
 *                   support with held-out loss argmin, averaging (Eq. 4).
 *   Alg. 2, Eq. 6-9 UoI_VAR: the same on the lagged design of a VAR(d) series,
 *                   vectorised into p LASSOs that share one design.
 *   Eq. 5           the LASSO is solved by ADMM (x-update, soft-threshold,
 *                   dual update).
 *
 * Conventions shared by every entry point
 *  - Matrices are row-major, float64.  "n x p" means n rows of p values.
 *  - Every pointer argument may point to host memory or to device memory of
 *    the current CUDA device; the kind is detected per pointer.  Host inputs
 *    are copied to the device and outputs copied back before return.
 *  - The caller owns every buffer it passes.  The library owns its scratch,
 *    taken from a stream-ordered pool of the current device; uoi_shutdown()
 *    returns it.
 *  - Work is issued on prm->stream / the stream argument (NULL = the legacy
 *    default stream); every entry point returns after the results are in the
 *    output buffers (it synchronises that stream).  Inside a mixed fit some
 *    independent work also runs on a second stream the library keeps per
 *    calling thread, ordered against the caller's stream by events (the small
 *    supports of the estimation's loss pass; half of the selection's systems in
 *    the tensor-core inverse, enqueued by a helper thread that ends before the
 *    inverse returns).
 *  - Outputs are written only when the status is UOI_OK or
 *    UOI_OK_WITH_WARNINGS.  No C++ exception crosses the boundary.
 *  - Not thread-safe per device: calls on one device must not overlap.
 */
#ifndef UOI_H
#define UOI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define UOI_OK                 0
#define UOI_OK_WITH_WARNINGS   1   /* non-converged ADMM columns or singular OLS supports */
#define UOI_ERR_INVALID_ARG   -1   /* null pointer, non-positive size, bad parameter       */
#define UOI_ERR_NONFINITE     -2   /* NaN/Inf in X or y (checked on the device)            */
#define UOI_ERR_NOT_PD        -3   /* Cholesky pivot <= 0 (only possible with rho <= 0)    */
#define UOI_ERR_CUDA          -4   /* a CUDA runtime call failed                           */
#define UOI_ERR_OOM           -5   /* device allocation failed                             */
#define UOI_ERR_TIMEOUT       -6   /* a bounded device loop ran out of iterations          */
#define UOI_ERR_BOUNDS        -7   /* an index check of the checked build failed            */
#define UOI_ERR_UNSUPPORTED   -8   /* e.g. an intercept on an entry with no output for it  */

/* ---- parameter enums ------------------------------------------------------ */
#define UOI_BAG_MEDIAN   0   /* coordinate-wise median over the B2 chosen estimates  */
#define UOI_BAG_MEAN     1   /* the paper's average (Alg. 1 last step, Eq. 4)        */
#define UOI_SPLIT_PER_BOOTSTRAP 0  /* a fresh train/eval reshuffle per bootstrap     */
#define UOI_SPLIT_FIXED         1  /* bootstrap 0's reshuffle for every bootstrap    */
#define UOI_PREC_FP64    0   /* plain FP64 form: every step in FP64                  */
#define UOI_PREC_MIXED   1   /* tensor-core Gram (two-piece bf16, FP32 accumulation
                                drained every 128 rows), FP32-accurate inverse,
                                FP32 ADMM (tensor-core x-update for p > 192), OLS by
                                FP32 factor + FP64 refinement                        */
#define UOI_WARM_NONE    0   /* every (bootstrap, lambda) column starts at z = u = 0 */
#define UOI_WARM_PATH    1   /* lambda descending; column j starts from j-1's (z,u)  */
#define UOI_WARM_LEARNED 2   /* learned initial (z,u) (MLP); judged by PATH          */
#define UOI_BLOCKS_FIXED  0  /* selection units: consecutive non-overlapping blocks */
#define UOI_BLOCKS_MOVING 1  /* selection units: ceil(m/L) blocks starting anywhere
                                in 0..m-L (overlapping, Kunsch); estimation split
                                keeps the non-overlapping units                       */

/* Parameters of a fit (Alg. 1 / Alg. 2 inputs lambda, B1, B2 plus the ADMM
 * and bootstrap settings).  Zero-initialise, set struct_size = sizeof(uoi_params)
 * and the fields you need; uoi_params_default() fills the documented defaults. */
typedef struct uoi_params {
    uint32_t struct_size;
    int32_t  B1;                /* selection bootstraps (> 0)                          */
    int32_t  B2;                /* estimation bootstraps (> 0)                         */
    int32_t  q;                 /* number of lambdas (> 0)                             */
    const double* lambdas;      /* q values (host or device), NULL = log grid          */
    double   lambda_min_ratio;  /* grid: lambda_j = lmax * ratio^(j/(q-1)); 1e-3       */
    double   rho;               /* ADMM penalty (> 0); 1                               */
    double   abs_tol, rel_tol;  /* ADMM stopping tolerances; 1e-6, 1e-6                */
    int32_t  max_iter;          /* ADMM iteration cap per column; 1000                 */
    double   train_frac;        /* estimation pool fraction in (0,1); 0.8              */
    uint64_t seed;              /* Philox key word 0; 0                                */
    uint64_t problem_id;        /* Philox key word 1; 0                                */
    int64_t  block_len;         /* 0/1 = iid rows, L > 1 = blocks of L lagged rows     */
    int32_t  bagging;           /* UOI_BAG_*; median                                   */
    int32_t  split_mode;        /* UOI_SPLIT_*; per bootstrap                          */
    int32_t  precision;         /* UOI_PREC_*; FP64                                    */
    int32_t  warm_start;        /* UOI_WARM_*; path                                    */
    const char* mlp_weights_path; /* learned warm start weights, NULL = none           */
    void*    stream;            /* cudaStream_t, NULL = default stream                 */
    int32_t  intercept;         /* 1 = fit an unpenalised offset mu per response       */
                                /* (uoi_var_fit and uoi_fit_traced; 0 = none).         */
                                /* A struct_size that ends before this field reads 0.  */
    int32_t  block_mode;        /* UOI_BLOCKS_*: selection blocks of block_len rows,   */
                                /* non-overlapping (0) or moving (1); read as 0 when   */
                                /* struct_size ends before this field.                 */
} uoi_params;

/* Timings and counters of the last fit (every field written when non-NULL). */
typedef struct uoi_diag {
    uint32_t struct_size;
    float    ms_total, ms_bootstrap, ms_gram, ms_factor, ms_admm, ms_support, ms_estimation;
                                  /* ms_support: supports are ANDed into the family at ADMM
                                     column completion, so this is only what follows the
                                     ADMM launches (the family's tail mask)              */
    int64_t  admm_columns;        /* (bootstrap, equation, lambda) columns solved        */
    int64_t  admm_nonconverged;   /* columns that stopped at max_iter                    */
    int64_t  admm_iterations;     /* sum of iterations over all columns                  */
    int32_t  admm_max_iterations; /* largest per-column iteration count                  */
    int64_t  ols_singular;        /* supports whose OLS took the regularised fallback    */
    int64_t  gpu_launches;        /* kernels this library launched during the fit        */
    /* Live timing of the two kernels that bound a fit, from CUDA events on their
     * launch stream, with their algorithmic work (flops of the math, not of the
     * split products or padding; bytes of the streams the math must move). */
    float    ms_gram_tc;          /* tensor-core Gram launches (mixed form)              */
    int64_t  n_gram_tc;
    double   flops_gram_tc;       /* 2 n_k (p(p+1)/2 + p r) per bootstrap item           */
    float    ms_xupdate;          /* streaming ADMM x-update launches                    */
    int64_t  n_xupdate;
    double   flops_xupdate;       /* 2 p^2 per active column-iteration                   */
    double   bytes_xupdate;       /* M once per group-iteration + 6 p-vectors per column */
    int32_t  warm_start_used;     /* UOI_WARM_* actually used (LEARNED falls back to PATH) */
    int64_t  ols_fp64;            /* OLS solves refused by the FP32-factor + FP64-refinement
                                     solver (small pivot or stalled refinement) and
                                     factored in FP64 instead                            */
    /* The fields below are written when struct_size covers them (or is 0). */
    int64_t  admm_near_threshold; /* features of finished selection columns whose final
                                     margin |v_i| - lambda/rho (v = z + u) lies within 1e-6
                                     of zero: the support test of Eq. 3 is decided by less
                                     than that at those features                         */
    int64_t  admm_iter_hist[8];   /* selection columns by ADMM iterations: <= 16, 17-32,
                                     33-64, 65-128, 129-256, 257-512, > 512 (converged),
                                     and stopped at max_iter without converging          */
} uoi_diag;

/* Optional intermediate results of a fit, for testing (every pointer nullable,
 * host or device).  Shapes use r = response columns (1 for LASSO, p for VAR). */
typedef struct uoi_trace {
    double*   lambdas;      /* q                                                  */
    uint32_t* sel_weights;  /* B1 x m   bootstrap multiplicities of T^k           */
    uint32_t* est_weights;  /* B2 x m   multiplicities of the training sample T^k */
    uint8_t*  est_eval;     /* B2 x m   1 = row in the evaluation set E^k         */
    double*   sel_beta;     /* B1 x q x r x p  LASSO estimates (final z)          */
    int32_t*  sel_iters;    /* B1 x q x r                                         */
    uint8_t*  sel_conv;     /* B1 x q x r                                         */
    uint64_t* family;       /* q x r x ceil(p/64)  supports S_j (Eq. 3)           */
    double*   est_loss;     /* B2 x q x r  held-out squared-error sums            */
    int32_t*  est_jstar;    /* B2  chosen support index per bootstrap             */
    double*   est_beta;     /* B2 x r x pe the chosen OLS estimate per bootstrap, */
                            /* pe = p + intercept (mu last, original coordinates) */
    int32_t*  est_singular; /* B2 x q x r  1 = regularised fallback               */
} uoi_trace;

/* Fill *prm with the defaults listed above (B1 = B2 = 20, q = 16). */
void uoi_params_default(uoi_params* prm);

/* UoI_LASSO (Alg. 1).  X: n x p, y: n.  beta_out: p (the bagged estimate that
 * Alg. 1 returns); prm->intercept must be 0 (UOI_ERR_UNSUPPORTED).  family_out: q x ceil(p/64) words, bit i of S_j (Eq. 3),
 * nullable.  diag nullable. */
int uoi_lasso_fit(const double* X, const double* y, int64_t n, int64_t p,
                  const uoi_params* prm, double* beta_out, uint64_t* family_out,
                  uoi_diag* diag);

/* Many independent UoI_LASSO problems of uneven n and p in one call (the
 * "batched" workload: Alg. 1 applied to each problem separately).  Problem i is
 * X[i] (n[i] x p[i], row-major), y[i] (n[i]) -> beta_out[i] (p[i]); pointers host
 * or device, per problem.  One parameter set for all; prm->lambdas must be NULL
 * (each problem gets its own grid from its lambda_max) and problem i draws its
 * bootstraps with problem_id = prm->problem_id + i, so its result equals
 * uoi_lasso_fit on that problem with that problem_id.
 *   streams == 0 (grouped): every problem is fitted on its own stream by its own
 *     host thread (in waves of at most 128 problems, largest n*p^2 first), and the
 *     ADMM selection solves (Alg. 1's B1 x q LASSO problems, Eq. 5) of all the
 *     problems whose solve runs on the tensor cores (mixed precision, p above the
 *     shared-memory schedule's limit) iterate together: each step is one x-update
 *     launch over every live (problem, bootstrap, row tile, chain tile) and one
 *     convergence-check launch over every live chain tile, replayed eight steps
 *     at a time as a CUDA graph; a problem joins as soon as its inverse is ready
 *     and leaves, to its estimation, as soon as its columns have finished.  The
 *     chain tile and the pipeline depth are chosen by timing the first replays of
 *     a batch shape and reused by later calls with that shape.  Each problem's
 *     iterates are those of its own solve, so results do not change.
 *   streams > 0: `streams` worker streams, largest n*p^2 first, each worker
 *     fitting one problem at a time.
 * The call returns once all are done.  status_out (count, nullable) receives each
 * problem's status and diags (count, nullable) each problem's diagnostics (in the
 * grouped form each replay's launches and time are counted in the diagnostics of
 * one problem it advanced).  Returns UOI_OK, or UOI_OK_WITH_WARNINGS if any
 * problem warned, or the first failing problem's error (the others still ran and
 * their outputs are valid). */
int uoi_lasso_fit_batch(int32_t count, const double* const* X, const double* const* y,
                        const int64_t* n, const int64_t* p, const uoi_params* prm,
                        double* const* beta_out, int32_t* status_out, uoi_diag* diags,
                        int32_t streams);

/* UoI_VAR(order) (Alg. 2).  series: N x p, time ascending (row t = X_t),
 * order >= 1, N - order >= 2 (else UOI_ERR_INVALID_ARG).  The lagged design
 * pairs the response X_t (Eq. 7) with the regressors X_{t-1} .. X_{t-order}
 * (Eq. 8), rows t = order .. N-1 in ascending time, and is solved as p LASSOs
 * sharing that design (Eq. 9); a block of the block bootstrap holds block_len
 * consecutive such rows.  A_out: order x p x p,
 * A_out[(j-1)*p*p + e*p + i] = coefficient of X_{t-j,i} in equation e (the
 * last step of Alg. 2 splits beta* into A_1 .. A_d and mu).  mu_out: p
 * (nullable), the intercepts when prm->intercept = 1 (each fit then has an
 * unpenalised offset: the LASSO of the bootstrap-weighted centred data in the
 * selection, [X 1] in the estimation OLS and held-out loss, lambda_max of the
 * centred data), else zero-filled. */
int uoi_var_fit(const double* series, int64_t N, int64_t p, int32_t order,
                const uoi_params* prm, double* A_out, double* mu_out, uoi_diag* diag);

/* General form used by both fits: r response columns Y (m x r, row stride ldy)
 * on the design X (m x p, row stride ldx).  beta_out: r x pe, pe = p + 1 when
 * prm->intercept = 1 (row e: p coefficients, then mu_e) else p.  trace nullable. */
int uoi_fit_traced(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                   int64_t m, int64_t p, int64_t r, const uoi_params* prm,
                   double* beta_out, uoi_trace* trace, uoi_diag* diag);

/* Batched LASSO by ADMM (Eq. 5) -- the selection step's solver on caller
 * supplied weights: for every weight vector k < B (weights: B x n counts,
 * NULL = unweighted, then B must be 1), response column e < r of Y (n x r)
 * and lambda_j, minimise (1/(2 n_k)) ||y_e - X b||^2_{W_k} + lambda_j ||b||_1
 * with n_k = sum of weights k.  beta_out: B x q x r x p (final z).
 * iters_out, converged_out: B x q x r, nullable. precision: UOI_PREC_*,
 * warm_start: UOI_WARM_NONE or UOI_WARM_PATH.  stream: cudaStream_t or NULL. */
int lasso_admm_batch(const double* X, const double* Y, int64_t n, int64_t p, int64_t r,
                     const uint32_t* weights, int32_t B, const double* lambdas, int32_t q,
                     double rho, double abs_tol, double rel_tol, int32_t max_iter,
                     int32_t precision, int32_t warm_start, double* beta_out,
                     int32_t* iters_out, uint8_t* converged_out, void* stream);

/* Weighted moments of the selection step (G1; Alg. 1 "Compute LASSO estimate
 * ... from T^k" only needs these): for every k < B,
 *   G_out[k] = X^T diag(w_k) X   (p x p),   B_out[k] = X^T diag(w_k) Y   (p x r)
 * with X: n x p, Y: n x r, weights: B x n bootstrap multiplicities (not NULL).
 * precision UOI_PREC_FP64: FP64 CUDA cores.  UOI_PREC_MIXED: two-piece bf16 on
 * tensor cores (tcgen05), FP32 accumulation drained every 128 sample rows into
 * FP32 running sums, written in FP64; error within about 5e-7 of the largest
 * diagonal entry (2e-6 is the tested bound). */
int uoi_weighted_moments(const double* X, const double* Y, int64_t n, int64_t p, int64_t r,
                         const uint32_t* weights, int32_t B, int32_t precision,
                         double* G_out, double* B_out, void* stream);

/* Batched LASSO-ADMM for callers that cannot allocate device memory.
 *
 * lasso_admm_batch obtains its working memory from the device's memory pool.
 * Some callers cannot allow that: applications that reserve all of the
 * device's memory at start-up for their own allocator, hosts that run under a
 * fixed device-memory quota, and latency-critical loops where an allocation
 * may block and a free synchronises the device.  This variant allocates
 * nothing: it works in one fixed scratch array of UOI_NOALLOC_SCRATCH_BYTES
 * that is part of the library's device image, so every GPU that loads the
 * library holds that array until the process exits.
 * (The paper has no counterpart of this entry point.)
 *
 * Same arguments and results as lasso_admm_batch with precision UOI_PREC_FP64,
 * with these limits:
 *  - every pointer must be device memory of the current device, or managed
 *    memory (else UOI_ERR_INVALID_ARG);
 *  - p <= UOI_NOALLOC_MAX_P, and the working set
 *    3*B*p*p*8 + 2*B*p*r*8 + B*p*8 + B*q*r bytes (plus a few KB) must fit in
 *    the scratch array; larger problems return UOI_ERR_INVALID_ARG with a
 *    message from uoi_get_last_error_detail.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device) and caches it; make that first call
 * before any stream capture.
 * Every call shares the one array and overwrites it: calls that overlap on the
 * GPU (different streams or threads) race and must be serialised by the
 * caller.  Each call clears the counters it needs, so back-to-back calls on
 * one stream are independent.  Like every entry point, the call returns after
 * its results are in the output buffers (it synchronises the stream). */
#define UOI_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
#define UOI_NOALLOC_MAX_P 128
int lasso_admm_batch_noalloc(const double* X, const double* Y, int64_t n, int64_t p, int64_t r,
                             const uint32_t* weights, int32_t B, const double* lambdas, int32_t q,
                             double rho, double abs_tol, double rel_tol, int32_t max_iter,
                             int32_t warm_start, double* beta_out, int32_t* iters_out,
                             uint8_t* converged_out, void* stream);

/* ---- learned warm start (an extension: the paper warm-starts nothing) ----
 * A per-feature network (8 inputs -> 3 hidden layers of 512 with GELU -> 3
 * outputs, BF16 weights, FP32 accumulation) predicts the converged scaled ADMM
 * state (scaled z, rho u/lambda, active logit) of every (bootstrap, lambda,
 * equation, feature) from lambda and moment statistics (see the feature list
 * in uoi_ws_dataset).  A fit with warm_start = UOI_WARM_LEARNED and
 * mlp_weights_path set runs the lambda batch cold-scheduled from the
 * predicted state; without usable weights it falls back to UOI_WARM_PATH.
 * Parameters are a flat FP32 array: W1 (512x8) b1 W2 (512x512) b2 W3 b3
 * W4 (3x512) b4, matrices row-major [out][in].  Handles are not thread-safe. */
typedef struct uoi_ws_model uoi_ws_model;
int64_t uoi_ws_param_count(void);
int uoi_ws_create(uint64_t seed, uoi_ws_model** out);          /* Kaiming-uniform init */
int uoi_ws_load(const char* path, uoi_ws_model** out);
int uoi_ws_save(uoi_ws_model* model, const char* path);
void uoi_ws_free(uoi_ws_model* model);
int uoi_ws_set_params(uoi_ws_model* model, const float* params);  /* host or device */
int uoi_ws_get_params(uoi_ws_model* model, float* params);
/* out (N x 3) = network(X (N x 8)); host or device buffers. */
int uoi_ws_forward(uoi_ws_model* model, const float* X, int64_t N, float* out);
/* Mean loss over the N rows and its gradient (uoi_ws_param_count floats). */
int uoi_ws_loss_grad(uoi_ws_model* model, const float* X, const float* T, int64_t N,
                     double* loss, float* grad);
/* Adam (lr, beta 0.9/0.999, weight decay 1e-5) over shuffled mini-batches. */
int uoi_ws_train(uoi_ws_model* model, const float* X, const float* T, int64_t N, int32_t epochs,
                 int32_t batch, float lr, uint64_t seed, double* final_loss);
/* Training rows from the method's own solutions: path-warm FP64 ADMM over
 * B bootstraps (weights B x n) x q lambdas x r responses, then for every
 * (k, j, e, i) the 8 features (c = X^T W y_e / n_k, d = diag(X^T W X)/n_k,
 * x0 = (X^T W X/n_k + rho I)^{-1} c the ridge solution, a_j = x0 d / lambda_j,
 * ratios clipped to [-50, 50])
 *   lambda_j/lambda_0, log(lambda_j/lambda_0)/log(lambda_{q-1}/lambda_0),
 *   c/lambda_j, d, a_j, |a_j|, c/lambda_{j-1}, a_{j-1}
 * and the 3 targets z/s clipped to [-4, 4] with s = (lambda_j/d) max(1, |a_j|),
 * rho u/lambda_j and [z != 0].  features_out: N x 8, targets_out: N x 3 floats
 * (N = B q r p), host or device. */
int uoi_ws_dataset(const double* X, const double* Y, int64_t n, int64_t p, int64_t r,
                   const uint32_t* weights, int32_t B, const double* lambdas, int32_t q,
                   double rho, double abs_tol, double rel_tol, int32_t max_iter,
                   float* features_out, float* targets_out, void* stream);

/* Test support for the fault path of the tensor-core kernels (the paper has no
 * counterpart).  Every mbarrier wait of those kernels is bounded (one second by
 * default); when a limit runs out the kernel records UOI_ERR_TIMEOUT in its
 * error word and returns, leaving the context usable, and the call returns
 * UOI_ERR_TIMEOUT.  This runs that bounded wait alone: one thread waits, with
 * limit_ns (0 < limit_ns <= 10 s, else UOI_ERR_INVALID_ARG), for an arrival on
 * an mbarrier that nothing arrives on (arrive = 0: returns UOI_ERR_TIMEOUT once
 * the limit has passed) or that it arrives on itself first (arrive = 1: returns
 * UOI_OK).  waited_ms (host, nullable): the time the wait took, by the GPU's
 * global timer. */
int uoi_selftest_wait(uint64_t limit_ns, int32_t arrive, double* waited_ms, void* stream);

/* Test support for the index checks of the checked build (the paper has no
 * counterpart).  The checked build (compiled with UOI_BOUNDS_CHECK=1) checks the
 * indices of its kernels' main stores; a failed check records UOI_ERR_BOUNDS and
 * skips the access, and the call returns UOI_ERR_BOUNDS.  This runs that check
 * once on the device, in either build: one thread stores into element `index` of
 * a buffer of `extent` floats (0 < extent <= 4096) if 0 <= index < extent and
 * returns UOI_OK, else skips the store and returns UOI_ERR_BOUNDS. */
int uoi_selftest_index_check(int64_t index, int64_t extent, void* stream);

/* Text of a status code (static storage). */
const char* uoi_status_string(int status);

/* Copy the detail message of the last error on this thread into buf (NUL
 * terminated, truncated to len).  Returns the message length. */
int uoi_get_last_error_detail(char* buf, size_t len);

/* Free the library's device scratch on the current device. */
void uoi_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif
