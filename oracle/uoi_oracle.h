/*
 * uoi_oracle.h -- FP64 CPU oracle for the UoI_LASSO / UoI_VAR(d) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library under
 * paper_1808_06992_gb300/ and never calls it.
 *
 * Everything here is plain, single-threaded (per bootstrap) FP64 C written
 * from the paper (Balasubramanian et al., "Optimizing the Union of
 * Intersections LASSO and VAR algorithms ...", arXiv 1808.06992):
 *   Sec. II-B Eq. 1-2       linear model and LASSO objective
 *   Sec. II-C Eq. 3         selection by intersection of bootstrap supports
 *   Sec. II-D Eq. 4         estimation by union (averaging) of OLS fits
 *   Sec. II-E Eq. 5         LASSO by ADMM; OLS as the lambda = 0 problem
 *   Algorithm 1             UoI_LASSO
 *   Algorithm 2, Eq. 6-9    UoI_VAR: VAR(d) model, lagged design, vectorisation
 *   Sec. III-A              bootstrap / block bootstrap / reshuffled split
 * plus Philox4x64-10 from Salmon et al., SC'11 ("Parallel random numbers:
 * as easy as 1, 2, 3") for the counter-based random draws.
 *
 * All matrices are row-major.  Status codes: 0 ok, 1 ok with warnings
 * (non-converged ADMM column or min-norm OLS fallback), <0 error.
 *
 * Parity status per function: every function is pinned by a test in
 * tests/test_oracle_pins.py (ref_kkt_polish in tests/test_oracle_kkt.py).
 * ref_uoi_fit as a whole is pinned through its parts, the noiseless-recovery
 * special case, the cases whose selection is decided in advance, and the
 * general case on LASSO (with and without an intercept) and VAR(1) fixtures
 * with varying supports (tests/test_oracle_whole_fit.py): an independent route
 * of scikit-learn's LASSO on the bootstrap rows repeated by multiplicity, then
 * intersection, least squares on the training draws, held-out losses, argmin
 * and median in numpy, with the fixtures' KKT margins asserted so that the
 * comparison is decided.
 */
#ifndef UOI_ORACLE_H
#define UOI_ORACLE_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes of the oracle (its own numbering; the values agree with the
 * CUDA library's so that tests can compare them, but nothing is shared). */
#define REF_OK                0
#define REF_OK_WITH_WARNINGS  1
#define REF_ERR_INVALID_ARG  -1
#define REF_ERR_NONFINITE    -2
#define REF_ERR_NOT_PD       -3
#define REF_ERR_UNSUPPORTED  -8

/* Philox stream tags (word 2 of the counter). */
#define REF_TAG_SELECTION  1u   /* Alg. 1/2 selection bootstrap draws        */
#define REF_TAG_SPLIT      2u   /* estimation reshuffle keys (Fig. 1(c))     */
#define REF_TAG_RESAMPLE   3u   /* estimation training resample draws        */

/* Philox4x64-10 block function (Salmon et al. 2011): out = F_key(ctr). */
void ref_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* The i-th 64-bit draw of stream (k, tag): lane (i mod 4) of
 * Philox4x64-10(counter = (i/4, k, tag, 0), key = (seed, problem)). */
uint64_t ref_draw(uint64_t seed, uint64_t problem, uint64_t k, uint64_t tag, uint64_t i);

/* floor(r * n / 2^64): maps a uniform 64-bit draw onto [0, n). */
uint64_t ref_range_map(uint64_t r, uint64_t n);

/* Selection bootstrap T^k (Alg. 1 selection loop; Alg. 2 with blocks,
 * Sec. III-A-2).  Rows 0..m-1 are grouped into ceil(m/L) consecutive blocks
 * of L rows (the last one short); L <= 1 means single rows.  ceil(m/L) block
 * draws with replacement; w[row] = how many times the row was drawn. */
void ref_selection_weights(int64_t m, int64_t block_len, uint64_t seed, uint64_t problem,
                           int64_t k, uint32_t* w);

/* Moving-block selection bootstrap (Kunsch's overlapping blocks, the
 * alternative to the non-overlapping blocks above): ceil(m/L) starts, start i =
 * floor(r_i (m - L + 1) / 2^64) from draw i of stream (k, REF_TAG_SELECTION);
 * each adds one to rows start .. start+L-1.  L <= 1: identical to
 * ref_selection_weights.  Requires L <= m. */
void ref_selection_weights_moving(int64_t m, int64_t block_len, uint64_t seed, uint64_t problem,
                                  int64_t k, uint32_t* w);

/* Estimation split for bootstrap k (Alg. 1/2 estimation loop, Fig. 1(c)):
 * units (rows or blocks) are reshuffled by sorting (draw, unit index); the
 * first floor(train_frac * units) units form the training pool, the rest the
 * evaluation set E^k.  T^k = as many unit draws with replacement from the
 * pool as the pool has units.  split_fixed != 0 uses bootstrap 0's reshuffle
 * for every k.  perm (nullable, length units) receives the reshuffle.
 * Returns REF_ERR_INVALID_ARG when the pool or E^k would be empty. */
int ref_estimation_weights(int64_t m, int64_t block_len, double train_frac, int split_fixed,
                           uint64_t seed, uint64_t problem, int64_t k,
                           uint32_t* w_train, uint8_t* eval_mask, int64_t* perm);

/* G = X^T diag(w) X (p x p), B = X^T diag(w) Y (p x r), yy[e] = sum_t w_t Y_te^2.
 * X is m x p with row stride ldx, Y is m x r with row stride ldy; w NULL = ones.
 * yy may be NULL. */
void ref_weighted_moments(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                          int64_t m, int64_t p, int64_t r, const uint32_t* w,
                          double* G, double* B, double* yy);

/* Textbook unblocked Cholesky A = L L^T (A, L p x p; upper part of L zeroed).
 * Returns 0, or -(j+1) when pivot j is not positive. */
int ref_cholesky(const double* A, int64_t p, double* L);

/* Solve L L^T x = b with a factor from ref_cholesky. */
void ref_cholesky_solve(const double* L, int64_t p, const double* b, double* x);

/* lambda_max = max_e || X^T y_e ||_inf / m over the full unweighted data. */
double ref_lambda_max(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                      int64_t m, int64_t p, int64_t r);

/* Descending log grid: lambda_j = lmax * ratio^(j/(q-1)), j = 0..q-1. */
void ref_lambda_grid(double lmax, int32_t q, double ratio, double* lambdas);

/* One LASSO column by scaled-form ADMM (Eq. 5), for the objective
 * (1/(2 nk)) ||y - X b||_W^2 + lambda ||b||_1 with G = X^T W X, bn = X^T W y / nk:
 *   x = (G/nk + rho I)^{-1} (bn + rho (z - u))      (x-minimisation)
 *   z = S_{lambda/rho}(x + u)                        (z-minimisation)
 *   u = u + x - z                                    (dual update)
 * stopping when ||x - z|| <= sqrt(p) abs + rel max(||x||, ||z||) and
 * rho ||z - z_prev|| <= sqrt(p) abs + rel rho ||u||.
 * L is the Cholesky factor of G/nk + rho I.  z, u hold the initial state on
 * entry and the final state on exit; x_out, v_out (nullable) receive the last
 * x and v = x + u.  Returns 1 when converged, 0 when max_iter was reached. */
int ref_admm_column(const double* L, const double* bn, int64_t p, double lambda, double rho,
                    double abs_tol, double rel_tol, int32_t max_iter,
                    double* z, double* u, double* x_out, double* v_out, int32_t* iters);

/* Exact LASSO minimiser by KKT polish (reference for the error statements of
 * forms that stop ADMM at a tolerance).  With H = G/nk and c = b/nk (reading 1's
 * scaling of Eq. 2), b* minimises (1/2) b^T H b - c^T b + lambda ||b||_1 exactly
 * when, with g = c - H b*,
 *   g_i = lambda sign(b*_i) on the support A of b*,  |g_i| <= lambda off it.
 * Given A and the signs s from z_start (the nonzeros of an ADMM iterate), the
 * rows of the first condition are the active-set equation H_AA b_A = c_A - lambda s_A,
 * solved by Cholesky in FP64.  The result is certified when every b_A has the
 * sign s and |g_i| <= lambda (1 + 1e-10) off A.  Otherwise one move is made and the
 * equation solved again: features whose sign flipped leave A; if none did, the
 * inactive feature with the largest |g_i| - lambda > 0 enters with the sign of
 * g_i (an active-set method, Osborne, Presnell and Turlach 2000).
 * G: p x p, b: p (stride ldb).  beta, grad: p.  moves (nullable): moves made.
 * Returns 0 when certified, 1 when max_moves ran out (beta then holds the last
 * solve), REF_ERR_NOT_PD when an active-set matrix is singular. */
int ref_kkt_polish(const double* G, const double* b, int64_t ldb, int64_t p, double nk,
                   double lambda, const double* z_start, int32_t max_moves,
                   double* beta, double* grad, int32_t* moves);

/* Batched LASSO-ADMM: for each bootstrap weight vector k (weights B x m, NULL =
 * one unweighted problem), each response column e < r and each lambda_j, one
 * ADMM column.  warm_start 0: z = u = 0 for every column; 1 (path): the column
 * (k, e, j) starts from the final (z, u) of (k, e, j-1).
 * beta_out: B x q x r x p (the final z).  iters_out, conv_out: B x q x r
 * (nullable).  v_out: B x q x r x p final x + u (nullable).
 * eq_list (nullable): only the r_sel response columns listed are solved, and
 * the outputs are laid out B x q x r_sel x p. */
int ref_lasso_admm_batch(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                         int64_t m, int64_t p, int64_t r, const uint32_t* weights, int32_t B,
                         const double* lambdas, int32_t q, double rho, double abs_tol,
                         double rel_tol, int32_t max_iter, int32_t warm_start,
                         const int64_t* eq_list, int64_t r_sel,
                         double* beta_out, int32_t* iters_out, uint8_t* conv_out, double* v_out);

/* LASSO with an unpenalised intercept for one weight vector w (m, NULL = ones):
 * minimises (1/(2 nk)) sum_t w_t (y_t - mu - x_t^T b)^2 + lambda ||b||_1 per
 * column.  The optimal mu for any b is ybar_w - xbar_w^T b, so this is the
 * plain LASSO (ref_lasso_admm_batch, B = 1) of the w-centred data, followed by
 * mu_out[j*r + e] = ybar_w[e] - xbar_w^T beta_{j,e}.  beta_out: q x r x p;
 * mu_out, iters_out, conv_out: q x r; v_out: q x r x p (all but beta nullable).
 * REF_ERR_INVALID_ARG when every weight is zero. */
int ref_lasso_admm_intercept(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                             int64_t m, int64_t p, int64_t r, const uint32_t* w,
                             const double* lambdas, int32_t q, double rho, double abs_tol,
                             double rel_tol, int32_t max_iter, int32_t warm_start,
                             double* beta_out, double* mu_out, int32_t* iters_out,
                             uint8_t* conv_out, double* v_out);

/* Lagged design of a VAR(d) (Eq. 7-8) from series (N x p, time ascending),
 * rows in ascending time: row t - d (t = d..N-1) holds Y = X_t and
 * X = (X_{t-1}, X_{t-2}, ..., X_{t-d}), lag j in columns (j-1)p .. jp-1.
 * X: (N-d) x dp, Y: (N-d) x p, both row-major and contiguous. */
void ref_lagged_design(const double* series, int64_t N, int64_t p, int32_t d, double* X, double* Y);

/* Least squares restricted to the support S (bitset of ceil(p/64) words):
 * beta_S = argmin || W^{1/2} (y - X_S beta) ||, minimum-norm when X_S is rank
 * deficient, zero outside S.  Uses Cholesky of G[S,S] when every pivot exceeds
 * 1e-12 * max diag(G[S,S]); otherwise a Jacobi eigendecomposition
 * pseudo-inverse.  Returns 0 (Cholesky path) or 1 (min-norm fallback). */
int ref_ols_support(const double* G, const double* b, int64_t ldb, int64_t p,
                    const uint64_t* S, double* beta);

/* Parameters of a full fit (the oracle's own struct). */
typedef struct {
    int32_t B1, B2, q;
    const double* lambdas;     /* q values, NULL = log grid from lambda_max */
    double lambda_min_ratio;   /* 1e-3 */
    double rho, abs_tol, rel_tol;
    int32_t max_iter;
    double train_frac;         /* 0.8 */
    uint64_t seed;
    uint64_t problem_id;
    int64_t block_len;         /* 0/1 = rows (LASSO), L > 1 = blocks (VAR) */
    int32_t bagging;           /* 0 median, 1 mean */
    int32_t split_fixed;       /* 0 per-bootstrap reshuffle, 1 fixed */
    int32_t warm_start;        /* 0 cold, 1 path */
    int32_t n_threads;         /* <= 1: sequential */
    int32_t intercept;         /* 1: every fit gains an unpenalised offset mu */
    int32_t block_mode;        /* selection blocks: 0 non-overlapping, 1 moving */
} ref_params;

/* Optional intermediate outputs (every pointer nullable). */
typedef struct {
    double*   lambdas;     /* q                                    */
    double*   sel_beta;    /* B1 x q x r x p  selection estimates  */
    double*   sel_v;       /* B1 x q x r x p  final x + u          */
    int32_t*  sel_iters;   /* B1 x q x r                           */
    uint8_t*  sel_conv;    /* B1 x q x r                           */
    uint64_t* family;      /* q x r x ceil(p/64)  S_j (Eq. 3)      */
    double*   est_beta;    /* B2 x q x r x pa  OLS on S_j from T^k (pa = p + intercept) */
    double*   est_loss;    /* B2 x q x r  held-out squared error sums per equation */
    int32_t*  est_jstar;   /* B2                                   */
    int32_t*  est_fallback;/* B2 x q x r  1 = min-norm fallback    */
    int32_t*  eval_count;  /* B2  |E^k| in rows                    */
} ref_trace;

/* Full UoI fit of r response columns that share the design X (m x p):
 * UoI_LASSO is r = 1 (Alg. 1); UoI_VAR(d) is the lagged design of Eq. 8 with
 * r = p (Alg. 2 with Eq. 9 solved as p LASSOs sharing that design).
 * beta_out: r x pa, pa = p + intercept (row e = the bagged coefficients of
 * response e, then its intercept when prm->intercept).  With an intercept the
 * selection fits are ref_lasso_admm_intercept, lambda_max comes from the
 * unweighted centred data, and the estimation OLS and held-out loss use the
 * design [X 1] with the ones column in every support. */
int ref_uoi_fit(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                int64_t m, int64_t p, int64_t r, const ref_params* prm,
                double* beta_out, ref_trace* trace);

/* UoI_LASSO (Alg. 1): X n x p, y n. */
int ref_uoi_lasso_fit(const double* X, const double* y, int64_t n, int64_t p,
                      const ref_params* prm, double* beta_out, ref_trace* trace);

/* UoI_VAR(order) (Alg. 2): series N x p, time ascending, order >= 1 and
 * N - order >= 2.  Fits the lagged design of ref_lagged_design, then
 * partitions beta* (Alg. 2, last step): A_out (order x p x p),
 * A_out[(j-1)*p*p + e*p + i] = coefficient of X_{t-j,i} in equation e;
 * mu_out (p, nullable) = the intercepts, zero when prm->intercept is 0. */
int ref_uoi_var_fit(const double* series, int64_t N, int64_t p, int32_t order,
                    const ref_params* prm, double* A_out, double* mu_out, ref_trace* trace);

#ifdef __cplusplus
}
#endif
#endif
