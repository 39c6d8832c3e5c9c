/*
 * uoi_oracle.c -- FP64 CPU oracle for the UoI_LASSO / UoI_VAR(d) hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see uoi_oracle.h).  Plain loops in the paper's
 * order; no blocking, fusion or reordering beyond what the definitions state.
 * Readings of places where the paper is silent are marked "Reading:".
 */
#include "uoi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x64-10, Salmon, Moraes, Dror, Shaw, SC'11, Sec. 5 (Philox-4x64):     */
/* two 64x64->128 multiplications per round, Weyl-sequence key schedule.      */
/* ------------------------------------------------------------------------- */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ull;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ull;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ull; /* golden ratio      */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73Bull; /* sqrt(3) - 1       */

static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(prod >> 64);
    *lo = (uint64_t)prod;
}

void ref_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {            /* key bump between rounds */
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mul_hi_lo(PHILOX_M0, c0, &hi0, &lo0);
        mul_hi_lo(PHILOX_M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint64_t ref_draw(uint64_t seed, uint64_t problem, uint64_t k, uint64_t tag, uint64_t i)
{
    uint64_t ctr[4] = { i >> 2, k, tag, 0 };
    uint64_t key[2] = { seed, problem };
    uint64_t out[4];
    ref_philox4x64_10(ctr, key, out);
    return out[i & 3u];
}

uint64_t ref_range_map(uint64_t r, uint64_t n)
{
    unsigned __int128 prod = (unsigned __int128)r * (unsigned __int128)n;
    return (uint64_t)(prod >> 64);
}

/* ------------------------------------------------------------------------- */
/* Bootstrap samples (Alg. 1 / Alg. 2 "Generate bootstrap sample T^k")       */
/* ------------------------------------------------------------------------- */
static int64_t unit_len(int64_t block_len) { return block_len > 1 ? block_len : 1; }

/* Reading: a unit is one row (UoI_LASSO) or one run of L consecutive rows of
 * the lagged pair (Y_t, X_{t-1}) (UoI_VAR block bootstrap, Sec. III-A-2). */
static void add_unit(uint32_t* w, int64_t m, int64_t L, int64_t unit)
{
    int64_t r0 = unit * L;
    int64_t r1 = r0 + L < m ? r0 + L : m;
    for (int64_t row = r0; row < r1; ++row) w[row] += 1u;
}

void ref_selection_weights(int64_t m, int64_t block_len, uint64_t seed, uint64_t problem,
                           int64_t k, uint32_t* w)
{
    int64_t L = unit_len(block_len);
    int64_t units = (m + L - 1) / L;
    memset(w, 0, (size_t)m * sizeof(uint32_t));
    for (int64_t i = 0; i < units; ++i) {
        uint64_t r = ref_draw(seed, problem, (uint64_t)k, REF_TAG_SELECTION, (uint64_t)i);
        int64_t unit = (int64_t)ref_range_map(r, (uint64_t)units);
        add_unit(w, m, L, unit);
    }
}

/* Moving-block variant (Kunsch's overlapping blocks): ceil(m/L) block starts
 * drawn uniformly from 0..m-L, each adding one to the L rows it covers.
 * Reading: an alternative to the non-overlapping blocks of Sec. III-A-2 for
 * the selection bootstrap only; with L <= 1 it is the row bootstrap. */
void ref_selection_weights_moving(int64_t m, int64_t block_len, uint64_t seed, uint64_t problem,
                                  int64_t k, uint32_t* w)
{
    int64_t L = unit_len(block_len);
    int64_t units = (m + L - 1) / L;
    memset(w, 0, (size_t)m * sizeof(uint32_t));
    for (int64_t i = 0; i < units; ++i) {
        uint64_t r = ref_draw(seed, problem, (uint64_t)k, REF_TAG_SELECTION, (uint64_t)i);
        int64_t start = (int64_t)ref_range_map(r, (uint64_t)(m - L + 1));
        for (int64_t row = start; row < start + L; ++row) w[row] += 1u;
    }
}

typedef struct { uint64_t key; int64_t unit; } keyed_unit;

static int cmp_keyed_unit(const void* a, const void* b)
{
    const keyed_unit* x = (const keyed_unit*)a;
    const keyed_unit* y = (const keyed_unit*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->unit != y->unit) return x->unit < y->unit ? -1 : 1;
    return 0;
}

int ref_estimation_weights(int64_t m, int64_t block_len, double train_frac, int split_fixed,
                           uint64_t seed, uint64_t problem, int64_t k,
                           uint32_t* w_train, uint8_t* eval_mask, int64_t* perm)
{
    int64_t L = unit_len(block_len);
    int64_t units = (m + L - 1) / L;
    int64_t pool = (int64_t)floor(train_frac * (double)units);
    if (pool < 1 || pool >= units) return REF_ERR_INVALID_ARG;

    /* Reshuffle: sort the units by their (64-bit draw, index) key. */
    keyed_unit* ku = (keyed_unit*)malloc((size_t)units * sizeof(keyed_unit));
    uint64_t split_k = split_fixed ? 0u : (uint64_t)k;
    for (int64_t u = 0; u < units; ++u) {
        ku[u].key = ref_draw(seed, problem, split_k, REF_TAG_SPLIT, (uint64_t)u);
        ku[u].unit = u;
    }
    qsort(ku, (size_t)units, sizeof(keyed_unit), cmp_keyed_unit);
    if (perm)
        for (int64_t u = 0; u < units; ++u) perm[u] = ku[u].unit;

    memset(w_train, 0, (size_t)m * sizeof(uint32_t));
    memset(eval_mask, 0, (size_t)m);
    for (int64_t pos = pool; pos < units; ++pos) {          /* E^k */
        int64_t r0 = ku[pos].unit * L;
        int64_t r1 = r0 + L < m ? r0 + L : m;
        for (int64_t row = r0; row < r1; ++row) eval_mask[row] = 1;
    }
    for (int64_t i = 0; i < pool; ++i) {                    /* T^k */
        uint64_t r = ref_draw(seed, problem, (uint64_t)k, REF_TAG_RESAMPLE, (uint64_t)i);
        int64_t pos = (int64_t)ref_range_map(r, (uint64_t)pool);
        add_unit(w_train, m, L, ku[pos].unit);
    }
    free(ku);
    return REF_OK;
}

/* ------------------------------------------------------------------------- */
/* Moments, Cholesky, lambda grid                                            */
/* ------------------------------------------------------------------------- */
void ref_weighted_moments(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                          int64_t m, int64_t p, int64_t r, const uint32_t* w,
                          double* G, double* B, double* yy)
{
    memset(G, 0, (size_t)(p * p) * sizeof(double));
    memset(B, 0, (size_t)(p * r) * sizeof(double));
    if (yy) memset(yy, 0, (size_t)r * sizeof(double));
    for (int64_t t = 0; t < m; ++t) {
        double wt = w ? (double)w[t] : 1.0;
        if (wt == 0.0) continue;
        const double* xt = X + t * ldx;
        const double* yt = Y + t * ldy;
        for (int64_t a = 0; a < p; ++a) {
            double wa = wt * xt[a];
            for (int64_t b = 0; b < p; ++b) G[a * p + b] += wa * xt[b];
            for (int64_t e = 0; e < r; ++e) B[a * r + e] += wa * yt[e];
        }
        if (yy)
            for (int64_t e = 0; e < r; ++e) yy[e] += wt * yt[e] * yt[e];
    }
}

int ref_cholesky(const double* A, int64_t p, double* L)
{
    memset(L, 0, (size_t)(p * p) * sizeof(double));
    for (int64_t j = 0; j < p; ++j) {
        double d = A[j * p + j];
        for (int64_t s = 0; s < j; ++s) d -= L[j * p + s] * L[j * p + s];
        if (!(d > 0.0)) return (int)(-(j + 1));
        double ljj = sqrt(d);
        L[j * p + j] = ljj;
        for (int64_t i = j + 1; i < p; ++i) {
            double v = A[i * p + j];
            for (int64_t s = 0; s < j; ++s) v -= L[i * p + s] * L[j * p + s];
            L[i * p + j] = v / ljj;
        }
    }
    return 0;
}

void ref_cholesky_solve(const double* L, int64_t p, const double* b, double* x)
{
    for (int64_t i = 0; i < p; ++i) {          /* L y = b */
        double v = b[i];
        for (int64_t s = 0; s < i; ++s) v -= L[i * p + s] * x[s];
        x[i] = v / L[i * p + i];
    }
    for (int64_t i = p - 1; i >= 0; --i) {     /* L^T x = y */
        double v = x[i];
        for (int64_t s = i + 1; s < p; ++s) v -= L[s * p + i] * x[s];
        x[i] = v / L[i * p + i];
    }
}

double ref_lambda_max(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                      int64_t m, int64_t p, int64_t r)
{
    double best = 0.0;
    for (int64_t e = 0; e < r; ++e)
        for (int64_t i = 0; i < p; ++i) {
            double s = 0.0;
            for (int64_t t = 0; t < m; ++t) s += X[t * ldx + i] * Y[t * ldy + e];
            double a = fabs(s) / (double)m;
            if (a > best) best = a;
        }
    return best;
}

void ref_lambda_grid(double lmax, int32_t q, double ratio, double* lambdas)
{
    for (int32_t j = 0; j < q; ++j)
        lambdas[j] = q > 1 ? lmax * pow(ratio, (double)j / (double)(q - 1)) : lmax;
}

/* ------------------------------------------------------------------------- */
/* LASSO by ADMM (Sec. II-E, Eq. 5), scaled form                             */
/* ------------------------------------------------------------------------- */
static double soft_threshold(double v, double kappa)
{
    if (v > kappa) return v - kappa;
    if (v < -kappa) return v + kappa;
    return 0.0;
}

int ref_admm_column(const double* L, const double* bn, int64_t p, double lambda, double rho,
                    double abs_tol, double rel_tol, int32_t max_iter,
                    double* z, double* u, double* x_out, double* v_out, int32_t* iters)
{
    double* rhs = (double*)malloc((size_t)p * sizeof(double));
    double* x = (double*)malloc((size_t)p * sizeof(double));
    double* v = (double*)malloc((size_t)p * sizeof(double));
    double kappa = lambda / rho;
    double sqrtp = sqrt((double)p);
    int converged = 0;
    int32_t it = 0;
    for (it = 1; it <= max_iter; ++it) {
        for (int64_t i = 0; i < p; ++i) rhs[i] = bn[i] + rho * (z[i] - u[i]);
        ref_cholesky_solve(L, p, rhs, x);                       /* x-minimisation */
        double r2 = 0.0, s2 = 0.0, x2 = 0.0, z2 = 0.0, u2 = 0.0;
        for (int64_t i = 0; i < p; ++i) {
            double z_prev = z[i];
            v[i] = x[i] + u[i];
            z[i] = soft_threshold(v[i], kappa);                 /* z-minimisation */
            u[i] = v[i] - z[i];                                 /* dual update    */
            double d = x[i] - z[i];
            double dz = z[i] - z_prev;
            r2 += d * d;
            s2 += dz * dz;
            x2 += x[i] * x[i];
            z2 += z[i] * z[i];
            u2 += u[i] * u[i];
        }
        double r_norm = sqrt(r2);
        double s_norm = rho * sqrt(s2);
        double xn = sqrt(x2), zn = sqrt(z2);
        double eps_pri = sqrtp * abs_tol + rel_tol * (xn > zn ? xn : zn);
        double eps_dual = sqrtp * abs_tol + rel_tol * rho * sqrt(u2);
        if (r_norm <= eps_pri && s_norm <= eps_dual) { converged = 1; break; }
    }
    if (it > max_iter) it = max_iter;
    if (iters) *iters = it;
    if (x_out) memcpy(x_out, x, (size_t)p * sizeof(double));
    if (v_out) memcpy(v_out, v, (size_t)p * sizeof(double));
    free(rhs); free(x); free(v);
    return converged;
}

/* ------------------------------------------------------------------------- */
/* Exact minimiser by KKT polish (optimality conditions of Eq. 2)            */
/* ------------------------------------------------------------------------- */
/* Solves H_AA b_A = c_A - lambda s_A for the active set A (H = G/nk, c = b/nk);
 * returns 0, or REF_ERR_NOT_PD when H_AA is not positive definite. */
static int active_set_solve(const double* G, const double* b, int64_t ldb, int64_t p, double nk,
                            double lambda, const int8_t* s, double* beta)
{
    int64_t* idx = (int64_t*)malloc((size_t)p * sizeof(int64_t));
    int64_t na = 0;
    for (int64_t i = 0; i < p; ++i)
        if (s[i]) idx[na++] = i;
    memset(beta, 0, (size_t)p * sizeof(double));
    int st = 0;
    if (na > 0) {
        double* H = (double*)malloc((size_t)(na * na) * sizeof(double));
        double* L = (double*)malloc((size_t)(na * na) * sizeof(double));
        double* rhs = (double*)malloc((size_t)na * sizeof(double));
        double* x = (double*)malloc((size_t)na * sizeof(double));
        for (int64_t a = 0; a < na; ++a) {
            for (int64_t c = 0; c < na; ++c) H[a * na + c] = G[idx[a] * p + idx[c]] / nk;
            rhs[a] = b[idx[a] * ldb] / nk - lambda * (double)s[idx[a]];
        }
        if (ref_cholesky(H, na, L) != 0) {
            st = REF_ERR_NOT_PD;
        } else {
            ref_cholesky_solve(L, na, rhs, x);
            for (int64_t a = 0; a < na; ++a) beta[idx[a]] = x[a];
        }
        free(H); free(L); free(rhs); free(x);
    }
    free(idx);
    return st;
}

int ref_kkt_polish(const double* G, const double* b, int64_t ldb, int64_t p, double nk,
                   double lambda, const double* z_start, int32_t max_moves,
                   double* beta, double* grad, int32_t* moves)
{
    int8_t* s = (int8_t*)malloc((size_t)p);
    for (int64_t i = 0; i < p; ++i)
        s[i] = z_start[i] > 0.0 ? 1 : (z_start[i] < 0.0 ? -1 : 0);
    int32_t mv = 0;
    int status = 1;
    for (;;) {
        int st = active_set_solve(G, b, ldb, p, nk, lambda, s, beta);
        if (st != 0) { status = st; break; }
        /* g = c - H beta */
        for (int64_t i = 0; i < p; ++i) {
            double hb = 0.0;
            for (int64_t j = 0; j < p; ++j) hb += G[i * p + j] * beta[j];
            grad[i] = (b[i * ldb] - hb) / nk;
        }
        /* sign condition on A */
        int flipped = 0;
        for (int64_t i = 0; i < p; ++i)
            if (s[i] && !((double)s[i] * beta[i] > 0.0)) flipped = 1;
        /* inactive condition off A: the largest violation */
        int64_t worst = -1;
        double worst_excess = 0.0;
        for (int64_t i = 0; i < p; ++i) {
            if (s[i]) continue;
            double excess = fabs(grad[i]) - lambda * (1.0 + 1e-10);
            if (excess > worst_excess) { worst_excess = excess; worst = i; }
        }
        if (!flipped && worst < 0) { status = 0; break; }
        if (mv >= max_moves) break;
        ++mv;
        if (flipped) {
            for (int64_t i = 0; i < p; ++i)
                if (s[i] && !((double)s[i] * beta[i] > 0.0)) s[i] = 0;
        } else {
            s[worst] = grad[worst] > 0.0 ? 1 : -1;
        }
    }
    if (moves) *moves = mv;
    free(s);
    return status;
}

/* A = G / nk + rho I */
static void admm_system(const double* G, int64_t p, double nk, double rho, double* A)
{
    for (int64_t a = 0; a < p; ++a)
        for (int64_t b = 0; b < p; ++b)
            A[a * p + b] = G[a * p + b] / nk + (a == b ? rho : 0.0);
}

static uint64_t sum_weights(const uint32_t* w, int64_t m)
{
    uint64_t s = 0;
    for (int64_t t = 0; t < m; ++t) s += w ? w[t] : 1u;
    return s;
}

int ref_lasso_admm_batch(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                         int64_t m, int64_t p, int64_t r, const uint32_t* weights, int32_t B,
                         const double* lambdas, int32_t q, double rho, double abs_tol,
                         double rel_tol, int32_t max_iter, int32_t warm_start,
                         const int64_t* eq_list, int64_t r_sel,
                         double* beta_out, int32_t* iters_out, uint8_t* conv_out, double* v_out)
{
    if (!X || !Y || m <= 0 || p <= 0 || r <= 0 || q <= 0 || B <= 0 || !(rho > 0.0) || !lambdas)
        return REF_ERR_INVALID_ARG;
    if (!weights && B != 1) return REF_ERR_INVALID_ARG;
    int64_t re = eq_list ? r_sel : r;
    double* G = (double*)malloc((size_t)(p * p) * sizeof(double));
    double* Bm = (double*)malloc((size_t)(p * r) * sizeof(double));
    double* A = (double*)malloc((size_t)(p * p) * sizeof(double));
    double* L = (double*)malloc((size_t)(p * p) * sizeof(double));
    double* bn = (double*)malloc((size_t)p * sizeof(double));
    double* z = (double*)malloc((size_t)p * sizeof(double));
    double* u = (double*)malloc((size_t)p * sizeof(double));
    int status = REF_OK;
    for (int32_t k = 0; k < B && status >= 0; ++k) {
        const uint32_t* w = weights ? weights + (int64_t)k * m : NULL;
        double nk = (double)sum_weights(w, m);
        ref_weighted_moments(X, ldx, Y, ldy, m, p, r, w, G, Bm, NULL);
        admm_system(G, p, nk, rho, A);
        if (ref_cholesky(A, p, L) != 0) { status = REF_ERR_NOT_PD; break; }
        for (int64_t es = 0; es < re; ++es) {
            int64_t e = eq_list ? eq_list[es] : es;
            for (int64_t i = 0; i < p; ++i) bn[i] = Bm[i * r + e] / nk;
            memset(z, 0, (size_t)p * sizeof(double));
            memset(u, 0, (size_t)p * sizeof(double));
            for (int32_t j = 0; j < q; ++j) {
                if (!warm_start) {
                    memset(z, 0, (size_t)p * sizeof(double));
                    memset(u, 0, (size_t)p * sizeof(double));
                }
                int64_t col = ((int64_t)k * q + j) * re + es;
                int32_t its = 0;
                int conv = ref_admm_column(L, bn, p, lambdas[j], rho, abs_tol, rel_tol, max_iter,
                                           z, u, NULL, v_out ? v_out + col * p : NULL, &its);
                memcpy(beta_out + col * p, z, (size_t)p * sizeof(double));
                if (iters_out) iters_out[col] = its;
                if (conv_out) conv_out[col] = (uint8_t)conv;
                if (!conv) status = REF_OK_WITH_WARNINGS;
            }
        }
    }
    free(G); free(Bm); free(A); free(L); free(bn); free(z); free(u);
    return status;
}

/* ------------------------------------------------------------------------- */
/* OLS restricted to a support (Alg. 1 estimation "Compute OLS estimate")    */
/* ------------------------------------------------------------------------- */

/* Cyclic Jacobi eigendecomposition of a symmetric s x s matrix (Golub & Van
 * Loan, Sec. 8.5): on exit A holds the eigenvalues on its diagonal and V the
 * eigenvectors in its columns. */
static void jacobi_eigen(double* A, double* V, int64_t s)
{
    for (int64_t i = 0; i < s; ++i)
        for (int64_t j = 0; j < s; ++j) V[i * s + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int64_t i = 0; i < s; ++i)
            for (int64_t j = 0; j < s; ++j) {
                tot += A[i * s + j] * A[i * s + j];
                if (i != j) off += A[i * s + j] * A[i * s + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int64_t a = 0; a < s; ++a)
            for (int64_t b = a + 1; b < s; ++b) {
                double apq = A[a * s + b];
                if (apq == 0.0) continue;
                double theta = (A[b * s + b] - A[a * s + a]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double sn = t * c;
                for (int64_t kk = 0; kk < s; ++kk) {      /* columns a, b */
                    double ka = A[kk * s + a], kb = A[kk * s + b];
                    A[kk * s + a] = c * ka - sn * kb;
                    A[kk * s + b] = sn * ka + c * kb;
                }
                for (int64_t kk = 0; kk < s; ++kk) {      /* rows a, b */
                    double ak = A[a * s + kk], bk = A[b * s + kk];
                    A[a * s + kk] = c * ak - sn * bk;
                    A[b * s + kk] = sn * ak + c * bk;
                }
                for (int64_t kk = 0; kk < s; ++kk) {
                    double va = V[kk * s + a], vb = V[kk * s + b];
                    V[kk * s + a] = c * va - sn * vb;
                    V[kk * s + b] = sn * va + c * vb;
                }
            }
    }
}

int ref_ols_support(const double* G, const double* b, int64_t ldb, int64_t p,
                    const uint64_t* S, double* beta)
{
    int64_t* idx = (int64_t*)malloc((size_t)p * sizeof(int64_t));
    int64_t s = 0;
    for (int64_t i = 0; i < p; ++i)
        if ((S[i >> 6] >> (i & 63)) & 1u) idx[s++] = i;
    memset(beta, 0, (size_t)p * sizeof(double));
    if (s == 0) { free(idx); return 0; }

    double* Gs = (double*)malloc((size_t)(s * s) * sizeof(double));
    double* L = (double*)malloc((size_t)(s * s) * sizeof(double));
    double* bs = (double*)malloc((size_t)s * sizeof(double));
    double* xs = (double*)malloc((size_t)s * sizeof(double));
    double dmax = 0.0;
    for (int64_t a = 0; a < s; ++a) {
        for (int64_t c = 0; c < s; ++c) Gs[a * s + c] = G[idx[a] * p + idx[c]];
        bs[a] = b[idx[a] * ldb];
        if (Gs[a * s + a] > dmax) dmax = Gs[a * s + a];
    }
    /* Cholesky with the pivot test d_j > 1e-12 * max diag. */
    int ok = dmax > 0.0;
    memset(L, 0, (size_t)(s * s) * sizeof(double));
    for (int64_t j = 0; j < s && ok; ++j) {
        double d = Gs[j * s + j];
        for (int64_t t = 0; t < j; ++t) d -= L[j * s + t] * L[j * s + t];
        if (!(d > 1e-12 * dmax)) { ok = 0; break; }
        double ljj = sqrt(d);
        L[j * s + j] = ljj;
        for (int64_t i = j + 1; i < s; ++i) {
            double v = Gs[i * s + j];
            for (int64_t t = 0; t < j; ++t) v -= L[i * s + t] * L[j * s + t];
            L[i * s + j] = v / ljj;
        }
    }
    int fallback = 0;
    if (ok) {
        ref_cholesky_solve(L, s, bs, xs);
    } else {
        /* Minimum-norm solution G^+ b via the eigendecomposition of G[S,S]. */
        fallback = 1;
        double* V = L;
        jacobi_eigen(Gs, V, s);
        double emax = 0.0;
        for (int64_t a = 0; a < s; ++a) if (Gs[a * s + a] > emax) emax = Gs[a * s + a];
        for (int64_t a = 0; a < s; ++a) xs[a] = 0.0;
        for (int64_t c = 0; c < s; ++c) {
            double ev = Gs[c * s + c];
            if (!(ev > 1e-12 * emax)) continue;
            double proj = 0.0;
            for (int64_t a = 0; a < s; ++a) proj += V[a * s + c] * bs[a];
            proj /= ev;
            for (int64_t a = 0; a < s; ++a) xs[a] += V[a * s + c] * proj;
        }
    }
    for (int64_t a = 0; a < s; ++a) beta[idx[a]] = xs[a];
    free(idx); free(Gs); free(L); free(bs); free(xs);
    return fallback;
}

/* ------------------------------------------------------------------------- */
/* Unpenalised intercept (Alg. 2 returns mu next to A_1..A_d; the paper does  */
/* not say how it is fitted).  Reading: the objective of every fit gains a    */
/* free offset, (1/(2 nk)) sum_t w_t (y_t - mu - x_t^T b)^2 + lambda ||b||_1.  */
/* For fixed b the best mu is ybar_w - xbar_w^T b (w-weighted means), and     */
/* putting it back leaves the plain LASSO of the w-centred data.              */
/* ------------------------------------------------------------------------- */
static int weighted_means(const double* A, int64_t lda, int64_t m, int64_t c, const uint32_t* w,
                          double* mean)
{
    double n = 0.0;
    for (int64_t i = 0; i < c; ++i) mean[i] = 0.0;
    for (int64_t t = 0; t < m; ++t) {
        double wt = w ? (double)w[t] : 1.0;
        if (wt == 0.0) continue;
        n += wt;
        for (int64_t i = 0; i < c; ++i) mean[i] += wt * A[t * lda + i];
    }
    if (!(n > 0.0)) return -1;
    for (int64_t i = 0; i < c; ++i) mean[i] /= n;
    return 0;
}

static double* centred_copy(const double* A, int64_t lda, int64_t m, int64_t c, const double* mean)
{
    double* out = (double*)malloc((size_t)(m * c) * sizeof(double));
    for (int64_t t = 0; t < m; ++t)
        for (int64_t i = 0; i < c; ++i) out[t * c + i] = A[t * lda + i] - mean[i];
    return out;
}

int ref_lasso_admm_intercept(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                             int64_t m, int64_t p, int64_t r, const uint32_t* w,
                             const double* lambdas, int32_t q, double rho, double abs_tol,
                             double rel_tol, int32_t max_iter, int32_t warm_start,
                             double* beta_out, double* mu_out, int32_t* iters_out,
                             uint8_t* conv_out, double* v_out)
{
    if (!X || !Y || !lambdas || !beta_out || m <= 0 || p <= 0 || r <= 0 || q <= 0)
        return REF_ERR_INVALID_ARG;
    double* xbar = (double*)malloc((size_t)p * sizeof(double));
    double* ybar = (double*)malloc((size_t)r * sizeof(double));
    if (weighted_means(X, ldx, m, p, w, xbar) || weighted_means(Y, ldy, m, r, w, ybar)) {
        free(xbar); free(ybar);
        return REF_ERR_INVALID_ARG;                  /* every weight zero */
    }
    double* Xc = centred_copy(X, ldx, m, p, xbar);
    double* Yc = centred_copy(Y, ldy, m, r, ybar);
    int st = ref_lasso_admm_batch(Xc, p, Yc, r, m, p, r, w, 1, lambdas, q, rho, abs_tol, rel_tol,
                                  max_iter, warm_start, NULL, 0, beta_out, iters_out, conv_out, v_out);
    if (st >= 0 && mu_out)
        for (int32_t j = 0; j < q; ++j)
            for (int64_t e = 0; e < r; ++e) {
                const double* b = beta_out + ((int64_t)j * r + e) * p;
                double mu = ybar[e];
                for (int64_t i = 0; i < p; ++i) mu -= xbar[i] * b[i];
                mu_out[(int64_t)j * r + e] = mu;
            }
    free(xbar); free(ybar); free(Xc); free(Yc);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Lagged design of a VAR(d) (Eq. 7-8), rows in ascending time               */
/* ------------------------------------------------------------------------- */
void ref_lagged_design(const double* series, int64_t N, int64_t p, int32_t d, double* X, double* Y)
{
    const int64_t P = (int64_t)d * p;
    for (int64_t t = d; t < N; ++t) {
        const int64_t row = t - d;
        for (int64_t e = 0; e < p; ++e) Y[row * p + e] = series[t * p + e];       /* X_t      */
        for (int32_t j = 1; j <= d; ++j)                                            /* X_{t-j}  */
            for (int64_t c = 0; c < p; ++c)
                X[row * P + (int64_t)(j - 1) * p + c] = series[(t - j) * p + c];
    }
}

/* ------------------------------------------------------------------------- */
/* Full fit: Alg. 1 (r = 1) and Alg. 2 (r = p, lagged design)                */
/* ------------------------------------------------------------------------- */
static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

int ref_uoi_fit(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                int64_t m, int64_t p, int64_t r, const ref_params* prm,
                double* beta_out, ref_trace* trace)
{
    if (!X || !Y || !prm || !beta_out || m <= 0 || p <= 0 || r <= 0) return REF_ERR_INVALID_ARG;
    if (prm->B1 <= 0 || prm->B2 <= 0 || prm->q <= 0 || !(prm->rho > 0.0) || prm->max_iter <= 0)
        return REF_ERR_INVALID_ARG;
    if (!(prm->train_frac > 0.0 && prm->train_frac < 1.0)) return REF_ERR_INVALID_ARG;
    if (prm->block_len > m) return REF_ERR_INVALID_ARG;
    for (int64_t t = 0; t < m; ++t) {
        for (int64_t i = 0; i < p; ++i) if (!isfinite(X[t * ldx + i])) return REF_ERR_NONFINITE;
        for (int64_t e = 0; e < r; ++e) if (!isfinite(Y[t * ldy + e])) return REF_ERR_NONFINITE;
    }
    const int32_t B1 = prm->B1, B2 = prm->B2, q = prm->q;
    const int64_t W = (p + 63) / 64;
    /* with an intercept the estimation works on pa = p + 1 coordinates: the p
     * features, then mu (a column of ones that every support contains) */
    const int icpt = prm->intercept != 0;
    const int64_t pa = p + icpt;
    const int64_t Wa = (pa + 63) / 64;
    int status = REF_OK;

    /* lambda grid (Eq. 2 scaled by 1/(2 nk); descending) */
    double* lam = (double*)malloc((size_t)q * sizeof(double));
    if (prm->lambdas) {
        memcpy(lam, prm->lambdas, (size_t)q * sizeof(double));
    } else if (icpt) {
        /* Reading: with an intercept, lambda_max of the (unweighted) centred data */
        double* xbar = (double*)malloc((size_t)p * sizeof(double));
        double* ybar = (double*)malloc((size_t)r * sizeof(double));
        weighted_means(X, ldx, m, p, NULL, xbar);
        weighted_means(Y, ldy, m, r, NULL, ybar);
        double* Xc = centred_copy(X, ldx, m, p, xbar);
        double* Yc = centred_copy(Y, ldy, m, r, ybar);
        ref_lambda_grid(ref_lambda_max(Xc, p, Yc, r, m, p, r), q, prm->lambda_min_ratio, lam);
        free(xbar); free(ybar); free(Xc); free(Yc);
    } else {
        double lmax = ref_lambda_max(X, ldx, Y, ldy, m, p, r);
        ref_lambda_grid(lmax, q, prm->lambda_min_ratio, lam);
    }
    if (trace && trace->lambdas) memcpy(trace->lambdas, lam, (size_t)q * sizeof(double));

    /* ---- Model selection (Alg. 1 selection loop, Eq. 3) ---- */
    uint64_t* sup = (uint64_t*)calloc((size_t)((int64_t)B1 * q * r * W), sizeof(uint64_t));
    int sel_status = REF_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(prm->n_threads > 1 ? prm->n_threads : 1)
#endif
    for (int32_t k = 0; k < B1; ++k) {
        uint32_t* w = (uint32_t*)malloc((size_t)m * sizeof(uint32_t));
        double* beta = (double*)malloc((size_t)q * r * p * sizeof(double));
        double* v = (double*)malloc((size_t)q * r * p * sizeof(double));
        int32_t* its = (int32_t*)malloc((size_t)q * r * sizeof(int32_t));
        uint8_t* cv = (uint8_t*)malloc((size_t)q * r);
        if (prm->block_mode == 1)
            ref_selection_weights_moving(m, prm->block_len, prm->seed, prm->problem_id, k, w);
        else
            ref_selection_weights(m, prm->block_len, prm->seed, prm->problem_id, k, w);
        int st = icpt ? ref_lasso_admm_intercept(X, ldx, Y, ldy, m, p, r, w, lam, q, prm->rho,
                                                 prm->abs_tol, prm->rel_tol, prm->max_iter,
                                                 prm->warm_start, beta, NULL, its, cv, v)
                      : ref_lasso_admm_batch(X, ldx, Y, ldy, m, p, r, w, 1, lam, q, prm->rho,
                                             prm->abs_tol, prm->rel_tol, prm->max_iter,
                                             prm->warm_start, NULL, 0, beta, its, cv, v);
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (st < 0 || (st > sel_status && sel_status >= 0)) sel_status = st;
        }
        for (int32_t j = 0; j < q; ++j)
            for (int64_t e = 0; e < r; ++e) {
                int64_t col = (int64_t)j * r + e;
                uint64_t* bits = sup + (((int64_t)k * q + j) * r + e) * W;
                for (int64_t i = 0; i < p; ++i)                  /* S_j^k */
                    if (beta[col * p + i] != 0.0) bits[i >> 6] |= 1ull << (i & 63);
                int64_t gcol = (int64_t)k * q * r + col;
                if (trace && trace->sel_beta)
                    memcpy(trace->sel_beta + gcol * p, beta + col * p, (size_t)p * sizeof(double));
                if (trace && trace->sel_v)
                    memcpy(trace->sel_v + gcol * p, v + col * p, (size_t)p * sizeof(double));
                if (trace && trace->sel_iters) trace->sel_iters[gcol] = its[col];
                if (trace && trace->sel_conv) trace->sel_conv[gcol] = cv[col];
            }
        free(w); free(beta); free(v); free(its); free(cv);
    }
    if (sel_status < 0) { free(lam); free(sup); return sel_status; }
    if (sel_status > status) status = sel_status;

    /* S_j = AND over k of S_j^k, per response column (Eq. 3) */
    uint64_t* fam = (uint64_t*)malloc((size_t)((int64_t)q * r * W) * sizeof(uint64_t));
    for (int64_t c = 0; c < (int64_t)q * r; ++c)
        for (int64_t wd = 0; wd < W; ++wd) {
            uint64_t acc = ~0ull;
            for (int32_t k = 0; k < B1; ++k) acc &= sup[((int64_t)k * q * r + c) * W + wd];
            if (wd == W - 1 && (p & 63)) acc &= (1ull << (p & 63)) - 1ull;
            fam[c * W + wd] = acc;
        }
    if (trace && trace->family) memcpy(trace->family, fam, (size_t)q * r * W * sizeof(uint64_t));

    /* ---- Model estimation (Alg. 1 estimation loop, Eq. 4) ---- */
    /* design and supports of the estimation: X and S_j, or [X 1] and S_j + {mu} */
    const double* Xe = X;
    int64_t lde = ldx;
    const uint64_t* fe = fam;
    double* Xa = NULL;
    uint64_t* fa = NULL;
    if (icpt) {
        Xa = (double*)malloc((size_t)(m * pa) * sizeof(double));
        for (int64_t t = 0; t < m; ++t) {
            for (int64_t i = 0; i < p; ++i) Xa[t * pa + i] = X[t * ldx + i];
            Xa[t * pa + p] = 1.0;
        }
        fa = (uint64_t*)calloc((size_t)((int64_t)q * r * Wa), sizeof(uint64_t));
        for (int64_t c = 0; c < (int64_t)q * r; ++c) {
            for (int64_t wd = 0; wd < W; ++wd) fa[c * Wa + wd] = fam[c * W + wd];
            fa[c * Wa + (p >> 6)] |= 1ull << (p & 63);
        }
        Xe = Xa; lde = pa; fe = fa;
    }
    const int64_t We = icpt ? Wa : W;
    double* chosen = (double*)malloc((size_t)B2 * r * pa * sizeof(double));
    int est_status = REF_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(prm->n_threads > 1 ? prm->n_threads : 1)
#endif
    for (int32_t k = 0; k < B2; ++k) {
        uint32_t* wt = (uint32_t*)malloc((size_t)m * sizeof(uint32_t));
        uint8_t* ev = (uint8_t*)malloc((size_t)m);
        double* G = (double*)malloc((size_t)(pa * pa) * sizeof(double));
        double* Bm = (double*)malloc((size_t)(pa * r) * sizeof(double));
        double* ols = (double*)malloc((size_t)q * r * pa * sizeof(double));
        double* loss = (double*)malloc((size_t)q * sizeof(double));
        int st = ref_estimation_weights(m, prm->block_len, prm->train_frac, prm->split_fixed,
                                        prm->seed, prm->problem_id, k, wt, ev, NULL);
        int32_t n_eval = 0;
        for (int64_t t = 0; t < m; ++t) n_eval += ev[t];
        if (st == REF_OK) {
            ref_weighted_moments(Xe, lde, Y, ldy, m, pa, r, wt, G, Bm, NULL);
            for (int32_t j = 0; j < q; ++j) {
                loss[j] = 0.0;
                for (int64_t e = 0; e < r; ++e) {
                    int64_t col = (int64_t)j * r + e;
                    double* bj = ols + col * pa;
                    int fb = ref_ols_support(G, Bm + e, r, pa, fe + col * We, bj);
                    if (fb) {
#ifdef _OPENMP
#pragma omp critical
#endif
                        { if (est_status == REF_OK) est_status = REF_OK_WITH_WARNINGS; }
                    }
                    /* held-out loss on E^k: explicit residuals */
                    double le = 0.0;
                    for (int64_t t = 0; t < m; ++t) {
                        if (!ev[t]) continue;
                        double pred = 0.0;
                        for (int64_t i = 0; i < pa; ++i) pred += Xe[t * lde + i] * bj[i];
                        double res = Y[t * ldy + e] - pred;
                        le += res * res;
                    }
                    loss[j] += le;
                    if (trace && trace->est_loss)
                        trace->est_loss[((int64_t)k * q + j) * r + e] = le;
                    if (trace && trace->est_fallback)
                        trace->est_fallback[((int64_t)k * q + j) * r + e] = fb;
                    if (trace && trace->est_beta)
                        memcpy(trace->est_beta + (((int64_t)k * q + j) * r + e) * pa, bj,
                               (size_t)pa * sizeof(double));
                }
            }
            /* best model for this bootstrap: argmin over j, ties -> smallest j */
            int32_t jbest = 0;
            for (int32_t j = 1; j < q; ++j) if (loss[j] < loss[jbest]) jbest = j;
            memcpy(chosen + (int64_t)k * r * pa, ols + (int64_t)jbest * r * pa,
                   (size_t)r * pa * sizeof(double));
            if (trace && trace->est_jstar) trace->est_jstar[k] = jbest;
        } else {
#ifdef _OPENMP
#pragma omp critical
#endif
            { est_status = st; }
        }
        if (trace && trace->eval_count) trace->eval_count[k] = n_eval;
        free(wt); free(ev); free(G); free(Bm); free(ols); free(loss);
    }
    free(Xa); free(fa);
    if (est_status < 0) { free(lam); free(sup); free(fam); free(chosen); return est_status; }
    if (est_status > status) status = est_status;

    /* bagging over the B2 chosen estimates (median or mean, Eq. 4) */
    double* col = (double*)malloc((size_t)B2 * sizeof(double));
    for (int64_t c = 0; c < r * pa; ++c) {
        for (int32_t k = 0; k < B2; ++k) col[k] = chosen[(int64_t)k * r * pa + c];
        double out;
        if (prm->bagging == 1) {
            double s = 0.0;
            for (int32_t k = 0; k < B2; ++k) s += col[k];
            out = s / (double)B2;
        } else {
            qsort(col, (size_t)B2, sizeof(double), cmp_double);
            out = (B2 & 1) ? col[B2 / 2] : 0.5 * (col[B2 / 2 - 1] + col[B2 / 2]);
        }
        beta_out[c] = out;
    }
    free(col); free(lam); free(sup); free(fam); free(chosen);
    return status;
}

int ref_uoi_lasso_fit(const double* X, const double* y, int64_t n, int64_t p,
                      const ref_params* prm, double* beta_out, ref_trace* trace)
{
    return ref_uoi_fit(X, p, y, 1, n, p, 1, prm, beta_out, trace);
}

int ref_uoi_var_fit(const double* series, int64_t N, int64_t p, int32_t order,
                    const ref_params* prm, double* A_out, double* mu_out, ref_trace* trace)
{
    if (!series || !prm || !A_out || p <= 0 || order < 1) return REF_ERR_INVALID_ARG;
    if (N - order < 2) return REF_ERR_INVALID_ARG;
    /* Eq. 7-9: row t - d of the design pairs the response X_t with the
     * regressors (X_{t-1}, ..., X_{t-d}), t = d..N-1.  Row order does not change
     * any Gram; it fixes which rows a block of the block bootstrap holds. */
    const int64_t m = N - order, P = (int64_t)order * p;
    const int icpt = prm->intercept != 0;
    const int64_t pa = P + icpt;
    double* X = (double*)malloc((size_t)(m * P) * sizeof(double));
    double* Y = (double*)malloc((size_t)(m * p) * sizeof(double));
    double* beta = (double*)malloc((size_t)(p * pa) * sizeof(double));
    ref_lagged_design(series, N, p, order, X, Y);
    int st = ref_uoi_fit(X, P, Y, p, m, P, p, prm, beta, trace);
    if (st >= 0) {
        /* Alg. 2: partition beta* into A_1..A_d and mu */
        for (int32_t j = 0; j < order; ++j)
            for (int64_t e = 0; e < p; ++e)
                for (int64_t c = 0; c < p; ++c)
                    A_out[((int64_t)j * p + e) * p + c] = beta[e * pa + (int64_t)j * p + c];
        if (mu_out)
            for (int64_t e = 0; e < p; ++e) mu_out[e] = icpt ? beta[e * pa + P] : 0.0;
    }
    free(X); free(Y); free(beta);
    return st;
}
