// design.cu -- VAR(d) lagged design and the unpenalised intercept.
//
// Alg. 2 fits a VAR(d) through the lagged design of Eq. 7-8 (response X_t,
// regressors X_{t-1} .. X_{t-d}) and returns the intercept mu beside
// A_1 .. A_d.  The intercept is an unpenalised offset in every fit:
//   (1/(2 n_k)) sum_t w_t (y_t - mu - x_t^T b)^2 + lambda ||b||_1.
// GPU form: the design is centred once by its unweighted column means and a
// column of ones is appended (index p).  The Gram kernels then produce the
// (p+1) x (p+1) moments of [X~ 1] for each bootstrap; eliminating the ones
// coordinate (the Schur complement G - g g^T / n_k, g = X~^T w) leaves the
// moments of the w-centred data, i.e. the LASSO with mu profiled out, and the
// ADMM runs unchanged on p columns.  The estimation keeps the ones column in
// every support, so the OLS fits (b, mu~) jointly and the held-out loss counts
// mu~.  mu~ is mapped back to the original coordinates before bagging:
// mu = mu~ + ybar - xbar^T b.  Centring first keeps the Schur step free of
// cancellation when the columns have large means (the tensor-core Gram is
// FP32-accurate, relative to the size of its entries).
#include "kernels.h"

#include <algorithm>

namespace uoi {
namespace {

// Row t - d (t = d .. N-1) of Eq. 7-8: Y = X_t, X = (X_{t-1}, ..., X_{t-d}).
__global__ void k_lagged_design(const double* __restrict__ S, int64_t N, int64_t p, int d,
                                double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                int64_t ldy)
{
    const int64_t m = N - d;
    const int64_t cols = (int64_t)(d + 1) * p;
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y) {
        const int64_t t = i + d;
        for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cols;
             c += (int64_t)gridDim.x * blockDim.x) {
            if (c < p) {
                Y[i * ldy + c] = S[t * p + c];
            } else {
                const int64_t lag = (c - p) / p + 1, cc = (c - p) % p;
                X[i * ldx + (lag - 1) * p + cc] = S[(t - lag) * p + cc];
            }
        }
    }
}

// part[chunk * c + j] = sum of A[i, j] over the chunk's `rows` rows (fixed order).
__global__ void k_col_partial(const double* __restrict__ A, int64_t lda, int64_t m, int64_t c,
                              int64_t rows, double* __restrict__ part)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= c) return;
    const int64_t i0 = (int64_t)blockIdx.y * rows, i1 = min(m, i0 + rows);
    double acc = 0.0;
    for (int64_t i = i0; i < i1; ++i) acc += A[i * lda + j];
    part[(int64_t)blockIdx.y * c + j] = acc;
}

__global__ void k_col_finish(const double* __restrict__ part, int64_t chunks, int64_t c, int64_t m,
                             double* __restrict__ mean)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= c) return;
    double acc = 0.0;
    for (int64_t k = 0; k < chunks; ++k) acc += part[k * c + j];
    mean[j] = acc / (double)m;
}

// dst[i, j] = src[i, j] - mean[j] (j < c); dst[i, c] = 1 when ones.
__global__ void k_center_copy(const double* __restrict__ src, int64_t lds, int64_t m, int64_t c,
                              const double* __restrict__ mean, int ones, double* __restrict__ dst,
                              int64_t ldd)
{
    const int64_t cols = c + (ones ? 1 : 0);
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y)
        for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols;
             j += (int64_t)gridDim.x * blockDim.x)
            dst[i * ldd + j] = j < c ? src[i * lds + j] - mean[j] : 1.0;
}

// G_k = Ga_k[:p, :p] - g g^T / n_k and Bm_k = Ba_k[:p, :] - g b^T / n_k with
// g = Ga_k[:p, p] (= X~^T w_k) and b = Ba_k[p, :] (= Y~^T w_k).
__global__ void k_schur_intercept(const double* __restrict__ Ga, const double* __restrict__ Ba,
                                  const double* __restrict__ nk, int nk_count, int64_t p, int64_t r,
                                  int32_t B, double* __restrict__ G, double* __restrict__ Bm)
{
    const int64_t pa = p + 1;
    const int64_t per = p * p + p * r;
    const int64_t total = per * B;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = x / per, o = x % per;
        const double n = nk[nk_count > 1 ? k : 0];
        const double* ga = Ga + k * pa * pa;
        if (o < p * p) {
            const int64_t i = o / p, j = o % p;
            G[k * p * p + o] = ga[i * pa + j] - ga[i * pa + p] * ga[j * pa + p] / n;
        } else {
            const int64_t q = o - p * p, i = q / r, e = q % r;
            const double* ba = Ba + k * pa * r;
            Bm[k * p * r + q] = ba[i * r + e] - ga[i * pa + p] * ba[p * r + e] / n;
        }
    }
}

// out[c] = fam[c] with bit `bit` set, re-packed from W to Wa words per member.
__global__ void k_family_add_bit(const uint64_t* __restrict__ fam, int64_t count, int64_t W,
                                 int64_t Wa, int64_t bit, uint64_t* __restrict__ out)
{
    const int64_t total = count * Wa;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = x / Wa, w = x % Wa;
        uint64_t v = w < W ? fam[c * W + w] : 0ull;
        if (w == (bit >> 6)) v |= 1ull << (bit & 63);
        out[x] = v;
    }
}

// chosen[(k r + e)(p+1) + p] += ybar[e] - xbar^T chosen[(k r + e)(p+1) + 0..p-1]:
// one warp per (k, e), lanes strided over i, tree sum.
__global__ void k_intercept_original(double* __restrict__ chosen, int64_t count, int64_t r, int64_t p,
                                     const double* __restrict__ xbar, const double* __restrict__ ybar)
{
    const int64_t col = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (col >= count) return;
    double* b = chosen + col * (p + 1);
    double acc = 0.0;
    for (int64_t i = lane; i < p; i += 32) acc += xbar[i] * b[i];
    acc = warp_sum(acc);
    if (lane == 0) b[p] += ybar[col % r] - acc;
}

// A[(j-1) p p + e p + c] = beta[e * pe + (j-1) p + c]; mu[e] = beta[e * pe + d p] or 0.
__global__ void k_partition_var(const double* __restrict__ beta, int64_t p, int d, int icpt,
                                double* __restrict__ A, double* __restrict__ mu)
{
    const int64_t pe = (int64_t)d * p + icpt;
    const int64_t total = (int64_t)d * p * p;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total + p;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (x < total) {
            const int64_t j = x / (p * p), e = (x / p) % p, c = x % p;
            A[x] = beta[e * pe + j * p + c];
        } else if (mu) {
            const int64_t e = x - total;
            mu[e] = icpt ? beta[e * pe + (int64_t)d * p] : 0.0;
        }
    }
}

int grid_for(int64_t n, int threads)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), 152 * 16));
}

void column_means(const double* A, int64_t lda, int64_t m, int64_t c, double* mean, cudaStream_t s)
{
    const int64_t rows = std::max<int64_t>(256, ceil_div(m, 65535));   // partial sums per chunk
    const int64_t chunks = ceil_div(m, rows);
    DevBuf part(sizeof(double) * (size_t)(chunks * c), s);
    k_col_partial<<<dim3((unsigned)ceil_div(c, 128), (unsigned)chunks), 128, 0, s>>>(A, lda, m, c, rows,
                                                                                 part.as<double>());
    UOI_CHECK_LAUNCH();
    k_col_finish<<<(unsigned)ceil_div(c, 128), 128, 0, s>>>(part.as<double>(), chunks, c, m, mean);
    UOI_CHECK_LAUNCH();
    count_launch(2);
}

dim3 rows_grid(int64_t m, int64_t cols, int threads)
{
    return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cols, threads), 64)),
                (unsigned)std::max<int64_t>(1, std::min<int64_t>(m, 65535)));
}

}  // namespace

void lagged_design(const double* S, int64_t N, int64_t p, int32_t d, double* X, int64_t ldx,
                   double* Y, int64_t ldy, cudaStream_t s)
{
    const int64_t m = N - d;
    if (m <= 0) return;
    k_lagged_design<<<rows_grid(m, (d + 1) * p, 256), 256, 0, s>>>(S, N, p, d, X, ldx, Y, ldy);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void center_with_ones(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p,
                      int64_t r, double* Xa, double* Ya, double* xbar, double* ybar, cudaStream_t s)
{
    column_means(X, ldx, m, p, xbar, s);
    column_means(Y, ldy, m, r, ybar, s);
    k_center_copy<<<rows_grid(m, p + 1, 256), 256, 0, s>>>(X, ldx, m, p, xbar, 1, Xa, p + 1);
    UOI_CHECK_LAUNCH();
    k_center_copy<<<rows_grid(m, r, 256), 256, 0, s>>>(Y, ldy, m, r, ybar, 0, Ya, r);
    UOI_CHECK_LAUNCH();
    count_launch(2);
}

void schur_intercept(const double* Ga, const double* Ba, const double* nk, int nk_count, int64_t p,
                     int64_t r, int32_t B, double* G, double* Bm, cudaStream_t s)
{
    const int64_t total = (p * p + p * r) * B;
    k_schur_intercept<<<grid_for(total, 256), 256, 0, s>>>(Ga, Ba, nk, nk_count, p, r, B, G, Bm);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void family_add_bit(const uint64_t* fam, int64_t count, int64_t W, int64_t Wa, int64_t bit,
                    uint64_t* out, cudaStream_t s)
{
    k_family_add_bit<<<grid_for(count * Wa, 256), 256, 0, s>>>(fam, count, W, Wa, bit, out);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void intercept_to_original(double* chosen, int64_t count, int64_t r, int64_t p, const double* xbar,
                           const double* ybar, cudaStream_t s)
{
    if (count <= 0) return;
    k_intercept_original<<<(unsigned)ceil_div(count, 8), 256, 0, s>>>(chosen, count, r, p, xbar, ybar);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void partition_var(const double* beta, int64_t p, int32_t d, int icpt, double* A, double* mu,
                   cudaStream_t s)
{
    const int64_t total = (int64_t)d * p * p + p;
    k_partition_var<<<grid_for(total, 256), 256, 0, s>>>(beta, p, d, icpt, A, mu);
    UOI_CHECK_LAUNCH();
    count_launch();
}

}  // namespace uoi
