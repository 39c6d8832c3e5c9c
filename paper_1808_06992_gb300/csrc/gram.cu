// gram.cu -- G1 in FP64 on CUDA cores: weighted Gram and moments, lambda grid.
//
// For bootstrap k the LASSO of Eq. 2 on T^k only needs G_k = X^T W_k X and
// B_k = X^T W_k Y (W_k = diag of the bootstrap multiplicities): the ADMM
// x-update of Eq. 5 then never touches the n rows again.  This is the plain
// FP64 form; the tensor-core form lives in gram_tc.cu.
#include <algorithm>

#include "kernels.h"

namespace uoi {

namespace {

constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // rows per K step

// Output column j of C = X^T W [X | Y]: j < p -> X[:, j], else Y[:, j - p].
__device__ __forceinline__ double zcol(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                                       int64_t t, int64_t j, int64_t p)
{
    return j < p ? X[t * ldx + j] : Y[t * ldy + (j - p)];
}

// grid: (tiles, B).  Tile list: lower-triangular tiles of G (tj <= ti) and every
// tile of the B block; b_only restricts to the B block.  256 threads, 4x4 each.
__global__ void __launch_bounds__(256)
k_moments_fp64(const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y,
               int64_t ldy, int64_t m, int64_t p, int64_t r, const uint32_t* __restrict__ w,
               const uint8_t* __restrict__ mask, double* __restrict__ G, double* __restrict__ Bm,
               int b_only)
{
    const int64_t k = blockIdx.y;
    const int64_t tp = (p + GT - 1) / GT;          // row tiles (i over features)
    const int64_t tb = (r + GT - 1) / GT;          // column tiles of the B block
    int64_t t = blockIdx.x;
    int64_t ti, j0, jend;
    bool gpart;
    const int64_t ng = b_only ? 0 : tp * (tp + 1) / 2;
    if (t < ng) {                                   // triangular index -> (ti, tj)
        ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while (ti * (ti + 1) / 2 > t) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        const int64_t tj = t - ti * (ti + 1) / 2;
        j0 = tj * GT;
        jend = p;
        gpart = true;
    } else {
        t -= ng;
        ti = t / tb;
        j0 = p + (t % tb) * GT;
        jend = p + r;
        gpart = false;
    }
    const int64_t i0 = ti * GT;
    const uint32_t* wk = w ? w + k * m : nullptr;
    const uint8_t* mk = mask ? mask + k * m : nullptr;

    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int64_t t0 = 0; t0 < m; t0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            const int rr = e / GT, cc = e % GT;
            const int64_t row = t0 + rr;
            double wt = 0.0, a = 0.0, b = 0.0;
            if (row < m) {
                wt = wk ? (double)wk[row] : (mk ? (double)mk[row] : 1.0);
                if (i0 + cc < p) a = X[row * ldx + i0 + cc];
                if (j0 + cc < jend) b = zcol(X, ldx, Y, ldy, row, j0 + cc, p);
            }
            As[rr][cc] = wt * a;
            Bs[rr][cc] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty + 16 * u]; b[u] = Bs[kk][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ty + 16 * u;
        if (i >= p) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t j = j0 + tx + 16 * v;
            if (j >= jend) continue;
            if (gpart && j > i) continue;    // lower triangle; the mirror fills the rest
            if (gpart) {
                G[k * p * p + i * p + j] = acc[u][v];
                if (i != j) G[k * p * p + j * p + i] = acc[u][v];   // mirror (j < i tiles only)
            } else {
                Bm[k * p * r + i * r + (j - p)] = acc[u][v];
            }
        }
    }
}

__global__ void k_masked_sumsq(const double* Y, int64_t ldy, int64_t m, int64_t r,
                               const uint8_t* mask, double* yy)
{
    const int64_t k = blockIdx.y;
    const int64_t e = blockIdx.x;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x)
        if (mask[k * m + t]) { const double v = Y[t * ldy + e]; s = fma(v, v, s); }
    s = warp_sum(s);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += part[i];
        yy[k * r + e] = tot;
    }
}

// lambda_max = max |X^T Y| / m, lambda_j = lmax * ratio^(j/(q-1)) (descending).
__global__ void k_lambda_grid(const double* XtY, int64_t count, int64_t m, int32_t q,
                              double ratio, double* lambdas)
{
    double best = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) best = fmax(best, fabs(XtY[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b = fmax(b, part[i]);
        part[0] = b / (double)m;
    }
    __syncthreads();
    const double lmax = part[0];
    for (int j = threadIdx.x; j < q; j += blockDim.x)
        lambdas[j] = q > 1 ? lmax * pow(ratio, (double)j / (double)(q - 1)) : lmax;
}

// Exponent field all ones = Inf or NaN.  Contiguous rows (ldx == cols): one flat
// loop; otherwise rows over blocks and columns over threads.  No division per
// element; one flag write per warp that saw a non-finite value.
__global__ void k_check_finite(const double* __restrict__ X, int64_t ldx, int64_t m, int64_t cols,
                               int32_t* flag)
{
    bool bad = false;
    if (ldx == cols) {
        const int64_t total = m * cols;
#pragma unroll 4
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
             t += (int64_t)gridDim.x * blockDim.x)
            bad |= ((__double_as_longlong(__ldg(X + t)) >> 52) & 0x7FF) == 0x7FF;
    } else {
        for (int64_t row = blockIdx.x; row < m; row += gridDim.x) {
            const double* xr = X + row * ldx;
#pragma unroll 4
            for (int64_t j = threadIdx.x; j < cols; j += blockDim.x)
                bad |= ((__double_as_longlong(__ldg(xr + j)) >> 52) & 0x7FF) == 0x7FF;
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

// Split-K X^T Y for r <= 4: block (column tile, row chunk) writes partial sums.
constexpr int XTY_ROWS = 128;      // short row chunks: many blocks in flight
__global__ void k_xty_partial(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                              int64_t m, int64_t p, int64_t r, double* part)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t c = blockIdx.y;
    const int64_t t0 = c * XTY_ROWS, t1 = min(m, t0 + XTY_ROWS);
    double acc[4] = { 0.0, 0.0, 0.0, 0.0 };
    if (j < p) {
        // batches of 16 rows: all sixteen loads of X and of y issued before the
        // multiply-adds
        int64_t t = t0;
        for (; t + 16 <= t1; t += 16) {
            double xv[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) xv[u] = __ldg(X + (t + u) * ldx + j);
            if (r == 1) {
                double yv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) yv[u] = __ldg(Y + (t + u) * ldy);
#pragma unroll
                for (int u = 0; u < 16; ++u) acc[0] = fma(xv[u], yv[u], acc[0]);
            } else {
#pragma unroll
                for (int u = 0; u < 16; ++u)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (e < r) acc[e] = fma(xv[u], __ldg(Y + (t + u) * ldy + e), acc[e]);
            }
        }
        for (; t < t1; ++t) {
            const double x = X[t * ldx + j];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e < r) acc[e] = fma(x, Y[t * ldy + e], acc[e]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < r) part[(c * p + j) * r + e] = acc[e];
    }
}

__global__ void k_xty_reduce(const double* part, int64_t chunks, int64_t count, double* out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t c = 0; c < chunks; ++c) s += part[c * count + i];
        out[i] = s;
    }
}

}  // namespace

void xty_small(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p,
               int64_t r, double* XtY, cudaStream_t s)
{
    const int64_t chunks = ceil_div(m, XTY_ROWS);
    DevBuf part(sizeof(double) * (size_t)(chunks * p * r), s);
    dim3 g((unsigned)ceil_div(p, 128), (unsigned)chunks);
    k_xty_partial<<<g, 128, 0, s>>>(X, ldx, Y, ldy, m, p, r, part.as<double>());
    UOI_CHECK_LAUNCH();
    k_xty_reduce<<<(unsigned)std::min<int64_t>(ceil_div(p * r, 256), 1024), 256, 0, s>>>(
        part.as<double>(), chunks, p * r, XtY);
    UOI_CHECK_LAUNCH();
    count_launch(2);
}

void moments_fp64(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m,
                  int64_t p, int64_t r, const uint32_t* w, const uint8_t* mask, int32_t B,
                  double* G, double* Bm, int b_only, cudaStream_t s)
{
    const int64_t tp = (p + GT - 1) / GT, tb = (r + GT - 1) / GT;
    const int64_t tiles = (b_only ? 0 : tp * (tp + 1) / 2) + tp * tb;
    dim3 grid((unsigned)tiles, (unsigned)B);
    k_moments_fp64<<<grid, 256, 0, s>>>(X, ldx, Y, ldy, m, p, r, w, mask, G, Bm, b_only);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void masked_sumsq(const double* Y, int64_t ldy, int64_t m, int64_t r, const uint8_t* mask,
                  int32_t B, double* yy, cudaStream_t s)
{
    dim3 grid((unsigned)r, (unsigned)B);
    k_masked_sumsq<<<grid, 256, 0, s>>>(Y, ldy, m, r, mask, yy);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void lambda_grid(const double* XtY, int64_t count, int64_t m, int32_t q, double ratio,
                 double* lambdas, cudaStream_t s)
{
    k_lambda_grid<<<1, 1024, 0, s>>>(XtY, count, m, q, ratio, lambdas);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void check_finite(const double* X, int64_t ldx, int64_t m, int64_t cols, int32_t* flag,
                  cudaStream_t s)
{
    int64_t g = (m * cols + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    k_check_finite<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(X, ldx, m, cols, flag);
    UOI_CHECK_LAUNCH();
    count_launch();
}

namespace {
__global__ void k_gather_cols_f64(const double* X, int64_t ldx, int64_t m, const int32_t* cols, int64_t nu,
                                  double* out)
{
    const int64_t total = m * nu;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        out[t] = X[(t / nu) * ldx + cols[t % nu]];
}

// G[k][cols[a]][cols[b]] = Gu[k][a][b], Bm[k][cols[a]][e] = Bu[k][a][e].
__global__ void k_scatter_moments(const double* Gu, const double* Bu, int64_t nu, int64_t r, int32_t B,
                                  const int32_t* cols, int64_t p_out, double* G, double* Bm)
{
    const int64_t per = nu * nu + nu * r, total = per * B;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / per, o = t % per;
        if (o < nu * nu) {
            const int64_t a = o / nu, b = o % nu;
            G[(k * p_out + cols[a]) * p_out + cols[b]] = Gu[k * nu * nu + o];
        } else {
            const int64_t q = o - nu * nu, a = q / r, e = q % r;
            Bm[(k * p_out + cols[a]) * r + e] = Bu[k * nu * r + q];
        }
    }
}
}  // namespace

void moments_fp64_cols(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p_out,
                       int64_t r, int64_t nu, const int32_t* cols, const uint32_t* w, const uint8_t* mask,
                       int32_t B, double* G, double* Bm, cudaStream_t s)
{
    if (nu <= 0) return;
    DevBuf Xu(sizeof(double) * (size_t)(m * nu), s);
    k_gather_cols_f64<<<(unsigned)std::min<int64_t>(ceil_div(m * nu, 256), 152 * 32), 256, 0, s>>>(
        X, ldx, m, cols, nu, Xu.as<double>());
    UOI_CHECK_LAUNCH();
    DevBuf Gu(sizeof(double) * (size_t)(B * nu * nu), s), Bu(sizeof(double) * (size_t)(B * nu * r), s);
    moments_fp64(Xu.as<double>(), nu, Y, ldy, m, nu, r, w, mask, B, Gu.as<double>(), Bu.as<double>(), 0, s);
    const int64_t total = (nu * nu + nu * r) * B;
    k_scatter_moments<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 32), 256, 0, s>>>(
        Gu.as<double>(), Bu.as<double>(), nu, r, B, cols, p_out, G, Bm);
    UOI_CHECK_LAUNCH();
    count_launch(2);
}

}  // namespace uoi
