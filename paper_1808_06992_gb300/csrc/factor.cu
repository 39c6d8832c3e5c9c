// factor.cu -- G3: batched FP64 Cholesky of A_k = G_k/n_k + rho I, inverse and RHS.
//
// The ADMM x-update of Eq. 5, x = (G/n_k + rho I)^{-1} (b/n_k + rho (z - u)),
// has a fixed matrix per bootstrap.  It is factored once (the paper's
// "triangular solve ... for matrix decomposition", Sec. IV-A-1) and turned
// into an explicit inverse M_k so that every iteration is one product
// x = c_k + rho M_k (z - u) with c_k = M_k b_k / n_k.  A_k is symmetric
// positive definite for rho > 0 and well conditioned, so the explicit
// inverse loses nothing measurable.
//
// Right-looking blocked Cholesky (panel factor, panel solve, trailing update),
// blocked triangular inverse and the product M = L^{-T} L^{-1}, all templated
// on the factor type T: FP64 in the plain form, FP32 in the mixed form (the
// FP32 ADMM state bounds that form's accuracy at the same level, and GB300's
// FP64 rate made the FP64 factor the largest single cost of a fit).
#include "kernels.h"
#include "tile.cuh"

namespace uoi {

namespace {

constexpr int NB = 32;    // Cholesky panel width
constexpr int IB = 64;    // inverse block

template <typename T>
__device__ __forceinline__ T system_entry(double g, double inv_n, double rho, bool diag);

template <>
__device__ __forceinline__ double system_entry<double>(double g, double inv_n, double rho, bool diag)
{
    return g * inv_n + (diag ? rho : 0.0);
}

// FP32 form: no FP64 arithmetic per element (this part's FP64 rate is ~1/64 of FP32).
template <>
__device__ __forceinline__ float system_entry<float>(double g, double inv_n, double rho, bool diag)
{
    return f64_to_f32_int(g) * (float)inv_n + (diag ? (float)rho : 0.f);
}

// One row per block-row step (no index division per element); the loads of four
// iterations are issued before their stores.
template <typename T>
__global__ void k_build_system(const double* __restrict__ G, const double* nk, double rho, int64_t p,
                               T* __restrict__ A)
{
    const int64_t k = blockIdx.y;
    const double inv_n = 1.0 / nk[k];
    for (int64_t i = blockIdx.x; i < p; i += gridDim.x) {
        const double* grow = G + (k * p + i) * p;
        T* arow = A + (k * p + i) * p;
#pragma unroll 4
        for (int64_t j = threadIdx.x; j < p; j += blockDim.x)
            arow[j] = system_entry<T>(__ldg(grow + j), inv_n, rho, i == j);
    }
}

// FP32 system from the lower triangle of G: 32 x 32 tiles through shared memory;
// each lower tile is written in place and, transposed, to its mirror (the
// diagonal tile's upper half from its lower half).  Block (32, 8), grid
// (tiles, tiles, B).
__global__ void k_build_system_lower(const double* __restrict__ G, const double* nk, double rho, int64_t p,
                                     float* __restrict__ A)
{
    // blockIdx.x enumerates the lower 32 x 32 tiles (by, bx), bx <= by, in groups of
    // LOWER_TILES consecutive tiles of one row of tiles; every thread issues its
    // loads for all of them before any store
    constexpr int LOWER_TILES = 4;
    __shared__ float tile[LOWER_TILES][32][33];
    const int64_t k = blockIdx.y;
    const int64_t tt = (p + 31) / 32;
    // row of tiles by holds ceil((by + 1) / LOWER_TILES) groups; find (by, first bx)
    int64_t grp = blockIdx.x, by = 0;
    for (;; ++by) {
        const int64_t ng = (by + LOWER_TILES) / LOWER_TILES;      // ceil((by + 1) / LOWER_TILES)
        if (grp < ng) break;
        grp -= ng;
    }
    if (by >= tt) return;
    const int64_t bx0 = grp * LOWER_TILES;
    const float inv_n = (float)(1.0 / nk[k]);
    const double* g = G + k * p * p;
    float* a = A + k * p * p;
    const int tx = threadIdx.x;
    double v[LOWER_TILES][4];
#pragma unroll
    for (int q = 0; q < LOWER_TILES; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t r = by * 32 + threadIdx.y + 8 * u, c = (bx0 + q) * 32 + tx;
            v[q][u] = (bx0 + q <= by && r < p && c < p && c <= r) ? __ldg(g + r * p + c) : 0.0;
        }
#pragma unroll
    for (int q = 0; q < LOWER_TILES; ++q) {
        if (bx0 + q > by) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int yy = threadIdx.y + 8 * u;
            const int64_t r = by * 32 + yy, c = (bx0 + q) * 32 + tx;
            if (r < p && c < p && c <= r) {
                const float e = system_entry<float>(v[q][u], (double)inv_n, rho, r == c);
                tile[q][yy][tx] = e;
                a[r * p + c] = e;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < LOWER_TILES; ++q) {
        const int64_t bx = bx0 + q;
        if (bx > by) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {                    // mirror: rows bx*32 + yy, columns by*32 + tx
            const int yy = threadIdx.y + 8 * u;
            const int64_t r = bx * 32 + yy, c = by * 32 + tx;
            if (r < p && c < p && c > r) a[r * p + c] = tile[q][tx][yy];
        }
    }
}

// Factor the nb x nb diagonal block at j0 (one block per matrix).
template <typename T>
__global__ void k_chol_diag(T* A, int64_t p, int64_t j0, int nb, DevStatus* st)
{
    const int64_t k = blockIdx.x;
    T* a = A + k * p * p;
    __shared__ T D[NB][NB + 1];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        D[i][j] = a[(j0 + i) * p + j0 + j];
    }
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
        if (threadIdx.x == 0) {
            const T d = D[c][c];
            if (!(d > T(0))) { bad = 1; D[c][c] = T(1); } else D[c][c] = sqrt(d);
        }
        __syncthreads();
        const T lcc = D[c][c];
        for (int i = c + 1 + threadIdx.x; i < nb; i += blockDim.x) D[i][c] /= lcc;
        __syncthreads();
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, j = e % nb;
            if (j > c && i >= j) D[i][j] -= D[i][c] * D[j][c];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        a[(j0 + i) * p + j0 + j] = j <= i ? D[i][j] : T(0);
    }
    if (threadIdx.x == 0 && bad) dev_fail(st, UOI_ERR_NOT_PD, (int)k);
}

// Rows below the diagonal block: L[i, j0:j0+nb] = A[i, j0:j0+nb] L_dd^{-T}.
template <typename T>
__global__ void k_chol_panel(T* A, int64_t p, int64_t j0, int nb)
{
    const int64_t k = blockIdx.y;
    T* a = A + k * p * p;
    __shared__ T D[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        D[i][j] = a[(j0 + i) * p + j0 + j];
    }
    __syncthreads();
    const int64_t i = j0 + nb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= p) return;
    T x[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) x[c] = c < nb ? a[i * p + j0 + c] : T(0);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        if (c >= nb) break;
        T v = x[c];
#pragma unroll
        for (int s = 0; s < NB; ++s)
            if (s < c) v -= x[s] * D[c][s];
        x[c] = v / D[c][c];
    }
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (c < nb) a[i * p + j0 + c] = x[c];
}

// Trailing update of the lower triangle: A[i][j] -= sum_s L[i][j0+s] L[j][j0+s].
template <typename T>
__global__ void __launch_bounds__(256) k_chol_update(T* A, int64_t p, int64_t j0, int nb)
{
    const int64_t k = blockIdx.y;
    T* a = A + k * p * p;
    const int64_t base = j0 + nb;
    int64_t ti, tj;
    tri_index(blockIdx.x, ti, tj);
    const int64_t i0 = base + ti * 64, jj0 = base + tj * 64;
    T acc[4][4] = {};
    auto fa = [&](int il, int64_t s) {
        const int64_t i = i0 + il;
        return i < p ? a[i * p + j0 + s] : T(0);
    };
    auto fb = [&](int64_t s, int jl) {
        const int64_t j = jj0 + jl;
        return j < p ? a[j * p + j0 + s] : T(0);
    };
    tile64_acc<T, true, true>(acc, fa, fb, 0, nb);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ty + 16 * u;
        if (i >= p) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t j = jj0 + tx + 16 * v;
            if (j < p && j <= i) a[i * p + j] -= acc[u][v];
        }
    }
}

// Inverse of each IB x IB lower-triangular diagonal block, in T.  The block of
// L is read from global memory (L2); the inverse is built in shared memory.
template <typename T>
__global__ void k_trinv_diag(const T* L, int64_t p, T* Linv)
{
    const int64_t k = blockIdx.y;
    const int64_t b0 = (int64_t)blockIdx.x * IB;
    const int nb = (int)(p - b0 < IB ? p - b0 : IB);
    const T* l = L + k * p * p + b0 * p + b0;          // l[i * p + j] = L[b0+i][b0+j]
    T* li = Linv + k * p * p;
    __shared__ T R[IB][IB + 1];
    const int j = threadIdx.x;                    // one column of the inverse per thread
    if (j < nb) {
        for (int i = 0; i < nb; ++i) {
            T v;
            if (i < j) v = T(0);
            else if (i == j) v = T(1) / (T)l[j * p + j];
            else {
                T s = T(0);
                for (int t = j; t < i; ++t) s = fma((T)l[i * p + t], R[t][j], s);
                v = -s / (T)l[i * p + i];
            }
            R[i][j] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, c = e % nb;
        li[(b0 + i) * p + b0 + c] = R[i][c];
    }
}

// Block row I of L^{-1}: for J < I, Linv_IJ = -Linv_II * sum_{K=J}^{I-1} L_IK Linv_KJ.
template <typename T>
__global__ void __launch_bounds__(256) k_trinv_row(const T* L, int64_t p, int64_t I, T* Linv)
{
    const int64_t k = blockIdx.y;
    const int64_t J = blockIdx.x;
    const T* l = L + k * p * p;
    T* li = Linv + k * p * p;
    const int64_t i0 = I * IB, j0 = J * IB;
    T acc[4][4] = {};
    auto fa = [&](int il, int64_t s) {
        const int64_t i = i0 + il;
        return i < p ? (T)l[i * p + s] : T(0);
    };
    auto fb = [&](int64_t s, int jl) {
        const int64_t jj = j0 + jl;
        return (T)li[s * p + jj];
    };
    tile64_acc<T, true, false>(acc, fa, fb, j0, i0);   // T_IJ (64 x 64)
    __shared__ T Tm[IB][IB + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) Tm[ty + 16 * u][tx + 16 * v] = acc[u][v];
    __syncthreads();
    T acc2[4][4] = {};
    auto ga = [&](int il, int64_t s) {
        const int64_t i = i0 + il, c = i0 + s;
        return (i < p && c < p && c <= i) ? li[i * p + c] : T(0);
    };
    auto gb = [&](int64_t s, int jl) { return Tm[s][jl]; };
    tile64_acc<T, true, false>(acc2, ga, gb, 0, IB);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ty + 16 * u;
        if (i >= p) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t jj = j0 + tx + 16 * v;
            li[i * p + jj] = -acc2[u][v];
        }
    }
}

// M = L^{-T} L^{-1}: M[i][j] = sum_{s >= max(i,j)} Linv[s][i] Linv[s][j], lower tiles + mirror.
template <typename T>
__global__ void __launch_bounds__(256) k_inverse_product(const T* Linv, int64_t p, T* M)
{
    const int64_t k = blockIdx.y;
    const T* li = Linv + k * p * p;
    T* mk = M + k * p * p;
    int64_t ti, tj;
    tri_index(blockIdx.x, ti, tj);
    const int64_t i0 = ti * 64, j0 = tj * 64;
    T acc[4][4] = {};
    auto fa = [&](int il, int64_t s) {
        const int64_t i = i0 + il;
        return i < p ? li[s * p + i] : T(0);
    };
    auto fb = [&](int64_t s, int jl) {
        const int64_t j = j0 + jl;
        return j < p ? li[s * p + j] : T(0);
    };
    tile64_acc<T>(acc, fa, fb, i0, p);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ty + 16 * u;
        if (i >= p) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t j = j0 + tx + 16 * v;
            if (j >= p || j > i) continue;
            mk[i * p + j] = acc[u][v];
            mk[j * p + i] = acc[u][v];
        }
    }
}

// c[k][e][i] = sum_j M[k][i][j] * (Bm[k][j][e] / nk[k]).
template <typename T>
__global__ void __launch_bounds__(256) k_rhs(const T* M, const double* Bm, const double* nk,
                                             int64_t p, int64_t r, T* c)
{
    const int64_t k = blockIdx.y;
    const int64_t tiles_e = (r + 63) / 64;
    const int64_t i0 = (blockIdx.x / tiles_e) * 64, e0 = (blockIdx.x % tiles_e) * 64;
    const T* mk = M + k * p * p;
    const double* bk = Bm + k * p * r;
    const double n_k = nk[k];
    T acc[4][4] = {};
    auto fa = [&](int il, int64_t j) {
        const int64_t i = i0 + il;
        return i < p ? mk[i * p + j] : T(0);
    };
    auto fb = [&](int64_t j, int el) {
        const int64_t e = e0 + el;
        return e < r ? (T)(bk[j * r + e] / n_k) : T(0);
    };
    tile64_acc<T, true, false>(acc, fa, fb, 0, p);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ty + 16 * u;
        if (i >= p) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t e = e0 + tx + 16 * v;
            if (e < r) c[(k * r + e) * p + i] = acc[u][v];
        }
    }
}

// b_k[j][e] / nk[k] in T, once per system (keeps FP64 division off the GEMV).
template <typename T>
__global__ void k_scale_rhs(const double* Bm, const double* nk, int64_t pr, int32_t B, T* out)
{
    const int64_t total = (int64_t)B * pr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (T)(Bm[t] / nk[t / pr]);
}

// c[k][e][i] = sum_j M[k][i][j] bs[k][j][e] for few responses: one warp per row
// (M streamed once, coalesced).
template <typename T, int R>
__global__ void __launch_bounds__(256) k_rhs_gemv(const T* M, const T* bs, int64_t p, T* c)
{
    const int64_t k = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= p) return;
    const T* row = M + (k * p + i) * p;
    const T* b = bs + k * p * R;
    T acc[R];
#pragma unroll
    for (int e = 0; e < R; ++e) acc[e] = T(0);
    for (int64_t j = lane; j < p; j += 32) {
        const T mv = row[j];
#pragma unroll
        for (int e = 0; e < R; ++e) acc[e] += mv * b[j * R + e];
    }
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const T v = warp_sum(acc[e]);
        if (lane == 0) c[(k * R + e) * p + i] = v;
    }
}

}  // namespace

template <typename T>
void build_system(const double* G, const double* nk, double rho, int64_t p, int32_t B, T* A,
                  cudaStream_t s)
{
    dim3 gb((unsigned)std::min<int64_t>(p, 1024), (unsigned)B);
    k_build_system<T><<<gb, 256, 0, s>>>(G, nk, rho, p, A);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void build_system_lower(const double* G, const double* nk, double rho, int64_t p, int32_t B, float* A,
                        cudaStream_t s)
{
    const int64_t tt = ceil_div(p, 32);
    int64_t groups = 0;                                  // groups of 4 lower tiles per row of tiles
    for (int64_t by = 0; by < tt; ++by) groups += (by + 4) / 4;
    k_build_system_lower<<<dim3((unsigned)groups, (unsigned)B), dim3(32, 8), 0, s>>>(G, nk, rho, p, A);
    UOI_CHECK_LAUNCH();
    count_launch();
}

template <typename T>
void cholesky_inplace(T* A, int64_t p, int32_t B, DevStatus* status, cudaStream_t s)
{
    for (int64_t j0 = 0; j0 < p; j0 += NB) {
        const int nb = (int)std::min<int64_t>(NB, p - j0);
        k_chol_diag<T><<<B, 256, 0, s>>>(A, p, j0, nb, status);
        UOI_CHECK_LAUNCH();
        count_launch();
        const int64_t rest = p - j0 - nb;
        if (rest <= 0) break;
        dim3 gp((unsigned)ceil_div(rest, 128), (unsigned)B);
        k_chol_panel<T><<<gp, 128, 0, s>>>(A, p, j0, nb);
        UOI_CHECK_LAUNCH();
        const int64_t tt = ceil_div(rest, 64);
        dim3 gu((unsigned)(tt * (tt + 1) / 2), (unsigned)B);
        k_chol_update<T><<<gu, 256, 0, s>>>(A, p, j0, nb);
        UOI_CHECK_LAUNCH();
        count_launch(2);
    }
}

template <typename T>
void build_and_factor(const double* G, const double* nk, double rho, int64_t p, int32_t B,
                      T* A, DevStatus* status, cudaStream_t s)
{
    build_system<T>(G, nk, rho, p, B, A, s);
    cholesky_inplace<T>(A, p, B, status, s);
}

template void build_system<float>(const double*, const double*, double, int64_t, int32_t, float*,
                                  cudaStream_t);
template void cholesky_inplace<float>(float*, int64_t, int32_t, DevStatus*, cudaStream_t);
template void build_and_factor<double>(const double*, const double*, double, int64_t, int32_t,
                                       double*, DevStatus*, cudaStream_t);
template void build_and_factor<float>(const double*, const double*, double, int64_t, int32_t,
                                      float*, DevStatus*, cudaStream_t);

template <typename T>
void spd_inverse_from_factor(const T* L, int64_t p, int32_t B, T* Linv, T* M, cudaStream_t s)
{
    UOI_CUDA(cudaMemsetAsync(Linv, 0, sizeof(T) * (size_t)(p * p * B), s));
    const int64_t nbk = ceil_div(p, IB);
    k_trinv_diag<T><<<dim3((unsigned)nbk, (unsigned)B), IB, 0, s>>>(L, p, Linv);
    UOI_CHECK_LAUNCH();
    count_launch();
    for (int64_t I = 1; I < nbk; ++I) {
        k_trinv_row<T><<<dim3((unsigned)I, (unsigned)B), 256, 0, s>>>(L, p, I, Linv);
        UOI_CHECK_LAUNCH();
        count_launch();
    }
    const int64_t tt = ceil_div(p, 64);
    k_inverse_product<T><<<dim3((unsigned)(tt * (tt + 1) / 2), (unsigned)B), 256, 0, s>>>(Linv, p, M);
    UOI_CHECK_LAUNCH();
    count_launch();
}

template <typename T>
void rhs_from_inverse(const T* M, const double* Bm, const double* nk, int64_t p, int64_t r, int32_t B,
                      T* c, cudaStream_t s, T* rhs_scratch)
{
    if (r == 1) {
        // b_k / n_k in T, from the caller's scratch when given (else a pool buffer)
        DevBuf bs;
        T* bsc = rhs_scratch;
        if (!bsc) {
            bs.alloc(sizeof(T) * (size_t)(B * p), s);
            bsc = bs.as<T>();
        }
        k_scale_rhs<T><<<(unsigned)std::min<int64_t>(ceil_div(B * p, 256), 4096), 256, 0, s>>>(
            Bm, nk, p, B, bsc);
        UOI_CHECK_LAUNCH();
        k_rhs_gemv<T, 1><<<dim3((unsigned)ceil_div(p, 8), (unsigned)B), 256, 0, s>>>(M, bsc, p, c);
        UOI_CHECK_LAUNCH();
        count_launch(2);
        return;
    }
    const int64_t tt = ceil_div(p, 64), te = ceil_div(r, 64);
    k_rhs<T><<<dim3((unsigned)(tt * te), (unsigned)B), 256, 0, s>>>(M, Bm, nk, p, r, c);
    UOI_CHECK_LAUNCH();
    count_launch();
}

template <typename T>
void inverse_and_rhs(const T* L, const double* Bm, const double* nk, int64_t p, int64_t r,
                     int32_t B, T* Linv, T* M, T* c, cudaStream_t s, T* rhs_scratch)
{
    spd_inverse_from_factor<T>(L, p, B, Linv, M, s);
    rhs_from_inverse<T>(M, Bm, nk, p, r, B, c, s, rhs_scratch);
}

template void spd_inverse_from_factor<float>(const float*, int64_t, int32_t, float*, float*,
                                             cudaStream_t);
template void rhs_from_inverse<float>(const float*, const double*, const double*, int64_t, int64_t,
                                      int32_t, float*, cudaStream_t, float*);
template void inverse_and_rhs<double>(const double*, const double*, const double*, int64_t,
                                      int64_t, int32_t, double*, double*, double*, cudaStream_t, double*);
template void inverse_and_rhs<float>(const float*, const double*, const double*, int64_t,
                                     int64_t, int32_t, float*, float*, float*, cudaStream_t, float*);

}  // namespace uoi
