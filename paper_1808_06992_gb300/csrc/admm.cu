// admm.cu -- G4: batched LASSO-ADMM (Sec. II-E, Eq. 5) over bootstraps x equations x lambdas.
//
// Scaled-form ADMM for (1/(2 n_k)) ||y - X b||^2_{W_k} + lambda ||b||_1 with the
// factor cached as M_k = (G_k/n_k + rho I)^{-1} and c_k = M_k b_k / n_k:
//   x = c_k + rho M_k (z - u)            x-minimisation (a multi-RHS product)
//   v = x + u,  z = S_{lambda/rho}(v)    z-minimisation (soft threshold)
//   u = v - z                            dual update
//   stop when ||x - z|| <= sqrt(p) abs + rel max(||x||, ||z||)
//        and rho ||z - z_prev|| <= sqrt(p) abs + rel rho ||u||, or at max_iter.
// A "chain" is one (bootstrap g, equation e) path over lambda_0 > lambda_1 > ...
// (warm = path: column j starts from column j-1's (z, u)) or one single
// (g, e, j) column (warm = none: z = u = 0).
//
// Two schedules:
//  * resident (p <= 128 in FP64, p <= 192 in FP32): one CTA keeps M_g in shared
//    memory; each warp runs its own chains to completion with no block-wide
//    barrier (the warp only reads its own columns of V = z - u), pulling new
//    chains from a per-group counter.  One launch solves everything.
//  * streaming (larger p): one launch per iteration computes x for every active
//    chain (row tiles x chain tiles x groups) with the soft-threshold / dual
//    update / partial norms fused into the epilogue; a second launch reduces the
//    norms in a fixed order, finishes converged columns and compacts the active
//    list.  The host checks the active count every few iterations.
#include <algorithm>
#include <vector>

#include "kernels.h"

namespace uoi {

namespace {

template <typename T>
struct AdmmDev {
    int32_t G, q, max_iter, warm;
    int32_t p, r, W;
    const T* M;
    const T* c;
    const double* lambdas;
    T rho, abs_tol, rel_tol, sqrtp;
    double* beta;
    int32_t* iters;
    uint8_t* conv;
    uint64_t* family;
    double* u_out;       // final scaled dual per column (nullable)
    const float* z0;     // initial state per column, cold schedule only (nullable)
    const float* u0;
    unsigned long long* near_count;   // near-threshold features (nullable)
};

template <typename T>
__device__ __forceinline__ void and_family_bits(const AdmmDev<T>& P, int64_t col_je, int a,
                                                unsigned ballot)
{
    // rows 32a .. 32a+31 form half of 64-bit word a/2
    const int shift = (a & 1) * 32;
    const uint64_t mask = ((uint64_t)ballot << shift) | ~(0xFFFFFFFFull << shift);
    atomicAnd((unsigned long long*)&P.family[col_je * P.W + (a >> 1)], (unsigned long long)mask);
}

// ----------------------------------------------------------------------------
// Resident schedule
// ----------------------------------------------------------------------------
template <typename T, int A, int SW>
__global__ void __launch_bounds__(256, 1) k_admm_resident(AdmmDev<T> P, int32_t* chain_next)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LD = A * 32;
    const int p = P.p;
    const int p4 = (p + 3) & ~3;
    T* Ms = reinterpret_cast<T*>(smem_raw);                  // p4 x LD, zero padded
    T* Vs = Ms + (size_t)p4 * LD;                             // 8 warps x SW x LD
    const int g = blockIdx.y;
    const T* Mg = P.M + (size_t)g * p * p;
    for (int idx = threadIdx.x; idx < p4 * LD; idx += blockDim.x) {
        const int row = idx / LD, col = idx % LD;
        Ms[idx] = (row < p && col < p) ? Mg[(size_t)row * p + col] : T(0);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* Vw = Vs + (size_t)warp * SW * LD;
    const int nchains = P.warm ? P.r : P.r * P.q;

    int e_[SW], j_[SW], jend_[SW], it_[SW];
    bool act[SW];
    T kappa[SW];
    T z[A][SW], u[A][SW];

    auto fetch = [&](int b) {
        int cid = 0;
        if (lane == 0) cid = atomicAdd(&chain_next[g], 1);
        cid = __shfl_sync(0xffffffffu, cid, 0);
        act[b] = cid < nchains;
        if (!act[b]) return;
        if (P.warm) { e_[b] = cid; j_[b] = 0; jend_[b] = P.q; }
        else        { e_[b] = cid % P.r; j_[b] = cid / P.r; jend_[b] = j_[b] + 1; }
        it_[b] = 0;
        kappa[b] = (T)P.lambdas[j_[b]] / P.rho;
        const int64_t col0 = ((int64_t)g * P.q + j_[b]) * P.r + e_[b];
#pragma unroll
        for (int a = 0; a < A; ++a) {
            const int i = lane + 32 * a;
            const bool init = P.z0 && !P.warm && i < p;
            z[a][b] = init ? (T)P.z0[col0 * p + i] : T(0);
            u[a][b] = init ? (T)P.u0[col0 * p + i] : T(0);
        }
    };
#pragma unroll
    for (int b = 0; b < SW; ++b) fetch(b);

    for (;;) {
        bool any = false;
#pragma unroll
        for (int b = 0; b < SW; ++b) any |= act[b];
        if (!any) break;
#pragma unroll
        for (int b = 0; b < SW; ++b)
#pragma unroll
            for (int a = 0; a < A; ++a) {
                const int i = lane + 32 * a;
                Vw[b * LD + i] = (act[b] && i < p) ? z[a][b] - u[a][b] : T(0);
            }
        __syncwarp();
        T acc[A][SW];
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
            for (int b = 0; b < SW; ++b) acc[a][b] = T(0);
        for (int k = 0; k < p4; k += 4) {
            T v[SW][4];
#pragma unroll
            for (int b = 0; b < SW; ++b)
#pragma unroll
                for (int t = 0; t < 4; ++t) v[b][t] = Vw[b * LD + k + t];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                T mrow[A];
#pragma unroll
                for (int a = 0; a < A; ++a) mrow[a] = Ms[(size_t)(k + t) * LD + lane + 32 * a];
#pragma unroll
                for (int a = 0; a < A; ++a)
#pragma unroll
                    for (int b = 0; b < SW; ++b) acc[a][b] = fma(mrow[a], v[b][t], acc[a][b]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < SW; ++b) {
            if (!act[b]) continue;
            const T* cg = P.c + ((size_t)g * P.r + e_[b]) * p;
            T r2 = 0, s2 = 0, x2 = 0, z2 = 0, u2 = 0;
#pragma unroll
            for (int a = 0; a < A; ++a) {
                const int i = lane + 32 * a;
                if (i < p) {
                    const T x = cg[i] + P.rho * acc[a][b];
                    const T zp = z[a][b];
                    const T v = x + u[a][b];
                    const T zn = soft_threshold(v, kappa[b]);
                    const T un = v - zn;
                    z[a][b] = zn;
                    u[a][b] = un;
                    const T d = x - zn, dz = zn - zp;
                    r2 += d * d; s2 += dz * dz; x2 += x * x; z2 += zn * zn; u2 += un * un;
                }
            }
            r2 = warp_sum(r2); s2 = warp_sum(s2); x2 = warp_sum(x2);
            z2 = warp_sum(z2); u2 = warp_sum(u2);
            it_[b] += 1;
            const T xn = sqrt(x2), zn = sqrt(z2);
            const T eps_pri = P.sqrtp * P.abs_tol + P.rel_tol * (xn > zn ? xn : zn);
            const T eps_dual = P.sqrtp * P.abs_tol + P.rel_tol * P.rho * sqrt(u2);
            const bool converged = sqrt(r2) <= eps_pri && P.rho * sqrt(s2) <= eps_dual;
            if (converged || it_[b] >= P.max_iter) {
                const int64_t col_je = (int64_t)j_[b] * P.r + e_[b];
                const int64_t col = (int64_t)g * P.q * P.r + col_je;
                if (P.beta) {
#pragma unroll
                    for (int a = 0; a < A; ++a) {
                        const int i = lane + 32 * a;
                        if (i < p && UOI_IN_BOUNDS(col * p + i, (int64_t)P.G * P.q * P.r * p, 201))
                            P.beta[col * p + i] = (double)z[a][b];
                    }
                }
                if (P.u_out) {
#pragma unroll
                    for (int a = 0; a < A; ++a) {
                        const int i = lane + 32 * a;
                        if (i < p) P.u_out[col * p + i] = (double)u[a][b];
                    }
                }
                if (P.family) {
#pragma unroll
                    for (int a = 0; a < A; ++a) {
                        const int i = lane + 32 * a;
                        const unsigned bal = __ballot_sync(0xffffffffu, i < p && z[a][b] != T(0));
                        if (lane == 0 && 32 * a < p) and_family_bits(P, col_je, a, bal);
                    }
                }
                if (P.near_count) {
#pragma unroll
                    for (int a = 0; a < A; ++a)
                        count_near_threshold<T>(lane + 32 * a < p, z[a][b], u[a][b], kappa[b],
                                                (T)kNearThreshold, P.near_count);
                }
                if (lane == 0) {
                    if (P.iters) P.iters[col] = it_[b];
                    if (P.conv) P.conv[col] = converged ? 1 : 0;
                }
                j_[b] += 1;
                if (j_[b] < jend_[b]) {
                    it_[b] = 0;
                    kappa[b] = (T)P.lambdas[j_[b]] / P.rho;
                } else {
                    fetch(b);
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Streaming schedule
// ----------------------------------------------------------------------------
struct StreamState {
    int32_t* slot_j;      // current lambda index per slot
    int32_t* slot_jend;
    int32_t* slot_it;
    int32_t* act[2];      // G x nchains active lists (double-buffered)
    int32_t* cnt[2];      // G counts
    int32_t* total[2];    // total active count
    int32_t nchains;
};

constexpr int GV_ROWS = 8;  // rows per GEMV block (one warp per row)

template <typename T>
__device__ __forceinline__ void slot_coords(const AdmmDev<T>& P, int32_t nchains, int32_t s,
                                            int& g, int& e)
{
    g = s / nchains;
    const int cid = s % nchains;
    e = P.warm ? cid : cid % P.r;
}

// Epilogue for one (row i, slot s) element; returns the five partial sums.
template <typename T>
__device__ __forceinline__ void admm_elem(const AdmmDev<T>& P, T acc, int g, int e, int64_t s,
                                          int i, T kappa, T* z, T* u, T* Vn, T (&part)[5])
{
    const int p = P.p;
    const T x = P.c[((size_t)g * P.r + e) * p + i] + P.rho * acc;
    const size_t o = (size_t)s * p + i;
    const T zp = z[o];
    const T v = x + u[o];
    const T zn = soft_threshold(v, kappa);
    const T un = v - zn;
    z[o] = zn;
    u[o] = un;
    Vn[o] = zn - un;
    const T d = x - zn, dz = zn - zp;
    part[0] += d * d; part[1] += dz * dz; part[2] += x * x; part[3] += zn * zn; part[4] += un * un;
}

// x-update tile: 128 rows x 64 chains, 256 threads with an 8 x 4 register block
// each (rows 8*ty .. +7, chains 4*tx .. +3).  M is symmetric, so the tile's
// column k (rows i0 .. i0+127) is the contiguous segment M[k][i0 .. i0+127]:
// it is copied row by row with coalesced loads and conflict-free stores.  The
// next K step is prefetched into registers while the current one is consumed
// (two shared-memory buffers).  The soft threshold, dual update and partial
// norms run in the epilogue; V = z - u of the next iteration goes to the other
// V buffer.
constexpr int SG_TM = 128;
constexpr int SG_TN = 64;

template <typename T>
__global__ void __launch_bounds__(256)
k_stream_gemm(AdmmDev<T> P, StreamState S, int cur, const T* __restrict__ Vc, T* Vn, T* z, T* u,
              T* norms, int RT)
{
    constexpr int TK = sizeof(T) == 8 ? 8 : 16;              // K per stage
    constexpr int LDB = SG_TN + 4;
    constexpr int A_PER = SG_TM * TK / 256;                  // M elements per thread per stage
    constexpr int B_PER = SG_TN * TK / 256;                  // V elements per thread per stage
    const int g = blockIdx.z;
    const int rt = blockIdx.x;
    const int i0 = rt * SG_TM;
    const int s0 = blockIdx.y * SG_TN;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x < 32) {
        for (int t = threadIdx.x; t < P.G; t += 32) S.cnt[cur ^ 1][t] = 0;
        if (threadIdx.x == 0) *S.total[cur ^ 1] = 0;
    }
    const int count = S.cnt[cur][g];
    if (s0 >= count) return;
    const int ncols = min(SG_TN, count - s0);
    const int32_t* act = S.act[cur] + (size_t)g * S.nchains + s0;
    const int p = P.p;
    const T* __restrict__ Mg = P.M + (size_t)g * p * p;

    __shared__ __align__(16) T As[2][TK][SG_TM];
    __shared__ __align__(16) T Bs[2][TK][LDB];
    __shared__ int32_t slots[SG_TN];
    __shared__ T red[8][SG_TN][5];
    if (threadIdx.x < SG_TN) slots[threadIdx.x] = threadIdx.x < ncols ? act[threadIdx.x] : -1;
    __syncthreads();

    T ra[A_PER], rb[B_PER];
    auto fetch = [&](int kb) {
#pragma unroll
        for (int h = 0; h < A_PER; ++h) {                    // A: row kb+kk of M, cols i0..
            const int e = threadIdx.x + 256 * h;
            const int kk = e / SG_TM, il = e % SG_TM;
            const int k = kb + kk, i = i0 + il;
            ra[h] = (k < p && i < p) ? Mg[(size_t)k * p + i] : T(0);
        }
#pragma unroll
        for (int h = 0; h < B_PER; ++h) {                    // B: V[slot][kb .. kb+TK)
            const int e = threadIdx.x + 256 * h;
            const int cl = e / TK, kk = e % TK;
            const int sl = slots[cl], k = kb + kk;
            rb[h] = (sl >= 0 && k < p) ? Vc[(size_t)sl * p + k] : T(0);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int h = 0; h < A_PER; ++h) {
            const int e = threadIdx.x + 256 * h;
            As[buf][e / SG_TM][e % SG_TM] = ra[h];
        }
#pragma unroll
        for (int h = 0; h < B_PER; ++h) {
            const int e = threadIdx.x + 256 * h;
            Bs[buf][e % TK][e / TK] = rb[h];
        }
    };

    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    fetch(0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int kb = 0; kb < p; kb += TK) {
        const bool more = kb + TK < p;
        if (more) fetch(kb + TK);                            // in flight during the FMAs
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[8], b[4];
#pragma unroll
            for (int w = 0; w < 8; ++w) a[w] = As[buf][kk][ty * 8 + w];
#pragma unroll
            for (int w = 0; w < 4; ++w) b[w] = Bs[buf][kk][tx * 4 + w];
#pragma unroll
            for (int w = 0; w < 8; ++w)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[w][v] = fma(a[w], b[v], acc[w][v]);
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    // epilogue: thread owns chains 4*tx + v and rows 8*ty + w
    T part[4][5];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
#pragma unroll
        for (int t = 0; t < 5; ++t) part[v][t] = T(0);
        const int sl = slots[tx * 4 + v];
        if (sl < 0) continue;
        int gg, e;
        slot_coords(P, S.nchains, sl, gg, e);
        const T kappa = (T)P.lambdas[S.slot_j[sl]] / P.rho;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int i = i0 + ty * 8 + w;
            if (i < p) admm_elem(P, acc[w][v], g, e, sl, i, kappa, z, u, Vn, part[v]);
        }
    }
    // lanes l and l^16 hold rows of the same chains (ty differs by one)
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int t = 0; t < 5; ++t) part[v][t] += __shfl_xor_sync(0xffffffffu, part[v][t], 16);
    if ((threadIdx.x & 31) < 16)
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int t = 0; t < 5; ++t) red[threadIdx.x >> 5][tx * 4 + v][t] = part[v][t];
    __syncthreads();
    if (threadIdx.x < ncols) {
        const int sl = slots[threadIdx.x];
        T tot[5] = {};
        for (int w = 0; w < 8; ++w)                        // fixed order over row groups
#pragma unroll
            for (int t = 0; t < 5; ++t) tot[t] += red[w][threadIdx.x][t];
#pragma unroll
        for (int t = 0; t < 5; ++t) norms[((size_t)sl * RT + rt) * 5 + t] = tot[t];
    }
}

// Few chains per group (path-warm LASSO: one): one warp per row computes the
// dot products of M_g[i, :] with every active chain of the group.
template <typename T, int NC>
__global__ void __launch_bounds__(256)
k_stream_gemv(AdmmDev<T> P, StreamState S, int cur, const T* __restrict__ Vc, T* Vn, T* z, T* u,
              T* norms, int RT)
{
    const int g = blockIdx.y;
    const int rt = blockIdx.x;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < 32) {
        for (int t = threadIdx.x; t < P.G; t += 32) S.cnt[cur ^ 1][t] = 0;
        if (threadIdx.x == 0) *S.total[cur ^ 1] = 0;
    }
    const int count = min(S.cnt[cur][g], NC);
    if (count == 0) return;
    const int p = P.p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = rt * GV_ROWS + warp;
    const int32_t* act = S.act[cur] + (size_t)g * S.nchains;
    __shared__ T red[GV_ROWS][NC][5];
    int sl[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sl[c] = c < count ? act[c] : -1;
    T part[NC][5];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int t = 0; t < 5; ++t) part[c][t] = T(0);
    if (i < p) {
        const T* Mi = P.M + (size_t)g * p * p + (size_t)i * p;
        T acc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = T(0);
        for (int k = lane; k < p; k += 32) {
            const T mv = Mi[k];
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (sl[c] >= 0) acc[c] = fma(mv, Vc[(size_t)sl[c] * p + k], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = warp_sum(acc[c]);
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (sl[c] < 0) continue;
                int gg, e;
                slot_coords(P, S.nchains, sl[c], gg, e);
                const T kappa = (T)P.lambdas[S.slot_j[sl[c]]] / P.rho;
                admm_elem(P, acc[c], g, e, sl[c], i, kappa, z, u, Vn, part[c]);
            }
        }
    }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int t = 0; t < 5; ++t) red[warp][c][t] = part[c][t];
    __syncthreads();
    if (threadIdx.x < count) {
        const int c = threadIdx.x;
        T tot[5] = {};
        for (int w = 0; w < GV_ROWS; ++w)
#pragma unroll
            for (int t = 0; t < 5; ++t) tot[t] += red[w][c][t];
#pragma unroll
        for (int t = 0; t < 5; ++t) norms[((size_t)act[c] * RT + rt) * 5 + t] = tot[t];
    }
}

// One warp per active slot: reduce the row-tile partial norms in order, test
// convergence, finish the column and advance the chain, compact the list.
template <typename T>
__global__ void k_stream_check(AdmmDev<T> P, StreamState S, int cur, T* z, T* u, T* Vn,
                               const T* norms, int RT)
{
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.y;
    const int count = S.cnt[cur][g];
    if (warp_global >= count) return;
    const int sl = S.act[cur][(size_t)g * S.nchains + warp_global];
    const int p = P.p;
    T tot[5] = {};
    for (int t0 = 0; t0 < RT; t0 += 32) {
        T loc[5] = {};
        const int t = t0 + lane;
        if (t < RT)
#pragma unroll
            for (int c = 0; c < 5; ++c) loc[c] = norms[((size_t)sl * RT + t) * 5 + c];
        // fixed-order tree over 32 lanes, then sequential over 32-chunks
#pragma unroll
        for (int c = 0; c < 5; ++c) tot[c] += warp_sum(loc[c]);
    }
    int it = S.slot_it[sl] + 1;
    const T xn = sqrt(tot[2]), zn = sqrt(tot[3]);
    const T eps_pri = P.sqrtp * P.abs_tol + P.rel_tol * (xn > zn ? xn : zn);
    const T eps_dual = P.sqrtp * P.abs_tol + P.rel_tol * P.rho * sqrt(tot[4]);
    const bool converged = sqrt(tot[0]) <= eps_pri && P.rho * sqrt(tot[1]) <= eps_dual;
    bool still = true;
    if (converged || it >= P.max_iter) {
        int gg, e;
        slot_coords(P, S.nchains, sl, gg, e);
        const int j = S.slot_j[sl];
        const int64_t col_je = (int64_t)j * P.r + e;
        const int64_t col = (int64_t)g * P.q * P.r + col_je;
        const T* zs = z + (size_t)sl * p;
        const T* us = u + (size_t)sl * p;
        // threshold lambda_j / rho, once per column (FP64 division off the loop)
        const T kappa_j = P.near_count ? (T)(P.lambdas[j] / (double)P.rho) : T(0);
        for (int a = 0; 32 * a < p; ++a) {
            const int i = lane + 32 * a;
            const T zi = i < p ? zs[i] : T(0);
            if (P.beta && i < p && UOI_IN_BOUNDS(col * p + i, (int64_t)P.G * P.q * P.r * p, 202))
                P.beta[col * p + i] = (double)zi;
            if (P.u_out && i < p) P.u_out[col * p + i] = (double)us[i];
            if (P.family) {
                const unsigned bal = __ballot_sync(0xffffffffu, zi != T(0));
                if (lane == 0) and_family_bits(P, col_je, a, bal);
            }
            if (P.near_count)
                count_near_threshold<T>(i < p, zi, i < p ? us[i] : T(0), kappa_j, (T)kNearThreshold,
                                        P.near_count);
        }
        if (lane == 0) {
            if (P.iters) P.iters[col] = it;
            if (P.conv) P.conv[col] = converged ? 1 : 0;
        }
        const int jn = j + 1;
        if (jn < S.slot_jend[sl]) {
            if (lane == 0) S.slot_j[sl] = jn;
            it = 0;
        } else {
            still = false;
        }
    }
    if (lane == 0) {
        S.slot_it[sl] = it;
        if (still) {
            const int pos = atomicAdd(&S.cnt[cur ^ 1][g], 1);
            S.act[cur ^ 1][(size_t)g * S.nchains + pos] = sl;
            atomicAdd(S.total[cur ^ 1], 1);
        }
    }
}

// Cold schedule with a learned start: slot s is column s, so z, u and
// V = z - u start from the given state.
template <typename T>
__global__ void k_stream_init_state(AdmmDev<T> P, int64_t count, T* z, T* u, T* V)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const T zz = (T)P.z0[t], uu = (T)P.u0[t];
        z[t] = zz;
        u[t] = uu;
        V[t] = zz - uu;
    }
}

template <typename T>
__global__ void k_stream_init(AdmmDev<T> P, StreamState S)
{
    const int64_t total = (int64_t)P.G * S.nchains;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int cid = (int)(s % S.nchains);
        const int g = (int)(s / S.nchains);
        if (P.warm) { S.slot_j[s] = 0; S.slot_jend[s] = P.q; }
        else        { S.slot_j[s] = cid / P.r; S.slot_jend[s] = cid / P.r + 1; }
        S.slot_it[s] = 0;
        S.act[0][s] = (int32_t)s;
        if (cid == 0) S.cnt[0][g] = S.nchains;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *S.total[0] = (int32_t)total;
}

template <typename T>
AdmmDev<T> to_dev(const AdmmProblem<T>& P)
{
    AdmmDev<T> d;
    d.G = P.G; d.q = P.q; d.max_iter = P.max_iter; d.warm = P.warm;
    d.p = (int32_t)P.p; d.r = (int32_t)P.r; d.W = (int32_t)((P.p + 63) / 64);
    d.M = P.M; d.c = P.c; d.lambdas = P.lambdas;
    d.rho = (T)P.rho; d.abs_tol = (T)P.abs_tol; d.rel_tol = (T)P.rel_tol;
    d.sqrtp = (T)sqrt((double)P.p);
    d.beta = P.beta; d.iters = P.iters; d.conv = P.conv; d.family = P.family;
    d.u_out = P.u_out; d.z0 = P.z0; d.u0 = P.u0; d.near_count = P.near_count;
    return d;
}

template <typename T, int A, int SW>
void launch_resident(const AdmmDev<T>& d, int32_t* chain_next, cudaStream_t s)
{
    const int p4 = (d.p + 3) & ~3;
    const size_t smem = sizeof(T) * ((size_t)p4 * A * 32 + (size_t)8 * SW * A * 32);
    auto kern = k_admm_resident<T, A, SW>;
    allow_max_dynamic_smem((const void*)kern);
    const int nchains = d.warm ? d.r : d.r * d.q;
    const int per_cta = 8 * SW;
    int ctas = (int)ceil_div(nchains, per_cta);
    const int fill = std::max(1, 152 / std::max(1, d.G));
    ctas = std::max(1, std::min(ctas, fill));
    k_admm_resident<T, A, SW><<<dim3((unsigned)ctas, (unsigned)d.G), 256, smem, s>>>(d, chain_next);
    UOI_CHECK_LAUNCH();
    count_launch();
}

template <typename T>
bool try_resident(const AdmmDev<T>& d, int32_t* chain_next, cudaStream_t s);

template <>
bool try_resident<double>(const AdmmDev<double>& d, int32_t* chain_next, cudaStream_t s)
{
    if (d.p <= 64) { launch_resident<double, 2, 4>(d, chain_next, s); return true; }
    if (d.p <= 128) { launch_resident<double, 4, 4>(d, chain_next, s); return true; }
    return false;
}

template <>
bool try_resident<float>(const AdmmDev<float>& d, int32_t* chain_next, cudaStream_t s)
{
    if (d.p <= 64) { launch_resident<float, 2, 4>(d, chain_next, s); return true; }
    if (d.p <= 128) { launch_resident<float, 4, 4>(d, chain_next, s); return true; }
    if (d.p <= 192) { launch_resident<float, 6, 4>(d, chain_next, s); return true; }
    return false;
}

}  // namespace

template <typename T>
void admm_solve(const AdmmProblem<T>& P, cudaStream_t s)
{
    if (P.G <= 0 || P.p <= 0 || P.r <= 0 || P.q <= 0) return;
    AdmmDev<T> d = to_dev(P);
    const int32_t nchains = P.warm ? (int32_t)P.r : (int32_t)(P.r * P.q);
    {
        DevBuf next(sizeof(int32_t) * P.G, s);
        UOI_CUDA(cudaMemsetAsync(next.ptr, 0, next.bytes, s));
        if (try_resident<T>(d, next.as<int32_t>(), s)) return;
    }
    if constexpr (sizeof(T) == 4) {
        if (admm_tc_available()) {               // FP32 state: x-update on the tensor cores
            const AdmmProblem<float>& Pf = reinterpret_cast<const AdmmProblem<float>&>(P);
            if (admm_batch_try_join(Pf, s)) return;   // solved with the rest of a batch
            admm_solve_tc(Pf, s);
            return;
        }
    }
    // streaming schedule
    const int64_t slots = (int64_t)P.G * nchains;
    const int p = (int)P.p;
    const bool gemv = nchains <= 4;
    const int RT = gemv ? (int)ceil_div(p, GV_ROWS) : (int)ceil_div(p, SG_TM);
    DevBuf zb(sizeof(T) * slots * p, s), ub(sizeof(T) * slots * p, s);
    DevBuf v0(sizeof(T) * slots * p, s), v1(sizeof(T) * slots * p, s);
    DevBuf nb(sizeof(T) * slots * RT * 5, s);
    DevBuf sj(sizeof(int32_t) * slots, s), sje(sizeof(int32_t) * slots, s), sit(sizeof(int32_t) * slots, s);
    DevBuf a0(sizeof(int32_t) * slots, s), a1(sizeof(int32_t) * slots, s);
    DevBuf c0(sizeof(int32_t) * P.G, s), c1(sizeof(int32_t) * P.G, s);
    DevBuf tot(sizeof(int32_t) * 2, s);
    UOI_CUDA(cudaMemsetAsync(zb.ptr, 0, zb.bytes, s));
    UOI_CUDA(cudaMemsetAsync(ub.ptr, 0, ub.bytes, s));
    UOI_CUDA(cudaMemsetAsync(v0.ptr, 0, v0.bytes, s));
    UOI_CUDA(cudaMemsetAsync(c0.ptr, 0, c0.bytes, s));
    StreamState S;
    S.slot_j = sj.as<int32_t>(); S.slot_jend = sje.as<int32_t>(); S.slot_it = sit.as<int32_t>();
    S.act[0] = a0.as<int32_t>(); S.act[1] = a1.as<int32_t>();
    S.cnt[0] = c0.as<int32_t>(); S.cnt[1] = c1.as<int32_t>();
    S.total[0] = tot.as<int32_t>(); S.total[1] = tot.as<int32_t>() + 1;
    S.nchains = nchains;
    k_stream_init<T><<<(unsigned)std::min<int64_t>(ceil_div(slots, 256), 4096), 256, 0, s>>>(d, S);
    UOI_CHECK_LAUNCH();
    count_launch();
    if (P.z0 && !P.warm) {
        k_stream_init_state<T><<<(unsigned)std::min<int64_t>(ceil_div(slots * p, 256), 8192), 256, 0, s>>>(
            d, slots * p, zb.as<T>(), ub.as<T>(), v0.as<T>());
        UOI_CHECK_LAUNCH();
        count_launch();
    }

    int32_t* host_total = pinned_scratch_i32();
    const int64_t bound = (int64_t)(P.warm ? P.q : 1) * P.max_iter + 2;
    const int check_every = 8;
    T* V[2] = { v0.as<T>(), v1.as<T>() };
    int cur = 0;
    bool done = false;
    try {
        for (int64_t it = 0; it < bound && !done; ++it) {
            if (gemv) {
                dim3 grid((unsigned)RT, (unsigned)P.G);
                k_stream_gemv<T, 4><<<grid, 256, 0, s>>>(d, S, cur, V[cur], V[cur ^ 1], zb.as<T>(),
                                                          ub.as<T>(), nb.as<T>(), RT);
            } else {
                dim3 grid((unsigned)RT, (unsigned)ceil_div(nchains, SG_TN), (unsigned)P.G);
                ktimer_begin(TK_XUPDATE, s);
                k_stream_gemm<T><<<grid, 256, 0, s>>>(d, S, cur, V[cur], V[cur ^ 1], zb.as<T>(),
                                                      ub.as<T>(), nb.as<T>(), RT);
                ktimer_end(TK_XUPDATE, s, 0.0, 0.0);
            }
            UOI_CHECK_LAUNCH();
            dim3 gc((unsigned)ceil_div(nchains, 8), (unsigned)P.G);
            k_stream_check<T><<<gc, 256, 0, s>>>(d, S, cur, zb.as<T>(), ub.as<T>(), V[cur ^ 1],
                                                  nb.as<T>(), RT);
            UOI_CHECK_LAUNCH();
            count_launch(2);
            cur ^= 1;
            if ((it + 1) % check_every == 0 || it + 1 == bound) {
                UOI_CUDA(cudaMemcpyAsync(host_total, S.total[cur], sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, s));
                UOI_CUDA(cudaStreamSynchronize(s));
                done = *host_total == 0;
            }
        }
    } catch (...) {
        throw;
    }
    if (!done) throw Error(UOI_ERR_TIMEOUT, "ADMM streaming loop exceeded its iteration bound");
}

template void admm_solve<double>(const AdmmProblem<double>&, cudaStream_t);
template void admm_solve<float>(const AdmmProblem<float>&, cudaStream_t);

template <typename T>
bool admm_solve_resident_with(const AdmmProblem<T>& P, int32_t* chain_next, cudaStream_t s)
{
    if (P.G <= 0 || P.p <= 0 || P.r <= 0 || P.q <= 0) return true;
    const AdmmDev<T> d = to_dev(P);
    return try_resident<T>(d, chain_next, s);
}

template bool admm_solve_resident_with<double>(const AdmmProblem<double>&, int32_t*, cudaStream_t);

}  // namespace uoi
