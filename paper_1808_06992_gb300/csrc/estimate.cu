// estimate.cu -- G5-G7: support family, support-restricted OLS, held-out loss,
// argmin over the family and bagging (Alg. 1/2 model estimation, Eq. 3-4).
//
// For estimation bootstrap k and family member S_j (per response e):
//   beta = argmin || W^{1/2} (y_e - X_S b) ||   from G'_k[S,S] (FP64 moments):
//   FP32 Cholesky + FP64 iterative refinement, FP64 Cholesky where FP32 is
//   not safe (see k_ols_mixed)
//   L_kje = sum_{t in E^k} (y_te - x_t beta)^2
//         = y_E'y_E - 2 beta' (X_E'y_E)_S + beta' G^E_k[S,S] beta
// j*_k = argmin_j sum_e L_kje (ties -> smallest j); beta*_e = median (or mean)
// over k of the chosen estimates (zero outside the support).
// Singular supports (a Cholesky pivot <= 1e-12 max diag) are solved as the
// paper states OLS, the LASSO ADMM at lambda = 0: with no threshold z = x and
// u stays 0, so the iteration is x_{t+1} = (G + rho I)^{-1} (b + rho x_t) from
// x_0 = 0, whose iterates stay in the range of G and converge to the
// minimum-norm least-squares solution; they are flagged.
#include <algorithm>
#include <vector>

#include "kernels.h"

namespace uoi {

namespace {

constexpr int OLS_SMEM_MAX = 160;   // supports up to this size factor in shared memory (FP64 path)
constexpr int OLS_SMALL = 128;      // mixed path: supports up to this size form the small class
// ADMM at lambda = 0 for singular supports: rho relative to the largest diagonal
// (directions with eigenvalue >> rho converge in a few steps), the stopping
// test on the relative change, and the iteration cap.
constexpr double OLS_PROX_RHO = 1e-6;
constexpr double OLS_PROX_TOL = 1e-14;
constexpr int OLS_PROX_MAX = 500;

struct OlsArgs {
    const double* Gt; const double* Bt;      // B2 x p x p, B2 x p x r
    const double* Ge; const double* Be;      // B2 x p x p, B2 x p x r
    const double* yye;                       // B2 x r
    const uint64_t* family;                  // q x r x W
    int64_t p, r; int32_t q, B2, W;
    const int32_t* jstar;                    // chosen pass: B2 (else null)
    const int32_t* dup;                      // q x r: first j with the same support (or null)
    double* losses;                          // B2 x q x r
    int32_t* singular;                       // B2 x q x r (nullable)
    double* chosen;                          // chosen pass: B2 x r x p
    double* scratch;                         // global factor scratch (per CTA), or null
    int64_t solves;
    int smax;                                // max support size
    bool use_smem;
    const int32_t* list;                     // solve indices to run (null: 0 .. solves-1)
    // Moments restricted to the union U of the family supports: Gt, Ge are
    // B2 x pu x pu and Bt, Be B2 x pu x r over U's columns; upos[i] = position of
    // feature i in U, ucols[t] = feature at position t.
    const int32_t* upos;
    const int32_t* ucols;
    int64_t pu;
    int32_t* fb_list;                        // mixed pass: solves left to the FP64 kernel
    int32_t* fb_count;
    float* fscratch;                         // mixed pass: global packed factor (per CTA), or null
    const int32_t* je_list;                  // mixed loss pass: the (j*r + e) it covers (else all)
    int32_t n_je;
    // mixed loss pass with je_list: when set, CTAs take solves in order from this
    // counter (preset to 0), support-major (t = rank of je in je_list * B2 + k), so a
    // list sorted by decreasing support size runs the largest factors first
    unsigned long long* next;
};

__global__ void __launch_bounds__(256) k_ols(OlsArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* idx = reinterpret_cast<int*>(smem_raw);                         // p ints
    double* bs = reinterpret_cast<double*>(smem_raw + sizeof(int) * ((a.smax + 1) & ~1));
    double* xs = bs + a.smax + 1;                                        // solution
    double* ws = xs + a.smax + 1;                                        // work vector
    double* red = ws + a.smax + 1;                                       // 32 doubles
    double* Gs = a.use_smem ? red + 32 : a.scratch + (size_t)blockIdx.x * a.smax * a.smax;
    __shared__ int s_count;
    __shared__ int s_bad;
    __shared__ int s_done;
    __shared__ double s_dmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int64_t it = blockIdx.x; it < a.solves; it += gridDim.x) {
        const int64_t t = a.list ? a.list[it] : it;
        int k, j, e;
        if (a.jstar) { k = (int)(t / a.r); e = (int)(t % a.r); j = a.jstar[k]; }
        else { k = (int)(t / ((int64_t)a.q * a.r)); const int64_t rem = t % ((int64_t)a.q * a.r);
               j = (int)(rem / a.r); e = (int)(rem % a.r);
               if (a.dup && a.dup[rem] != j) continue; }       // duplicate support: filled later
        const uint64_t* bits = a.family + ((int64_t)j * a.r + e) * a.W;
        // support indices (warp 0, ballot compaction in increasing i)
        if (warp == 0) {
            int cnt = 0;
            for (int64_t i0 = 0; i0 < a.p; i0 += 32) {
                const int64_t i = i0 + lane;
                const bool in = i < a.p && ((bits[i >> 6] >> (i & 63)) & 1ull);
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (in) idx[cnt + __popc(bal & ((1u << lane) - 1u))] = a.upos[i];
                cnt += __popc(bal);
            }
            if (lane == 0) { s_count = cnt; s_bad = 0; }
        }
        __syncthreads();
        const int s = s_count;
        const double* Gk = a.Gt + (size_t)k * a.pu * a.pu;
        const double* Bk = a.Bt + (size_t)k * a.pu * a.r;
        double ridge = 0.0;                   // rho of the lambda = 0 ADMM (0: plain solve)
        for (int attempt = 0; attempt < 2 && s > 0; ++attempt) {
            double dm = 0.0;
            for (int x = threadIdx.x; x < s * s; x += blockDim.x) {
                const int r0 = x / s, c0 = x % s;
                const double v = Gk[(size_t)idx[r0] * a.pu + idx[c0]];
                Gs[x] = v + (r0 == c0 ? ridge : 0.0);
                if (r0 == c0) dm = fmax(dm, v);
            }
            for (int x = threadIdx.x; x < s; x += blockDim.x) bs[x] = Bk[(size_t)idx[x] * a.r + e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
            if (lane == 0) red[warp] = dm;
            __syncthreads();
            if (threadIdx.x == 0) {
                double m = 0.0;
                for (int w = 0; w < 8; ++w) m = fmax(m, red[w]);
                s_dmax = m;
                s_bad = 0;
            }
            __syncthreads();
            const double thr = 1e-12 * s_dmax;
            // unblocked right-looking Cholesky of Gs (lower)
            for (int c = 0; c < s; ++c) {
                if (threadIdx.x == 0) {
                    const double d = Gs[c * s + c];
                    if (!(d > thr)) { s_bad = 1; Gs[c * s + c] = 1.0; } else Gs[c * s + c] = sqrt(d);
                }
                __syncthreads();
                const double lcc = Gs[c * s + c];
                for (int i = c + 1 + threadIdx.x; i < s; i += blockDim.x) Gs[i * s + c] /= lcc;
                __syncthreads();
                const int rem = s - c - 1;
                for (int x = threadIdx.x; x < rem * rem; x += blockDim.x) {
                    const int i = c + 1 + x / rem, jj = c + 1 + x % rem;
                    if (jj <= i) Gs[i * s + jj] -= Gs[i * s + c] * Gs[jj * s + c];
                }
                __syncthreads();
            }
            if (!s_bad) break;
            ridge = OLS_PROX_RHO * s_dmax;    // factor G + rho I for the lambda = 0 ADMM
            __syncthreads();
        }
        const bool singular = s > 0 && ridge > 0.0;
        // x = (G + rho I)^{-1} (b + rho x): once with rho = 0 (plain Cholesky solve),
        // else the lambda = 0 ADMM iterations from x = 0
        for (int x = threadIdx.x; x < s; x += blockDim.x) xs[x] = 0.0;
        for (int itp = 0; s > 0; ++itp) {
            for (int x = threadIdx.x; x < s; x += blockDim.x) ws[x] = bs[x] + ridge * xs[x];
            __syncthreads();
            // forward / back substitution by warp 0
            if (warp == 0) {
                for (int i = 0; i < s; ++i) {
                    double acc = 0.0;
                    for (int c = lane; c < i; c += 32) acc += Gs[i * s + c] * ws[c];
                    acc = warp_sum(acc);
                    if (lane == 0) ws[i] = (ws[i] - acc) / Gs[i * s + i];
                    __syncwarp();
                }
                for (int i = s - 1; i >= 0; --i) {
                    double acc = 0.0;
                    for (int c = i + 1 + lane; c < s; c += 32) acc += Gs[c * s + i] * ws[c];
                    acc = warp_sum(acc);
                    if (lane == 0) ws[i] = (ws[i] - acc) / Gs[i * s + i];
                    __syncwarp();
                }
            }
            __syncthreads();
            double dmx = 0.0, xmx = 0.0;
            for (int x = threadIdx.x; x < s; x += blockDim.x) {
                dmx = fmax(dmx, fabs(ws[x] - xs[x]));
                xmx = fmax(xmx, fabs(ws[x]));
                xs[x] = ws[x];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dmx = fmax(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
                xmx = fmax(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
            }
            if (lane == 0) { red[warp] = dmx; red[8 + warp] = xmx; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double d = 0.0, xm = 0.0;
                for (int w = 0; w < 8; ++w) { d = fmax(d, red[w]); xm = fmax(xm, red[8 + w]); }
                s_done = (!singular || d <= OLS_PROX_TOL * xm || itp + 1 >= OLS_PROX_MAX) ? 1 : 0;
            }
            __syncthreads();
            if (s_done) break;
        }
        __syncthreads();
        if (a.jstar) {
            double* out = a.chosen + ((size_t)k * a.r + e) * a.p;
            for (int x = threadIdx.x; x < s; x += blockDim.x) out[a.ucols[idx[x]]] = xs[x];
        } else {
            // held-out loss via the evaluation moments
            const double* Gek = a.Ge + (size_t)k * a.pu * a.pu;
            const double* Bek = a.Be + (size_t)k * a.pu * a.r;
            double part = 0.0;
            for (int x = threadIdx.x; x < s * s; x += blockDim.x) {
                const int r0 = x / s, c0 = x % s;
                part += xs[r0] * Gek[(size_t)idx[r0] * a.pu + idx[c0]] * xs[c0];
            }
            for (int x = threadIdx.x; x < s; x += blockDim.x)
                part -= 2.0 * xs[x] * Bek[(size_t)idx[x] * a.r + e];
            part = warp_sum(part);
            __syncthreads();
            if (lane == 0) red[warp] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < 8; ++w) tot += red[w];
                const int64_t o = ((int64_t)k * a.q + j) * a.r + e;
                a.losses[o] = a.yye[(size_t)k * a.r + e] + tot;
                if (a.singular) a.singular[o] = singular ? 1 : 0;
            }
        }
        __syncthreads();
    }
}

// Mixed-precision form of the same solve: Cholesky of G'_k[S,S] rounded to FP32
// (packed lower triangle), then iterative refinement with FP64 residuals
// r = b - G x until the correction is at FP64 rounding level, so the result
// agrees with an FP64 factorisation to ~kappa * 1e-16.  A solve whose FP32
// pivots fall below 1e-3 of the largest diagonal (where FP32 cannot certify the
// 1e-12 singularity test) or whose refinement stalls is queued for k_ols.
constexpr float OLS_F32_PIVOT = 1e-3f;
constexpr int OLS_REFINE_MAX = 8;

__device__ __forceinline__ int packed_row(int i) { return (i * (i + 1)) >> 1; }

// w <- L^{-T} L^{-1} w with L packed lower, by the whole block: 32-row diagonal
// blocks are solved by warp 0 in registers (one shuffle per column), the rows
// beyond them are updated by all threads.
__device__ __forceinline__ void chol_solve_f32(const float* L, const float* dinv, float* w, int s, int warp,
                                               int lane)
{
    for (int c0 = 0; c0 < s; c0 += 32) {
        const int nb = min(32, s - c0);
        if (warp == 0) {
            float wi = lane < nb ? w[c0 + lane] : 0.f;
            for (int c = 0; c < nb; ++c) {
                if (lane == c) wi *= dinv[c0 + c];
                const float wc = __shfl_sync(0xffffffffu, wi, c);
                if (lane > c && lane < nb) wi -= L[packed_row(c0 + lane) + c0 + c] * wc;
            }
            if (lane < nb) w[c0 + lane] = wi;
        }
        __syncthreads();
        for (int i = c0 + nb + threadIdx.x; i < s; i += blockDim.x) {
            const float* row = L + packed_row(i) + c0;
            float acc = 0.f;
            for (int c = 0; c < nb; ++c) acc += row[c] * w[c0 + c];
            w[i] -= acc;
        }
        __syncthreads();
    }
    for (int c0 = ((s - 1) / 32) * 32; c0 >= 0; c0 -= 32) {
        const int nb = min(32, s - c0);
        if (warp == 0) {
            float xi = lane < nb ? w[c0 + lane] : 0.f;
            for (int c = nb - 1; c >= 0; --c) {
                if (lane == c) xi *= dinv[c0 + c];
                const float xc = __shfl_sync(0xffffffffu, xi, c);
                if (lane < c) xi -= L[packed_row(c0 + c) + c0 + lane] * xc;
            }
            if (lane < nb) w[c0 + lane] = xi;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < c0; i += blockDim.x) {
            float acc = 0.f;
            for (int c = 0; c < nb; ++c) acc += L[packed_row(c0 + c) + i] * w[c0 + c];
            w[i] -= acc;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double block_max(double v, double* red, int lane, int warp)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double m = red[0];
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
    return m;
}

__device__ __forceinline__ double block_sum(double v, double* red, int lane, int warp)
{
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    return t;
}

// PB: k chunk of the trailing update's 4 x 4 register tiles; MINB: CTAs per SM
// the registers must allow (small supports want many).
template <int PB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_ols_mixed(OlsArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sm2 = (a.smax + 1) & ~1;
    int* idx = reinterpret_cast<int*>(smem_raw);                        // smax ints
    double* b64 = reinterpret_cast<double*>(smem_raw + sizeof(int) * sm2);
    double* x64 = b64 + sm2;
    double* red = x64 + sm2;                                            // 32 doubles
    float* w = reinterpret_cast<float*>(red + 32);                      // smax floats
    float* dinv = w + sm2;                                              // 1 / diagonal of the factor
    float* L = a.fscratch ? a.fscratch + (size_t)blockIdx.x * ((size_t)a.smax * (a.smax + 1) / 2) : dinv + sm2;
    __shared__ int s_count;
    __shared__ int64_t s_next;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // the next solve of this CTA: a fixed stride, or the shared counter (block-uniform)
    auto fetch = [&](int64_t cur) -> int64_t {
        if (!a.next) return cur < 0 ? (int64_t)blockIdx.x : cur + gridDim.x;
        __syncthreads();                               // every thread is done with s_next
        if (threadIdx.x == 0) s_next = (int64_t)atomicAdd(a.next, 1ull);
        __syncthreads();
        return s_next;
    };

    for (int64_t t = fetch(-1); t < a.solves; t = fetch(t)) {
        int k, j, e;
        if (a.jstar) { k = (int)(t / a.r); e = (int)(t % a.r); j = a.jstar[k]; }
        else if (a.je_list) {
            int32_t je;
            if (a.next) { k = (int)(t % a.B2); je = a.je_list[t / a.B2]; }
            else { k = (int)(t / a.n_je); je = a.je_list[t % a.n_je]; }
            j = (int)(je / a.r); e = (int)(je % a.r);
        } else { k = (int)(t / ((int64_t)a.q * a.r)); const int64_t rem = t % ((int64_t)a.q * a.r);
               j = (int)(rem / a.r); e = (int)(rem % a.r);
               if (a.dup && a.dup[rem] != j) continue; }
        // the solve's index in the numbering of k_ols (for the FP64 hand-over)
        const int64_t tg = a.jstar ? t : ((int64_t)k * a.q + j) * a.r + e;
        const uint64_t* bits = a.family + ((int64_t)j * a.r + e) * a.W;
        if (warp == 0) {
            int cnt = 0;
            for (int64_t i0 = 0; i0 < a.p; i0 += 32) {
                const int64_t i = i0 + lane;
                const bool in = i < a.p && ((bits[i >> 6] >> (i & 63)) & 1ull);
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (in) idx[cnt + __popc(bal & ((1u << lane) - 1u))] = a.upos[i];
                cnt += __popc(bal);
            }
            if (lane == 0) s_count = cnt;
        }
        __syncthreads();
        const int s = s_count;
        const double* Gk = a.Gt + (size_t)k * a.pu * a.pu;
        const double* Bk = a.Bt + (size_t)k * a.pu * a.r;
        // gather the packed lower triangle in FP32, b in FP64
        double dm = 0.0;
        for (int i = warp; i < s; i += 8) {
            const double* grow = Gk + (size_t)idx[i] * a.pu;
            float* lrow = L + packed_row(i);
#pragma unroll 4
            for (int c = lane; c <= i; c += 32) {
                const double v = grow[idx[c]];
                lrow[c] = f64_to_f32_int(v);
                if (c == i) dm = fmax(dm, v);
            }
        }
        for (int x = threadIdx.x; x < s; x += blockDim.x) b64[x] = Bk[(size_t)idx[x] * a.r + e];
        const double dmax = block_max(dm, red, lane, warp);
        const float thr = OLS_F32_PIVOT * (float)dmax;
        // blocked right-looking Cholesky with 32-column panels: warp 0 factors the
        // diagonal block in registers (no block barrier per column), every
        // thread solves one row of the panel below it against that block, then the
        // trailing triangle takes the rank-32 update in 4 x 4 register tiles
        // (k chunks of PB) over 64 x 64 blocks of 16 x 16 threads: three barriers
        // per 32 columns
        __shared__ int s_ok;
        bool ok = true;
        for (int c0 = 0; c0 < s; c0 += 32) {
            const int c1 = min(s, c0 + 32);
            if (warp == 0) {
                // lane i holds row c0 + i of the diagonal block in registers;
                // column c of the factor travels between lanes by shuffles
                const int nb = c1 - c0;
                const bool has = lane < nb;
                float* lrow = L + packed_row(c0 + (has ? lane : 0)) + c0;
                float a[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) a[j] = (has && j <= lane) ? lrow[j] : 0.f;
                bool wok = true;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    if (c >= nb || !wok) continue;                   // same in every lane
                    const float d = __shfl_sync(0xffffffffu, a[c], c);
                    if (!(d > thr)) { wok = false; continue; }
                    const float lcc = sqrtf(d);
                    const float inv = 1.f / lcc;
                    const float lic = lane > c ? a[c] * inv : 0.f;
                    if (lane == c) a[c] = lcc;
                    else if (lane > c) a[c] = lic;
                    if (lane == 0) dinv[c0 + c] = inv;
#pragma unroll
                    for (int j = c + 1; j < 32; ++j) {
                        const float ljc = __shfl_sync(0xffffffffu, lic, j);
                        if (lane >= j) a[j] -= lic * ljc;
                    }
                }
                if (wok && has) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j <= lane) lrow[j] = a[j];
                }
                if (lane == 0) s_ok = wok ? 1 : 0;
            }
            __syncthreads();
            if (!s_ok) { ok = false; break; }
            // panel rows below the block: L21 = A21 L11^{-T}, one row per thread
            for (int r = c1 + threadIdx.x; r < s; r += blockDim.x) {
                float* lr = L + packed_row(r);
                for (int c = c0; c < c1; ++c) {
                    const float* lc = L + packed_row(c);
                    float acc = lr[c];
                    for (int t = c0; t < c; ++t) acc -= lr[t] * lc[t];
                    lr[c] = acc * dinv[c];
                }
            }
            __syncthreads();
            const int T = s - c1;
            const int nbk = (T + 63) / 64;
            for (int pr = 0; pr < nbk * (nbk + 1) / 2; ++pr) {
                int bi = (int)((sqrtf(8.f * pr + 1.f) - 1.f) * 0.5f);
                while ((bi + 1) * (bi + 2) / 2 <= pr) ++bi;
                while (bi * (bi + 1) / 2 > pr) --bi;
                const int bj = pr - bi * (bi + 1) / 2;
                const int i0 = c1 + bi * 64, j0 = c1 + bj * 64;
                float acc[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
                for (int k0 = c0; k0 < c1; k0 += PB) {
                    float li[4][PB], lj[4][PB];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * u;
#pragma unroll
                        for (int t = 0; t < PB; ++t) {
                            const bool kin = k0 + t < c1;
                            li[u][t] = (i < s && kin) ? L[packed_row(i) + k0 + t] : 0.f;
                            lj[u][t] = (j < s && kin) ? L[packed_row(j) + k0 + t] : 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v)
#pragma unroll
                            for (int t = 0; t < PB; ++t) acc[u][v] += li[u][t] * lj[v][t];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + ty + 16 * u;
                    if (i >= s) break;
                    float* lrow = L + packed_row(i);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int j = j0 + tx + 16 * v;
                        if (j > i) break;
                        lrow[j] -= acc[u][v];
                    }
                }
            }
            __syncthreads();
        }
        bool done = false;
        if (ok) {
            // x = solve(b) in FP32, then x += solve(b - G x) with FP64 residuals
            for (int x = threadIdx.x; x < s; x += blockDim.x) { w[x] = (float)b64[x]; x64[x] = 0.0; }
            __syncthreads();
            double prev = 0.0;
            for (int itr = 0; itr <= OLS_REFINE_MAX; ++itr) {
                chol_solve_f32(L, dinv, w, s, warp, lane);
                double dd = 0.0, xx = 0.0;
                for (int x = threadIdx.x; x < s; x += blockDim.x) {
                    const double nx = x64[x] + (double)w[x];
                    dd = fmax(dd, fabs((double)w[x]));
                    xx = fmax(xx, fabs(nx));
                    x64[x] = nx;
                }
                const double dmx = block_max(dd, red, lane, warp);
                const double xmx = block_max(xx, red, lane, warp);
                // converged: the correction is at the level of FP64 rounding of the
                // residual, or it no longer shrinks (the residual is rounding noise)
                if (itr > 0 && (dmx <= 1e-14 * xmx || (dmx > 0.5 * prev && dmx <= 1e-12 * xmx))) {
                    done = true;
                    break;
                }
                if (itr == OLS_REFINE_MAX) { done = dmx <= 1e-12 * xmx; break; }
                prev = dmx;
                // residual r_i = b_i - sum_c G[S_i, S_c] x_c (one warp per row)
                for (int i = warp; i < s; i += 8) {
                    const double* grow = Gk + (size_t)idx[i] * a.pu;
                    double acc = 0.0;
#pragma unroll 4
                    for (int c = lane; c < s; c += 32) acc += grow[idx[c]] * x64[c];
                    acc = warp_sum(acc);
                    if (lane == 0) w[i] = (float)(b64[i] - acc);
                }
                __syncthreads();
            }
        }
        if (s > 0 && !done) {
            if (threadIdx.x == 0) a.fb_list[atomicAdd(a.fb_count, 1)] = (int32_t)tg;
            __syncthreads();
            continue;
        }
        if (a.jstar) {
            double* out = a.chosen + ((size_t)k * a.r + e) * a.p;
            for (int x = threadIdx.x; x < s; x += blockDim.x) out[a.ucols[idx[x]]] = x64[x];
        } else {
            const double* Gek = a.Ge + (size_t)k * a.pu * a.pu;
            const double* Bek = a.Be + (size_t)k * a.pu * a.r;
            double part = 0.0;
            for (int i = warp; i < s; i += 8) {
                const double* grow = Gek + (size_t)idx[i] * a.pu;
                double acc = 0.0;
#pragma unroll 4
                for (int c = lane; c < s; c += 32) acc += grow[idx[c]] * x64[c];
                acc = warp_sum(acc);
                if (lane == 0) part += x64[i] * acc;
            }
            for (int x = threadIdx.x; x < s; x += blockDim.x)
                part -= 2.0 * x64[x] * Bek[(size_t)idx[x] * a.r + e];
            const double tot = block_sum(part, red, lane, warp);
            if (threadIdx.x == 0) {
                const int64_t o = ((int64_t)k * a.q + j) * a.r + e;
                a.losses[o] = a.yye[(size_t)k * a.r + e] + tot;
                if (a.singular) a.singular[o] = 0;
            }
        }
        __syncthreads();
    }
}

// out[k][a][b] = G[k][cols[a]][cols[b]] (restriction to the union U).
__global__ void k_gather_gram(const double* G, int64_t p, const int32_t* cols, int64_t u, int32_t B,
                              double* out)
{
    const int64_t per = u * u, total = (int64_t)B * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / per, rem = t % per;
        out[t] = G[(k * p + cols[rem / u]) * p + cols[rem % u]];
    }
}

// out[k][a][e] = Bm[k][cols[a]][e].
__global__ void k_gather_rhs(const double* Bm, int64_t p, int64_t r, const int32_t* cols, int64_t u,
                             int32_t B, double* out)
{
    const int64_t per = u * r, total = (int64_t)B * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / per, rem = t % per;
        out[t] = Bm[(k * p + cols[rem / r]) * r + rem % r];
    }
}

__global__ void k_union_pos(const int32_t* cols, int64_t u, int32_t* pos)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < u;
         t += (int64_t)gridDim.x * blockDim.x)
        pos[cols[t]] = (int32_t)t;
}

// dup[j*r + e] = smallest j' <= j whose support for response e equals S_{j,e}.
__global__ void k_family_dedup(const uint64_t* fam, int32_t q, int64_t r, int W, int32_t* dup)
{
    const int64_t total = (int64_t)q * r;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / r);
        const int64_t e = t % r;
        const uint64_t* a = fam + t * W;
        int first = j;
        for (int jj = 0; jj < j; ++jj) {
            const uint64_t* b = fam + ((int64_t)jj * r + e) * W;
            bool same = true;
            for (int w = 0; w < W && same; ++w) same = a[w] == b[w];
            if (same) { first = jj; break; }
        }
        dup[t] = first;
    }
}

// Copy the loss (and flag) of the representative to every duplicate (k, j, e).
__global__ void k_fill_duplicates(const int32_t* dup, int32_t B2, int32_t q, int64_t r,
                                  double* losses, int32_t* singular)
{
    const int64_t total = (int64_t)B2 * q * r;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / ((int64_t)q * r), rem = t % ((int64_t)q * r);
        const int64_t e = rem % r;
        const int32_t j0 = dup[rem];
        if (j0 == (int32_t)(rem / r)) continue;
        const int64_t src = (k * q + j0) * r + e;
        losses[t] = losses[src];
        if (singular) singular[t] = singular[src];
    }
}

__global__ void k_support_sizes(const uint64_t* fam, int64_t count, int W, int32_t* out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        for (int w = 0; w < W; ++w) c += __popcll(fam[t * W + w]);
        out[t] = c;
    }
}

__global__ void k_support_max(const uint64_t* fam, int64_t count, int W, int32_t* out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        for (int w = 0; w < W; ++w) c += __popcll(fam[t * W + w]);
        atomicMax(out, c);
    }
}

__global__ void k_argmin(const double* losses, int32_t q, int64_t r, int32_t* jstar)
{
    const int k = blockIdx.x;
    if (threadIdx.x != 0) return;
    int best = 0;
    double bv = 0.0;
    for (int j = 0; j < q; ++j) {
        double s = 0.0;
        for (int64_t e = 0; e < r; ++e) s += losses[((int64_t)k * q + j) * r + e];
        if (j == 0 || s < bv) { bv = s; best = j; }
    }
    jstar[k] = best;
}

__global__ void k_bagging(const double* chosen, int32_t B2, int64_t count, int32_t mode, double* out)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < count;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (mode == UOI_BAG_MEAN) {
            double s = 0.0;
            for (int k = 0; k < B2; ++k) s += chosen[(int64_t)k * count + c];
            out[c] = s / (double)B2;
        } else {
            double v[128];
            const int n = B2 < 128 ? B2 : 128;
            for (int k = 0; k < n; ++k) {            // insertion sort
                const double x = chosen[(int64_t)k * count + c];
                int t = k;
                while (t > 0 && v[t - 1] > x) { v[t] = v[t - 1]; --t; }
                v[t] = x;
            }
            out[c] = (n & 1) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
        }
    }
}

__global__ void k_mask_tail(uint64_t* fam, int64_t count, int W, uint64_t mask)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        fam[t * W + (W - 1)] &= mask;
}

int32_t family_support_max(const OlsArgs& a, cudaStream_t s)
{
    DevBuf mx(sizeof(int32_t), s);
    UOI_CUDA(cudaMemsetAsync(mx.ptr, 0, sizeof(int32_t), s));
    const int64_t fam_count = (int64_t)a.q * a.r;
    k_support_max<<<(unsigned)std::min<int64_t>(ceil_div(fam_count, 256), 1024), 256, 0, s>>>(
        a.family, fam_count, a.W, mx.as<int32_t>());
    UOI_CHECK_LAUNCH();
    count_launch();
    int32_t smax = 0;
    UOI_CUDA(cudaMemcpyAsync(&smax, mx.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    return smax;
}

// FP64 solves (all of a.solves, or those listed in a.list); a.smax set.
void launch_ols_fp64(OlsArgs a, cudaStream_t s)
{
    a.use_smem = a.smax <= OLS_SMEM_MAX;
    size_t smem = sizeof(int) * ((a.smax + 1) & ~1) + sizeof(double) * (3 * (a.smax + 1) + 32);
    DevBuf scratch;
    int grid = (int)std::min<int64_t>(a.solves, 152 * 8);
    if (a.use_smem) {
        smem += sizeof(double) * (size_t)a.smax * a.smax;
    } else {
        grid = (int)std::min<int64_t>(a.solves, 152 * 2);
        scratch.alloc(sizeof(double) * (size_t)grid * a.smax * a.smax, s);
        a.scratch = scratch.as<double>();
    }
    allow_max_dynamic_smem((const void*)k_ols);
    if (a.solves > 0) {
        k_ols<<<grid, 256, smem, s>>>(a);
        UOI_CHECK_LAUNCH();
        count_launch();
    }
}

// Mixed pass: FP32 factor + FP64 refinement for every solve (ols_mixed_start,
// asynchronous on s), then the FP64 kernel for the solves it handed back
// (ols_mixed_finish, which waits for the count).
struct OlsMixedRun {
    OlsArgs a{};                  // solves = 0 until started: finish does nothing
    DevBuf fscratch, fbl, fbc;
};

void ols_mixed_start(OlsArgs a, cudaStream_t s, OlsMixedRun& R)
{
    R.a = a;
    if (a.solves == 0) return;
    const int sm2 = (a.smax + 1) & ~1;
    const size_t base = sizeof(int) * sm2 + 2 * sizeof(double) * sm2 + 32 * sizeof(double) +
                        2 * sizeof(float) * sm2;
    const size_t lbytes = sizeof(float) * (size_t)a.smax * (a.smax + 1) / 2;
    const size_t cap = 227 * 1024 - 64;
    const bool in_smem = base + lbytes <= cap;
    const size_t smem = base + (in_smem ? lbytes : 0);
    // small supports: narrow panels and few registers, many CTAs per SM (their
    // steps are short and latency-bound); large ones: wide register tiles
    const bool small = a.smax <= OLS_SMALL;
    const void* kern = small ? (const void*)k_ols_mixed<2, 4> : (const void*)k_ols_mixed<8, 1>;
    allow_max_dynamic_smem(kern);
    int dev = 0, nsm = 0, per = 0;
    UOI_CUDA(cudaGetDevice(&dev));
    UOI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    UOI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem));
    const int grid = (int)std::min<int64_t>(a.solves, (int64_t)nsm * std::max(1, per));
    if (!in_smem) {
        R.fscratch.alloc(lbytes * (size_t)grid, s);
        R.a.fscratch = R.fscratch.as<float>();
    }
    R.fbl.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(a.solves, (int64_t)a.B2 * a.q * a.r), s);
    R.fbc.alloc(sizeof(int32_t), s);
    UOI_CUDA(cudaMemsetAsync(R.fbc.ptr, 0, sizeof(int32_t), s));
    R.a.fb_list = R.fbl.as<int32_t>();
    R.a.fb_count = R.fbc.as<int32_t>();
    if (small) k_ols_mixed<2, 4><<<grid, 256, smem, s>>>(R.a);
    else k_ols_mixed<8, 1><<<grid, 256, smem, s>>>(R.a);
    UOI_CHECK_LAUNCH();
    count_launch();
}

int64_t ols_mixed_finish(OlsMixedRun& R, cudaStream_t s)
{
    if (R.a.solves == 0) return 0;
    int32_t nfb = 0;
    UOI_CUDA(cudaMemcpyAsync(&nfb, R.fbc.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    if (nfb > 0) {
        OlsArgs a = R.a;
        a.list = R.fbl.as<int32_t>();
        a.solves = nfb;
        a.fscratch = nullptr;
        launch_ols_fp64(a, s);
    }
    return nfb;
}

int64_t launch_ols_mixed(OlsArgs a, cudaStream_t s)
{
    OlsMixedRun R;
    ols_mixed_start(a, s, R);
    return ols_mixed_finish(R, s);
}

int64_t run_ols(OlsArgs a, cudaStream_t s)
{
    a.smax = std::max(1, (int)family_support_max(a, s));
    if (a.smax > 46000) throw Error(UOI_ERR_UNSUPPORTED, "OLS support larger than 46000 columns");
    return launch_ols_mixed(a, s);
}

// U = union over (j, e) of the family supports, compacted in increasing order.
__global__ void k_union_cols(const uint64_t* fam, int64_t count, int W, int64_t p, int32_t* cols,
                             int32_t* n_out)
{
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int w = 0; w < W; ++w) {
        // one block: OR of word w over all family members
        uint64_t acc = 0;
        for (int64_t t = threadIdx.x; t < count; t += blockDim.x) acc |= fam[t * W + w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, o);
        __shared__ uint64_t wred[32];
        if (lane == 0) wred[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t u = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) u |= wred[i];
            for (int b = 0; b < 64; ++b) {
                const int64_t i = (int64_t)w * 64 + b;
                if (i < p && ((u >> b) & 1ull)) cols[base++] = (int32_t)i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = base;
}

}  // namespace

// A second stream per host thread, for work that runs beside the thread's main
// stream (the small-support class of the loss pass, half of the batch of the
// tensor-core inverse); created once and kept for the thread's life.
cudaStream_t side_stream()
{
    thread_local cudaStream_t side = nullptr;
    if (!side) UOI_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    return side;
}

int32_t union_columns(const uint64_t* family, int64_t count, int64_t p, int32_t* cols,
                      cudaStream_t s)
{
    DevBuf n(sizeof(int32_t), s);
    k_union_cols<<<1, 256, 0, s>>>(family, count, (int)((p + 63) / 64), p, cols, n.as<int32_t>());
    UOI_CHECK_LAUNCH();
    count_launch();
    int32_t h = 0;
    UOI_CUDA(cudaMemcpyAsync(&h, n.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    return h;
}

void family_init(uint64_t* fam, int64_t words, cudaStream_t s)
{
    UOI_CUDA(cudaMemsetAsync(fam, 0xFF, sizeof(uint64_t) * (size_t)words, s));
}

void family_mask_tail(uint64_t* fam, int64_t count, int64_t p, cudaStream_t s)
{
    if ((p & 63) == 0) return;
    const int W = (int)((p + 63) / 64);
    k_mask_tail<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 1024), 256, 0, s>>>(
        fam, count, W, (1ull << (p & 63)) - 1ull);
    UOI_CHECK_LAUNCH();
    count_launch();
}

namespace {

// The OLS solves only touch rows and columns in the union U of the family
// supports: restricting the moments to U once per call makes every later
// access a read of a small, L2-resident matrix.
struct UnionMoments {
    DevBuf cols, pos, Gt, Bt, Ge, Be;
    int64_t pu = 0;
};

void restrict_to_union(const uint64_t* family, int64_t p, int64_t r, int32_t q, int32_t B2,
                       const double* Gt, const double* Bt, const double* Ge, const double* Be,
                       UnionMoments& U, cudaStream_t s)
{
    U.cols.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(p, 1), s);
    U.pu = union_columns(family, (int64_t)q * r, p, U.cols.as<int32_t>(), s);
    const int64_t u1 = std::max<int64_t>(U.pu, 1);
    U.pos.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(p, 1), s);
    UOI_CUDA(cudaMemsetAsync(U.pos.ptr, 0xFF, sizeof(int32_t) * (size_t)p, s));
    k_union_pos<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(U.pu, 256), 64)), 256, 0, s>>>(
        U.cols.as<int32_t>(), U.pu, U.pos.as<int32_t>());
    UOI_CHECK_LAUNCH();
    count_launch();
    auto gram = [&](const double* G, DevBuf& out) {
        out.alloc(sizeof(double) * (size_t)(B2 * u1 * u1), s);
        const int64_t total = (int64_t)B2 * U.pu * U.pu;
        if (total == 0) return;
        k_gather_gram<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 32), 256, 0, s>>>(
            G, p, U.cols.as<int32_t>(), U.pu, B2, out.as<double>());
        UOI_CHECK_LAUNCH();
        count_launch();
    };
    auto rhs = [&](const double* Bm, DevBuf& out) {
        out.alloc(sizeof(double) * (size_t)(B2 * u1 * r), s);
        const int64_t total = (int64_t)B2 * U.pu * r;
        if (total == 0) return;
        k_gather_rhs<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 32), 256, 0, s>>>(
            Bm, p, r, U.cols.as<int32_t>(), U.pu, B2, out.as<double>());
        UOI_CHECK_LAUNCH();
        count_launch();
    };
    gram(Gt, U.Gt);
    rhs(Bt, U.Bt);
    if (Ge) { gram(Ge, U.Ge); rhs(Be, U.Be); }
}

void use_union(OlsArgs& a, const UnionMoments& U)
{
    a.Gt = U.Gt.as<double>(); a.Bt = U.Bt.as<double>();
    a.Ge = U.Ge.ptr ? U.Ge.as<double>() : nullptr;
    a.Be = U.Be.ptr ? U.Be.as<double>() : nullptr;
    a.upos = U.pos.as<int32_t>(); a.ucols = U.cols.as<int32_t>(); a.pu = U.pu;
}

}  // namespace

int64_t ols_losses(const double* Gt, const double* Bt, const double* Ge, const double* Be,
                const double* yye, const uint64_t* family, int64_t p, int64_t r, int32_t q,
                int32_t B2, double* losses, int32_t* singular, cudaStream_t s)
{
    UnionMoments U;
    restrict_to_union(family, p, r, q, B2, Gt, Bt, Ge, Be, U, s);
    OlsArgs a{};
    use_union(a, U);
    a.yye = yye; a.family = family;
    a.p = p; a.r = r; a.q = q; a.B2 = B2; a.W = (int32_t)((p + 63) / 64);
    a.losses = losses; a.singular = singular;
    a.solves = (int64_t)B2 * q * r;
    DevBuf dup(sizeof(int32_t) * (size_t)(q * r), s);
    const unsigned gd = (unsigned)std::min<int64_t>(ceil_div((int64_t)q * r, 256), 1024);
    k_family_dedup<<<gd, 256, 0, s>>>(family, q, r, a.W, dup.as<int32_t>());
    UOI_CHECK_LAUNCH();
    a.dup = dup.as<int32_t>();
    // Size classes: small supports run with little shared memory per CTA (many
    // CTAs per SM hide the latency of their short dependent steps); large ones
    // with room for their factor.  Only first occurrences of a support are listed.
    const int64_t qr = (int64_t)q * r;
    DevBuf sizes(sizeof(int32_t) * (size_t)qr, s);
    k_support_sizes<<<(unsigned)std::min<int64_t>(ceil_div(qr, 256), 1024), 256, 0, s>>>(
        family, qr, a.W, sizes.as<int32_t>());
    UOI_CHECK_LAUNCH();
    count_launch();
    std::vector<int32_t> hsz((size_t)qr), hdup((size_t)qr);
    UOI_CUDA(cudaMemcpyAsync(hsz.data(), sizes.ptr, sizeof(int32_t) * qr, cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaMemcpyAsync(hdup.data(), dup.ptr, sizeof(int32_t) * qr, cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> small_je, large_je;
    int32_t smax_small = 1, smax_large = 1;
    for (int64_t t = 0; t < qr; ++t) {
        if (hdup[t] != (int32_t)(t / r)) continue;
        if (hsz[t] <= OLS_SMALL) { small_je.push_back((int32_t)t); smax_small = std::max(smax_small, hsz[t]); }
        else { large_je.push_back((int32_t)t); smax_large = std::max(smax_large, hsz[t]); }
    }
    if (std::max(smax_small, smax_large) > 46000)
        throw Error(UOI_ERR_UNSUPPORTED, "OLS support larger than 46000 columns");
    int64_t nfb = 0;
    // largest supports first within each class, taken from a counter as CTAs free up
    // (the factor costs grow as the cube of the support size)
    auto by_size = [&](int32_t x, int32_t y) { return hsz[(size_t)x] > hsz[(size_t)y]; };
    std::stable_sort(small_je.begin(), small_je.end(), by_size);
    std::stable_sort(large_je.begin(), large_je.end(), by_size);
    DevBuf ctr(sizeof(unsigned long long) * 2, s);
    UOI_CUDA(cudaMemsetAsync(ctr.ptr, 0, ctr.bytes, s));
    // the two classes run side by side: the large class on s, the small one on a
    // second stream that starts after everything s has queued so far
    cudaStream_t side = (small_je.empty() || large_je.empty()) ? s : side_stream();
    cudaEvent_t ready = nullptr, side_done = nullptr;
    if (side != s) {
        UOI_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        UOI_CUDA(cudaEventCreateWithFlags(&side_done, cudaEventDisableTiming));
        UOI_CUDA(cudaEventRecord(ready, s));
        UOI_CUDA(cudaStreamWaitEvent(side, ready, 0));
    }
    OlsMixedRun runs[2];
    DevBuf jl[2];
    for (int cls = 0; cls < 2; ++cls) {
        const std::vector<int32_t>& lst = cls == 0 ? small_je : large_je;
        if (lst.empty()) continue;
        cudaStream_t cs = cls == 0 ? side : s;
        jl[cls].alloc(sizeof(int32_t) * lst.size(), cs);
        UOI_CUDA(cudaMemcpyAsync(jl[cls].ptr, lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice, cs));
        OlsArgs b = a;
        b.je_list = jl[cls].as<int32_t>();
        b.n_je = (int32_t)lst.size();
        b.next = ctr.as<unsigned long long>() + cls;
        b.solves = (int64_t)B2 * b.n_je;
        b.smax = cls == 0 ? smax_small : smax_large;
        ols_mixed_start(b, cs, runs[cls]);
    }
    for (int cls = 1; cls >= 0; --cls) nfb += ols_mixed_finish(runs[cls], cls == 0 ? side : s);
    if (side != s) {
        // everything that follows on s (the duplicates' losses, the argmin) sees the side's results
        UOI_CUDA(cudaEventRecord(side_done, side));
        UOI_CUDA(cudaStreamWaitEvent(s, side_done, 0));
        cudaEventDestroy(ready);
        cudaEventDestroy(side_done);
    }
    const unsigned gf = (unsigned)std::min<int64_t>(ceil_div(a.solves, 256), 4096);
    k_fill_duplicates<<<gf, 256, 0, s>>>(dup.as<int32_t>(), B2, q, r, losses, singular);
    UOI_CHECK_LAUNCH();
    count_launch(2);
    return nfb;
}

void loss_argmin(const double* losses, int32_t B2, int32_t q, int64_t r, int32_t* jstar,
                 cudaStream_t s)
{
    k_argmin<<<B2, 32, 0, s>>>(losses, q, r, jstar);
    UOI_CHECK_LAUNCH();
    count_launch();
}

int64_t ols_chosen(const double* Gt, const double* Bt, const uint64_t* family, const int32_t* jstar,
                int64_t p, int64_t r, int32_t q, int32_t B2, double* chosen, cudaStream_t s)
{
    UOI_CUDA(cudaMemsetAsync(chosen, 0, sizeof(double) * (size_t)(B2 * r * p), s));
    UnionMoments U;
    restrict_to_union(family, p, r, q, B2, Gt, Bt, nullptr, nullptr, U, s);
    OlsArgs a{};
    use_union(a, U);
    a.family = family;
    a.p = p; a.r = r; a.q = q; a.B2 = B2; a.W = (int32_t)((p + 63) / 64);
    a.jstar = jstar; a.chosen = chosen;
    a.solves = (int64_t)B2 * r;
    return run_ols(a, s);
}

void bagging(const double* chosen, int32_t B2, int64_t count, int32_t mode, double* out,
             cudaStream_t s)
{
    k_bagging<<<(unsigned)std::min<int64_t>(ceil_div(count, 128), 4096), 128, 0, s>>>(
        chosen, B2, count, mode, out);
    UOI_CHECK_LAUNCH();
    count_launch();
}

}  // namespace uoi
