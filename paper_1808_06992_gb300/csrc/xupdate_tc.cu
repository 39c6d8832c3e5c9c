// xupdate_tc.cu -- G4 on the tensor cores: the ADMM x-update of the mixed form
// (x = c + rho M (z - u), Eq. 5 with the cached inverse) as tcgen05 products,
// with the soft threshold, dual update and residual norms fused into the
// epilogue.
//
// Accuracy: M and V = z - u are each scaled by an exact power of two and split
// into two fp16 pieces (v = h + l, residue <= 2^-22 |v|); the three products
// h.H, h.L, l.H are summed (the dropped l.L is below 2^-22).  The scale keeps
// every scaled value below 2^10, far from fp16's overflow, and puts the
// underflow floor at 2^-34 of the largest value: each row of M gets its own
// scale (from its largest entry, M is fixed for the solve), each chain of V one
// from a bound on ||V|| that holds for every ADMM step:
//   V' = 2 z' - v with v = x' + u and |z'| <= |v|, x' = c + rho M V, rho ||M|| <= 1
//   => ||V'|| <= 3 (||c|| + ||z|| + 2 ||u||),
// evaluated from the norms of the previous step (times 2 for rounding).  The
// large h.H products go to a double-buffered TMEM accumulator that the epilogue
// drains every 128 k into compensated FP32 pairs (the tensor core's FP32
// accumulation truncates about a third of an ulp per K=16 step); the two small
// products, 2^-11 smaller, share one accumulator read once at the end.  The
// x-update is then accurate to a few 1e-7 relative.  Once the products are done
// the folded sums go back to TMEM beside them, so that the update runs as a
// rolled loop over groups of 8 chains (one copy of its code in the instruction
// cache) reading 8 columns of each per pass.
//
// Work per launch: every chain of every group (converged chains are skipped in
// the epilogue and keep their state; tiles with no live chain exit at once).
// Grid: (row tiles of 128, chain tiles of NT <= 64, groups), two CTAs per SM so
// that one CTA's prologue and epilogue overlap the other's stream of M.  Warp 0:
// TMA producer (ring of 4 stages of k = 32); warp 1: TMEM allocation and MMA
// issue; warps 2-5: epilogue (one TMEM lane quarter each).
// Waits are bounded (~1 s) and report UOI_ERR_TIMEOUT.
#include <cuda_fp16.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "tc_common.cuh"

namespace uoi {

namespace {
using namespace tc;

constexpr int XT_TM = 128;
constexpr int XT_TK = 32;                              // k per stage (64-byte swizzled rows)
constexpr int XT_NT_MAX = 64;
constexpr int XT_PIECES = 2;                           // fp16 pieces of M and of V
constexpr int XT_STAGES = 4;                           // ring slots
constexpr int XT_A_BYTES = XT_TM * XT_TK * 2;          // 8 KB per piece
constexpr int XT_STAGE_MAX = XT_PIECES * XT_A_BYTES + XT_PIECES * XT_NT_MAX * XT_TK * 2;   // 24 KB
constexpr int XT_SMEM = XT_STAGES * XT_STAGE_MAX + 1024;
constexpr int XT_THREADS = 192;
constexpr uint32_t XT_TMEM_COLS = 256;                 // A1[0] at 0, A1[1] at 64, A2 at 128
constexpr int XT_CHUNK_STAGES = 4;                     // drain h.H every 128 k
constexpr int XT_SCALE_EXP = 10;                       // scaled magnitudes stay below 2^10

struct XtArgs {
    int32_t G, q, r, p, nchains, NT, kst, RT, warm;
    int64_t ppad;                 // rows per group (multiple of 128)
    int64_t kpad;                 // k extent (multiple of 32)
    int64_t slots;
    const float* c;               // G x r x p
    const double* lambdas;
    float rho;
    float* z; float* u;           // slots x p
    __half* vnext;                // 2 x slots x kpad
    const float* row_inv;         // G x ppad: 1 / scale of the row of M
    const float* vs_r;            // slots: scale of the V pieces read
    const float* vs_w;            // slots: scale for the V pieces written
    const int32_t* slot_j;
    const uint8_t* live;
    float* norms;                 // slots x RT x 5
    int32_t* err;
    const int32_t* tiles;         // live (group, chain tile) list, or null: grid y, z = tile, group
    const int32_t* ntiles;        // entries of the list in use
    int32_t nct;                  // chain tiles per group
    uint64_t wait_ns = tc::kWaitLimitNs;   // limit of every bounded mbarrier wait
};

// 4-byte asynchronous copy global -> shared (completion waited for by the issuing thread).
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void split2(float x, __half& h, __half& l)
{
    h = __float2half_rn(x);
    l = __float2half_rn(x - __half2float(h));
}

// 2^(XT_SCALE_EXP - e) for bound = f 2^e, f in [0.5, 1): bound * scale < 2^XT_SCALE_EXP.
__device__ __forceinline__ float pow2_scale(float bound)
{
    if (!(bound > 0.f) || !(bound < 3.0e38f)) return 1.f;
    int e;
    frexpf(bound, &e);
    return ldexpf(1.f, min(120, max(-120, XT_SCALE_EXP - e)));
}

// One CTA of the x-update: row tile rt, chain tile ct of group g, with a ring of
// STAGES slots (at least 4: the epilogue stages z, u and c in the idle ring).
template <int STAGES>
__device__ __forceinline__ void xupdate_tile(const CUtensorMap* tmM, const CUtensorMap* tmV, const XtArgs& a,
                                             int rt, int ct, int g)
{
    static_assert(3 * XT_NT_MAX * XT_TM * 4 <= STAGES * XT_STAGE_MAX, "epilogue staging fits the ring");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ float red[4][XT_NT_MAX][5];
    __shared__ float s_kappa[XT_NT_MAX];           // lambda_j / rho of each chain of the tile
    __shared__ float s_vrinv[XT_NT_MAX];           // 1 / scale of the chain's V pieces read
    __shared__ float s_vw[XT_NT_MAX];              // scale of the chain's V pieces written
    __shared__ int s_coff[XT_NT_MAX];              // row of c used by the chain
    __shared__ uint8_t s_live[XT_NT_MAX];          // chain exists and is still iterating

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = rt * XT_TM, n0 = ct * a.NT;
    const int nchunks = (a.kst + XT_CHUNK_STAGES - 1) / XT_CHUNK_STAGES;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t b_bytes = (uint32_t)a.NT * XT_TK * 2;
    const uint32_t stage_tx = XT_PIECES * XT_A_BYTES + XT_PIECES * b_bytes;
    const uint32_t stage_bytes = (stage_tx + 1023u) & ~1023u;
    const int nst = STAGES;

    // A tile whose chains have all stopped has nothing to update: skip it whole.
    // (Only the live flags are read before the pipeline starts; the epilogue
    // warps read the other per-chain scalars while M streams in.)
    {
        const int n = threadIdx.x, chain = n0 + n;
        const int64_t sl = (int64_t)g * a.nchains + chain;
        const bool mine = n < a.NT && chain < a.nchains && a.live[sl];
        if (n < XT_NT_MAX) s_live[n] = mine ? 1 : 0;
        if (!__syncthreads_or(mine)) return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&accf_bar[b], 1); mbar_init(&acce_bar[b], 128); }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(XT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        const int blkA = ((g * a.RT + rt) * a.kst) * XT_PIECES;   // first 8 KB block of this row tile
        const int rowB = g * a.nchains + n0;
        for (int s_ = 0; s_ < a.kst; ++s_) {
            const int s = s_ % nst;
            if (s_ >= nst && !mbar_wait(&empty_bar[s], ((s_ / nst) - 1) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            const uint32_t st = sbase + s * stage_bytes;
            mbar_expect_tx(&full_bar[s], stage_tx);
            const int k0 = s_ * XT_TK;
            tma_load_3d(st, tmM, &full_bar[s], 0, 0, blkA + XT_PIECES * s_);    // 2 pieces, 16 KB contiguous
            for (int pc = 0; pc < XT_PIECES; ++pc)
                tma_load_3d(st + XT_PIECES * XT_A_BYTES + pc * b_bytes, tmV, &full_bar[s], k0, rowB, pc);
        }
        if (abort_flag)
            for (int s_ = max(0, a.kst - nst); s_ < a.kst; ++s_)
                mbar_wait(&full_bar[s_ % nst], (s_ / nst) & 1, &abort_flag, a.wait_ns);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = idesc_f16(XT_TM, a.NT);
        const uint32_t d2 = tmem + 128u;
        bool first2 = true;
        int s_ = 0;
        for (int c = 0; c < nchunks && !abort_flag; ++c) {
            const int b = c & 1;
            if (c >= 2 && !mbar_wait(&acce_bar[b], ((c >> 1) - 1) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t d1 = tmem + (uint32_t)(b * 64);
            const int send = min(a.kst, (c + 1) * XT_CHUNK_STAGES);
            bool first1 = true;
            for (; s_ < send; ++s_) {
                const int s = s_ % nst;
                if (!mbar_wait(&full_bar[s], (s_ / nst) & 1, &abort_flag, a.wait_ns)) {
                    abort_flag = 1;
                    atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t st = sbase + s * stage_bytes;
                const uint64_t Ah = smem_desc_sw64(st), Al = smem_desc_sw64(st + XT_A_BYTES);
                const uint32_t bb = st + XT_PIECES * XT_A_BYTES;
                const uint64_t Bh = smem_desc_sw64(bb), Bl = smem_desc_sw64(bb + b_bytes);
#pragma unroll
                for (int ks = 0; ks < XT_TK / 16; ++ks) {
                    const uint64_t adv = (uint64_t)(ks * 32 >> 4);
                    mma_bf16(d1, Ah + adv, Bh + adv, idesc, first1 ? 0u : 1u);
                    mma_bf16(d2, Ah + adv, Bl + adv, idesc, first2 ? 0u : 1u);
                    mma_bf16(d2, Al + adv, Bh + adv, idesc, 1u);
                    first1 = false;
                    first2 = false;
                }
                mma_commit(&empty_bar[s]);
            }
            if (abort_flag) break;
            mma_commit(&accf_bar[b]);
        }
        mma_commit(&done_bar);
        int dummy = 0;
        mbar_wait(&done_bar, 0, &dummy, a.wait_ns);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int quad = warp & 3;
        const int i = i0 + quad * 32 + lane;
        const uint32_t lanes = (uint32_t)(quad * 32) << 16;
        {
            // per-chain scalars of the update, read once instead of per row, while the
            // products run; then a barrier of the four epilogue warps
            const int n = threadIdx.x - 64;
            if (n < XT_NT_MAX) {
                const int chain = n0 + n;
                const int64_t sl = (int64_t)g * a.nchains + chain;
                const bool mine = s_live[n] != 0;
                s_kappa[n] = mine ? (float)a.lambdas[a.slot_j[sl]] / a.rho : 0.f;
                s_vrinv[n] = mine ? 1.f / a.vs_r[sl] : 0.f;
                s_vw[n] = mine ? a.vs_w[sl] : 0.f;
                s_coff[n] = g * a.r + (a.warm ? chain : chain % a.r);
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
        }
        const float rinv_row = i < a.p ? a.row_inv[(int64_t)g * a.ppad + i] : 0.f;
        float acc[64], cmp[64];
#pragma unroll
        for (int t = 0; t < 64; ++t) { acc[t] = 0.f; cmp[t] = 0.f; }
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            const bool okw = mbar_wait(&accf_bar[b], (c >> 1) & 1, &abort_flag, a.wait_ns);
            if (!__all_sync(0xffffffffu, okw)) {               // warp-uniform exit
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                if (cb * 32 >= a.NT) break;
                float v[32];
                tmem_ld32(tmem + lanes + (uint32_t)(b * 64 + cb * 32), v);
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const float x = v[t], sa = acc[cb * 32 + t];
                    const float sum = sa + x;
                    const float bv = sum - sa;
                    cmp[cb * 32 + t] += (sa - (sum - bv)) + (x - bv);
                    acc[cb * 32 + t] = sum;
                }
            }
            tc_fence_before();
            mbar_arrive(&acce_bar[b]);
        }
        // fold the compensation terms (frees their registers for the epilogue)
#pragma unroll
        for (int t = 0; t < 64; ++t) acc[t] += cmp[t];
        // small products, once all MMAs are done
        {
            int dummy = 0;
            if (!abort_flag) mbar_wait(&done_bar, 0, &dummy, a.wait_ns);
        }
        __syncwarp();
        tc_fence_after();
        const bool rowok = i < a.p && !abort_flag;
        const float rinv = rowok ? rinv_row : 0.f;
        // The ring is idle now: stage this row's z, u and c of every live chain in
        // it with asynchronous copies, all in flight at once, so the update below
        // reads shared memory instead of waiting on DRAM once per group of chains.
        // Each thread copies (and later reads) only its own row: no barrier needed.
        float* stg = reinterpret_cast<float*>(smem_raw + (sbase - smem_u32(smem_raw)));   // [3][NT][128]
        const int r128 = quad * 32 + lane;
        if (rowok) {
            for (int n = 0; n < a.NT; ++n) {
                if (!s_live[n]) continue;
                const int64_t o = ((int64_t)g * a.nchains + n0 + n) * a.p + i;
                cp_async4(smem_u32(stg + (0 * a.NT + n) * XT_TM + r128), a.z + o);
                cp_async4(smem_u32(stg + (1 * a.NT + n) * XT_TM + r128), a.u + o);
                cp_async4(smem_u32(stg + (2 * a.NT + n) * XT_TM + r128), a.c + (int64_t)s_coff[n] * a.p + i);
            }
        }
        // The folded sums go back to TMEM, into the first drain buffer (columns
        // 0..NT-1, idle once all products are done), so that the update below is a
        // rolled loop over groups of 8 chains with one copy of its body: each pass
        // reads 8 columns of h.H and of the small products.
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            if (cb * 32 >= a.NT) break;
            float w[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) w[t] = acc[cb * 32 + t];
            tmem_st32(tmem + lanes + (uint32_t)(cb * 32), w);
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
#pragma unroll 1
        for (int nb = 0; nb < a.NT; nb += 8) {                       // first chain of the group of 8
            float hv[8];                                             // h.H + small products
            {
                float hh[8], v2[8];
                tmem_ld8x2(tmem + lanes + (uint32_t)nb, tmem + lanes + (uint32_t)(128 + nb), hh, v2);
#pragma unroll
                for (int t = 0; t < 8; ++t) hv[t] = hh[t] + v2[t];
            }
            {
                float zp[8], uo[8], cc[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const bool act = rowok && s_live[nb + t];
                    zp[t] = act ? stg[(0 * a.NT + nb + t) * XT_TM + r128] : 0.f;
                    uo[t] = act ? stg[(1 * a.NT + nb + t) * XT_TM + r128] : 0.f;
                    cc[t] = act ? stg[(2 * a.NT + nb + t) * XT_TM + r128] : 0.f;
                }
                float pr[5][8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
#pragma unroll
                    for (int qq = 0; qq < 5; ++qq) pr[qq][t] = 0.f;
                    if (!(rowok && s_live[nb + t])) continue;
                    const int tt = nb + t;
                    const float prod = hv[t] * (rinv * s_vrinv[tt]);
                    const float x = cc[t] + a.rho * prod;
                    const int64_t sl = (int64_t)g * a.nchains + n0 + nb + t;
                    const int64_t o = sl * a.p + i;
                    const float vv = x + uo[t];
                    const float zn = soft_threshold(vv, s_kappa[nb + t]);
                    const float un = vv - zn;
                    if (UOI_IN_BOUNDS(o, a.slots * a.p, 302)) {
                        a.z[o] = zn;
                        a.u[o] = un;
                    }
                    __half h, l;
                    split2((zn - un) * s_vw[tt], h, l);
                    const int64_t vo = sl * a.kpad + i;
                    if (UOI_IN_BOUNDS(vo, a.slots * a.kpad, 303)) {
                        a.vnext[vo] = h;
                        a.vnext[(int64_t)a.slots * a.kpad + vo] = l;
                    }
                    const float d = x - zn, dz = zn - zp[t];
                    pr[0][t] = d * d; pr[1][t] = dz * dz; pr[2][t] = x * x; pr[3][t] = zn * zn; pr[4][t] = un * un;
                }
                // column sums over the warp's 32 rows: halve the 8 columns per lane at
                // lane bits 4, 3, 2, then add across bits 1, 0 (fixed order)
                const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
#pragma unroll
                for (int qq = 0; qq < 5; ++qq) {
                    float w4[4], w3[2];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float send = b4 ? pr[qq][j] : pr[qq][j + 4];
                        const float keep = b4 ? pr[qq][j + 4] : pr[qq][j];
                        w4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float send = b3 ? w4[j] : w4[j + 2];
                        const float keep = b3 ? w4[j + 2] : w4[j];
                        w3[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
                    float w2 = (b2 ? w3[1] : w3[0]) + __shfl_xor_sync(0xffffffffu, b2 ? w3[0] : w3[1], 4);
                    w2 += __shfl_xor_sync(0xffffffffu, w2, 2);
                    w2 += __shfl_xor_sync(0xffffffffu, w2, 1);
                    if ((lane & 3) == 0) red[quad][nb + b4 * 4 + b3 * 2 + b2][qq] = w2;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // norms of this row tile: sum of the four row quarters in a fixed order
    if (threadIdx.x < XT_NT_MAX) {
        const int n = threadIdx.x;
        if (n < a.NT && s_live[n]) {
            const int64_t sl = (int64_t)g * a.nchains + n0 + n;
#pragma unroll
            for (int qq = 0; qq < 5; ++qq) {
                const float tot = ((red[0][n][qq] + red[1][n][qq]) + red[2][n][qq]) + red[3][n][qq];
                a.norms[(sl * a.RT + rt) * 5 + qq] = tot;
            }
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(XT_TMEM_COLS));
    }
}

// One problem: grid (row tiles, chain tiles, groups), or (row tiles, entries of
// the live tile list) when a.tiles is set.
__global__ void __launch_bounds__(XT_THREADS, 2)
k_xupdate_tc(const __grid_constant__ CUtensorMap tmM, const __grid_constant__ CUtensorMap tmV,
             XtArgs a)
{
    int ct = blockIdx.y, g = blockIdx.z;
    if (a.tiles) {                                     // only the tiles with a live chain
        if ((int)blockIdx.y >= *a.ntiles) return;
        const int tl = a.tiles[blockIdx.y];
        g = tl / a.nct;
        ct = tl % a.nct;
    }
    xupdate_tile<XT_STAGES>(&tmM, &tmV, a, (int)blockIdx.x, ct, g);
}

// Two fp16 pieces of 8 consecutive scaled values of row i of M_g, stored as 16 bytes
// per piece at column k8 of the [g][row tile][k block][piece][128][32] block order.
__device__ __forceinline__ void store_m_pieces8(const float (&x)[8], int64_t g, int64_t i, int64_t k8,
                                                int64_t RT, int64_t kst, __half* out)
{
    uint32_t ph[4], pl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __half h[2], l[2];
        split2(x[2 * q], h[0], l[0]);
        split2(x[2 * q + 1], h[1], l[1]);
        ph[q] = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
        pl[q] = (uint32_t)__half_as_ushort(l[0]) | ((uint32_t)__half_as_ushort(l[1]) << 16);
    }
    const int64_t blk = ((g * RT + i / XT_TM) * kst + k8 / XT_TK) * XT_PIECES;
    const int64_t o = (blk * XT_TM + i % XT_TM) * XT_TK + k8 % XT_TK;    // multiple of 8: 16 B aligned
    *reinterpret_cast<uint4*>(out + o) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
    *reinterpret_cast<uint4*>(out + o + XT_TM * XT_TK) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
}

// M_g (FP32, p x p) -> per-row scales and the two fp16 pieces of each row times its
// scale, one warp per row.  row_scale = 2^(10 - e) for the row's largest |M_ik| =
// f 2^e (1 for an all-zero or padding row), row_inv = 1 / row_scale.  The pieces go
// to 128 x 32 blocks ordered [g][row tile][k block][piece][128][32] (zero padded), so
// that the x-update streams each row tile as one contiguous run of 16 KB stages.
// Each lane takes 8 consecutive k at a time and writes 16 bytes per piece.  Rows of
// up to 256 x SSM_REG_GROUPS columns stay in registers between the maximum and the
// split; longer rows are read twice (the second time from L2).
constexpr int SSM_REG_GROUPS = 8;
__global__ void k_scale_split_m(const float* M, int32_t G, int64_t p, int64_t ppad, int64_t kpad,
                                float* row_scale, float* row_inv, __half* out)
{
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= (int64_t)G * ppad) return;
    const int64_t g = row / ppad, i = row % ppad;
    const bool real = i < p;
    const float* mr = M + ((size_t)g * p + (real ? i : 0)) * p;
    const int64_t RT = ppad / XT_TM, kst = kpad / XT_TK;
    float mx = 0.f;
    if (kpad <= 256 * SSM_REG_GROUPS) {
        float v[SSM_REG_GROUPS][8];
#pragma unroll
        for (int q = 0; q < SSM_REG_GROUPS; ++q) {
            const int64_t k8 = (int64_t)lane * 8 + 256 * q;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[q][u] = (real && k8 + u < p) ? mr[k8 + u] : 0.f;
                mx = fmaxf(mx, fabsf(v[q][u]));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = pow2_scale(mx);
        if (lane == 0) {
            row_scale[row] = sc;
            row_inv[row] = 1.f / sc;
        }
#pragma unroll
        for (int q = 0; q < SSM_REG_GROUPS; ++q) {
            const int64_t k8 = (int64_t)lane * 8 + 256 * q;
            if (k8 >= kpad) break;
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = (real && k8 + u < p) ? v[q][u] * sc : 0.f;
            store_m_pieces8(x, g, i, k8, RT, kst, out);
        }
        return;
    }
    if (real)
        for (int64_t k = lane; k < p; k += 32) mx = fmaxf(mx, fabsf(mr[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float sc = pow2_scale(mx);
    if (lane == 0) {
        row_scale[row] = sc;
        row_inv[row] = 1.f / sc;
    }
    for (int64_t k8 = (int64_t)lane * 8; k8 < kpad; k8 += 256) {
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = (real && k8 + u < p) ? mr[k8 + u] * sc : 0.f;
        store_m_pieces8(x, g, i, k8, RT, kst, out);
    }
}

// Per (group, equation): ||c_ge||_2 (one warp each).
__global__ void k_c_norms(const float* c, int64_t count, int64_t p, float* cn)
{
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= count) return;
    float acc = 0.f;
    for (int64_t i = lane; i < p; i += 32) {
        const float v = c[row * p + i];
        acc += v * v;
    }
    acc = warp_sum(acc);
    if (lane == 0) cn[row] = sqrtf(acc);
}

// Scales of the first two V buffers of every slot (one warp each): vs0 for
// V_0 = z0 - u0 from its largest entry, vs1 for V_1 (written by the first
// x-update) from the step bound 2 * 3 (||c|| + ||z0|| + 2 ||u0||).
__global__ void k_xt_vscale_init(int64_t slots, int64_t p, int32_t nchains, int32_t r, int32_t warm,
                                 const float* z0, const float* u0, const float* cn, float* vs0,
                                 float* vs1)
{
    const int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sl >= slots) return;
    float mx = 0.f, zz = 0.f, uu = 0.f;
    if (z0)
        for (int64_t i = lane; i < p; i += 32) {
            const float zi = z0[sl * p + i], ui = u0[sl * p + i];
            mx = fmaxf(mx, fabsf(zi - ui));
            zz += zi * zi;
            uu += ui * ui;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    zz = warp_sum(zz);
    uu = warp_sum(uu);
    if (lane == 0) {
        const int64_t g = sl / nchains, chain = sl % nchains;
        const float cnorm = cn[g * r + (warm ? chain : chain % r)];
        vs0[sl] = pow2_scale(mx);
        vs1[sl] = pow2_scale(6.f * (cnorm + sqrtf(zz) + 2.f * sqrtf(uu)));
    }
}

// Initial state: z, u (zero or the given start), the pieces of V = z - u
// (scaled by vs0), live flags.
__global__ void k_xt_init(int64_t slots, int64_t p, int64_t kpad, const float* z0, const float* u0,
                          const float* vs0, float* z, float* u, __half* v, uint8_t* live)
{
    const int64_t total = slots * kpad;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = t / kpad, i = t % kpad;
        float zz = 0.f, uu = 0.f;
        if (i < p) {
            if (z0) { zz = z0[sl * p + i]; uu = u0[sl * p + i]; }
            z[sl * p + i] = zz;
            u[sl * p + i] = uu;
        }
        __half h, l;
        split2((zz - uu) * vs0[sl], h, l);
        v[t] = h;
        v[slots * kpad + t] = l;
        if (i == 0) live[sl] = 1;
    }
}

// Convergence check of every live slot (one warp each): fixed-order sum of the
// row-tile norms, stopping test of Eq. 5's ADMM, output of finished columns,
// path advance, live count for the host.
struct XtCheck {
    int32_t G, q, r, p, nchains, RT, warm, max_iter;
    float rho, abs_tol, rel_tol, sqrtp;
    const float* z;
    const float* norms;
    int32_t* slot_j;
    const int32_t* slot_jend;
    int32_t* slot_it;
    uint8_t* live;
    double* beta;
    int32_t* iters;
    uint8_t* conv;
    uint64_t* family;
    int32_t W;
    int32_t* live_count;          // incremented once per slot still iterating
    const float* cn;
    float* vs_next;
    const float* u;
    const double* lambdas;
    unsigned long long* near_count;
};

// Slot sl of one problem, by one warp.
__device__ __forceinline__ void xt_check_slot(const XtCheck& ca, int64_t sl, int lane)
{
    const int32_t G = ca.G, q = ca.q, r = ca.r, p = ca.p, nchains = ca.nchains, RT = ca.RT, warm = ca.warm,
                  max_iter = ca.max_iter, W = ca.W;
    const float rho = ca.rho, abs_tol = ca.abs_tol, rel_tol = ca.rel_tol, sqrtp = ca.sqrtp;
    const float* z = ca.z;
    const float* norms = ca.norms;
    int32_t* slot_j = ca.slot_j;
    const int32_t* slot_jend = ca.slot_jend;
    int32_t* slot_it = ca.slot_it;
    uint8_t* live = ca.live;
    double* beta = ca.beta;
    int32_t* iters = ca.iters;
    uint8_t* conv = ca.conv;
    uint64_t* family = ca.family;
    int32_t* live_count = ca.live_count;
    const float* cn = ca.cn;
    float* vs_next = ca.vs_next;
    const float* u = ca.u;
    const double* lambdas = ca.lambdas;
    unsigned long long* near_count = ca.near_count;
    if (sl >= (int64_t)G * nchains || !live[sl]) return;
    float tot[5] = { 0.f, 0.f, 0.f, 0.f, 0.f };
    for (int t0 = 0; t0 < RT; t0 += 32) {
        float loc[5] = { 0.f, 0.f, 0.f, 0.f, 0.f };
        if (t0 + lane < RT)
#pragma unroll
            for (int c = 0; c < 5; ++c) loc[c] = norms[(sl * RT + t0 + lane) * 5 + c];
#pragma unroll
        for (int c = 0; c < 5; ++c) tot[c] += warp_sum(loc[c]);
    }
    int it = slot_it[sl] + 1;
    const float xn = sqrtf(tot[2]), zn = sqrtf(tot[3]);
    const float eps_pri = sqrtp * abs_tol + rel_tol * fmaxf(xn, zn);
    const float eps_dual = sqrtp * abs_tol + rel_tol * rho * sqrtf(tot[4]);
    const bool converged = sqrtf(tot[0]) <= eps_pri && rho * sqrtf(tot[1]) <= eps_dual;
    bool still = true;
    if (converged || it >= max_iter) {
        const int g = (int)(sl / nchains), cid = (int)(sl % nchains);
        const int e = warm ? cid : cid % r;
        const int j = slot_j[sl];
        const int64_t col_je = (int64_t)j * r + e;
        const int64_t col = (int64_t)g * q * r + col_je;
        // threshold lambda_j / rho, once per column (FP64 division off the loop)
        const float kappa = near_count ? (float)(lambdas[j] / (double)rho) : 0.f;
        // eight 32-feature chunks of z and u loaded before their ballots, so the
        // loads of a finishing column overlap instead of queueing behind the atomics
        for (int b0 = 0; 32 * b0 < p; b0 += 8) {
            float zc[8], uc[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int i = lane + 32 * (b0 + t);
                zc[t] = i < p ? z[sl * p + i] : 0.f;
                uc[t] = (near_count && i < p) ? u[sl * p + i] : 0.f;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int a0 = b0 + t;
                if (32 * a0 >= p) break;                         // warp-uniform
                const int i = lane + 32 * a0;
                const float zi = zc[t];
                if (beta && i < p && UOI_IN_BOUNDS(col * p + i, (int64_t)G * q * r * p, 301))
                    beta[col * p + i] = (double)zi;
                if (family) {
                    const unsigned bal = __ballot_sync(0xffffffffu, zi != 0.f);
                    if (lane == 0) {
                        const int shift = (a0 & 1) * 32;
                        const uint64_t mask = ((uint64_t)bal << shift) | ~(0xFFFFFFFFull << shift);
                        atomicAnd((unsigned long long*)&family[col_je * W + (a0 >> 1)],
                                  (unsigned long long)mask);
                    }
                }
                if (near_count)
                    count_near_threshold<float>(i < p, zi, uc[t], kappa, (float)kNearThreshold, near_count);
            }
        }
        if (lane == 0) {
            if (iters) iters[col] = it;
            if (conv) conv[col] = converged ? 1 : 0;
        }
        if (j + 1 < slot_jend[sl]) {
            if (lane == 0) slot_j[sl] = j + 1;
            it = 0;
        } else {
            still = false;
        }
    }
    if (lane == 0) {
        slot_it[sl] = it;
        if (!still) {
            live[sl] = 0;
        } else {
            atomicAdd(live_count, 1);
            // scale of the V pieces the next x-update writes: step bound on ||V||
            const int64_t g = sl / nchains, chain = sl % nchains;
            const float cnorm = cn[g * r + (warm ? chain : chain % r)];
            vs_next[sl] = pow2_scale(6.f * (cnorm + zn + 2.f * sqrtf(tot[4])));
        }
    }
}

__global__ void k_xt_check(XtCheck ca)
{
    xt_check_slot(ca, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31);
}

// ---- grouped form: many problems' solves in the same launches ----------------------
//
// A batch of independent problems (different p, groups, right-hand sides) iterates
// together: each step is one x-update launch over the live (problem, group, row
// tile, chain tile) items of every problem and one check launch over the live
// chain tiles of every problem.  A problem's tensor maps and arguments sit in a
// device table (XtMemberDev) that the kernels index by the item's problem; the
// arithmetic of an item is the single-problem kernel's, so each problem's iterates
// are those of its own solve.

struct XtItem {
    int32_t member, g, rt, ct;
};

struct __align__(64) XtMemberDev {
    CUtensorMap mM;               // the problem's split inverse
    CUtensorMap mV[2];            // V pieces read on even / odd steps
    XtArgs args[2];               // x-update arguments of even / odd steps
    XtCheck check[2];             // check arguments after even / odd steps
};

template <int STAGES>
__global__ void __launch_bounds__(XT_THREADS, STAGES <= 4 ? 2 : 1)
k_xupdate_tc_grouped(const XtMemberDev* mem, const XtItem* items, const int32_t* nitems, int32_t parity)
{
    if ((int)blockIdx.x >= *nitems) return;
    const XtItem it = items[blockIdx.x];
    const XtMemberDev& m = mem[it.member];
    // the arguments in shared memory: read there, they cannot alias the tile's stores
    __shared__ XtArgs sa;
    if (threadIdx.x == 0) sa = m.args[parity];
    __syncthreads();
    xupdate_tile<STAGES>(&m.mM, &m.mV[parity], sa, it.rt, it.ct, it.g);
}

constexpr int XT_CHECK_WARPS = 16;

// One block per live chain tile (an item with rt = 0 stands for its tile); warp w
// checks the tile's chains w, w + 16, ...
__global__ void __launch_bounds__(32 * XT_CHECK_WARPS)
k_xt_check_tiles(const XtMemberDev* mem, const XtItem* tiles, const int32_t* ntiles, int32_t parity)
{
    if ((int)blockIdx.x >= *ntiles) return;
    const XtItem t = tiles[blockIdx.x];
    const XtMemberDev& m = mem[t.member];
    const int NT = m.args[0].NT, nchains = m.args[0].nchains;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < NT; c += XT_CHECK_WARPS) {
        const int chain = t.ct * NT + c;
        if (chain >= nchains) break;
        xt_check_slot(m.check[parity], (int64_t)t.g * nchains + chain, lane);
    }
}

// The items whose chain tile still has a live chain, and those tiles (one thread
// per item; the order of the lists is unspecified: items are independent).
__global__ void k_xt_items(const XtMemberDev* mem, const XtItem* all, int64_t nall, XtItem* out, int32_t* nout,
                           XtItem* tiles, int32_t* ntiles)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nall) return;
    const XtItem it = all[t];
    const XtArgs& a = mem[it.member].args[0];
    const int64_t s0 = (int64_t)it.g * a.nchains + (int64_t)it.ct * a.NT;
    const int cend = min(a.NT, a.nchains - it.ct * a.NT);
    bool any = false;
    for (int c = 0; c < cend && !any; ++c) any = a.live[s0 + c] != 0;
    if (!any) return;
    out[atomicAdd(nout, 1)] = it;
    if (it.rt == 0) tiles[atomicAdd(ntiles, 1)] = it;
}

// List of the (group, chain tile) pairs with a live chain (order unspecified:
// tiles are independent), one thread per pair.
__global__ void k_xt_tiles(int32_t G, int32_t nchains, int32_t NT, int32_t nct, const uint8_t* live,
                           int32_t* tiles, int32_t* ntiles)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)G * nct) return;
    const int64_t g = t / nct, c0 = (t % nct) * NT;
    bool any = false;
    for (int64_t c = c0; c < c0 + NT && c < nchains && !any; ++c) any = live[g * nchains + c] != 0;
    if (any) tiles[atomicAdd(ntiles, 1)] = (int32_t)t;
}

__global__ void k_xt_slots(int32_t G, int32_t nchains, int32_t r, int32_t q, int32_t warm,
                           int32_t* slot_j, int32_t* slot_jend, int32_t* slot_it)
{
    const int64_t total = (int64_t)G * nchains;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int cid = (int)(s % nchains);
        slot_j[s] = warm ? 0 : cid / r;
        slot_jend[s] = warm ? q : cid / r + 1;
        slot_it[s] = 0;
    }
}

}  // namespace

bool admm_tc_available() { return gram_tc_available(); }

namespace {

// Host state of one problem's streaming ADMM on the tensor cores: geometry,
// device buffers and the tensor map of its split inverse.
struct XtMember {
    AdmmProblem<float> P;
    int32_t nchains = 0, p = 0, RT = 0, kst = 0, W = 0;
    int64_t slots = 0, ppad = 0, kpad = 0;
    DevBuf rs, rinv, mp, zb, ub, v0, v1, vs0, vs1, cn, nb, sj, sje, sit, live;
    CUtensorMap mM;
};

// Everything before the first iteration: row scales and fp16 pieces of M, the
// initial state and its V pieces, the per-slot path positions.
void xt_prepare(const AdmmProblem<float>& P, cudaStream_t s, XtMember& m)
{
    m.P = P;
    m.nchains = P.warm ? (int32_t)P.r : (int32_t)(P.r * P.q);
    m.slots = (int64_t)P.G * m.nchains;
    m.p = (int)P.p;
    m.ppad = ceil_div(m.p, XT_TM) * XT_TM;
    m.kpad = ceil_div(m.p, XT_TK) * XT_TK;
    m.RT = (int)(m.ppad / XT_TM);
    m.kst = (int)(m.kpad / XT_TK);
    m.W = (int)((m.p + 63) / 64);
    const int p = m.p;
    const int64_t ppad = m.ppad, kpad = m.kpad, slots = m.slots;
    m.rs.alloc(sizeof(float) * (size_t)P.G * ppad, s);
    m.rinv.alloc(sizeof(float) * (size_t)P.G * ppad, s);
    m.mp.alloc(sizeof(__half) * XT_PIECES * (size_t)P.G * ppad * kpad, s);
    k_scale_split_m<<<(unsigned)ceil_div((int64_t)P.G * ppad * 32, 256), 256, 0, s>>>(
        P.M, P.G, p, ppad, kpad, m.rs.as<float>(), m.rinv.as<float>(), m.mp.as<__half>());
    UOI_CHECK_LAUNCH();
    m.zb.alloc(sizeof(float) * (size_t)slots * p, s);
    m.ub.alloc(sizeof(float) * (size_t)slots * p, s);
    m.v0.alloc(sizeof(__half) * XT_PIECES * (size_t)slots * kpad, s);
    m.v1.alloc(sizeof(__half) * XT_PIECES * (size_t)slots * kpad, s);
    m.vs0.alloc(sizeof(float) * (size_t)slots, s);
    m.vs1.alloc(sizeof(float) * (size_t)slots, s);
    m.cn.alloc(sizeof(float) * (size_t)P.G * P.r, s);
    m.nb.alloc(sizeof(float) * (size_t)slots * m.RT * 5, s);
    m.sj.alloc(sizeof(int32_t) * slots, s);
    m.sje.alloc(sizeof(int32_t) * slots, s);
    m.sit.alloc(sizeof(int32_t) * slots, s);
    m.live.alloc(slots, s);
    const bool start = P.z0 && !P.warm;
    k_c_norms<<<(unsigned)ceil_div((int64_t)P.G * P.r * 32, 256), 256, 0, s>>>(P.c, (int64_t)P.G * P.r, p,
                                                                               m.cn.as<float>());
    UOI_CHECK_LAUNCH();
    k_xt_vscale_init<<<(unsigned)ceil_div(slots * 32, 256), 256, 0, s>>>(
        slots, p, m.nchains, (int32_t)P.r, P.warm, start ? P.z0 : nullptr, start ? P.u0 : nullptr,
        m.cn.as<float>(), m.vs0.as<float>(), m.vs1.as<float>());
    UOI_CHECK_LAUNCH();
    k_xt_init<<<(unsigned)std::min<int64_t>(ceil_div(slots * kpad, 256), 8192), 256, 0, s>>>(
        slots, p, kpad, start ? P.z0 : nullptr, start ? P.u0 : nullptr, m.vs0.as<float>(), m.zb.as<float>(),
        m.ub.as<float>(), m.v0.as<__half>(), m.live.as<uint8_t>());
    UOI_CHECK_LAUNCH();
    // v1 holds the pieces of V for slots that do not change in an iteration
    UOI_CUDA(cudaMemcpyAsync(m.v1.ptr, m.v0.ptr, m.v0.bytes, cudaMemcpyDeviceToDevice, s));
    k_xt_slots<<<(unsigned)std::min<int64_t>(ceil_div(slots, 256), 4096), 256, 0, s>>>(
        P.G, m.nchains, (int32_t)P.r, P.q, P.warm, m.sj.as<int32_t>(), m.sje.as<int32_t>(), m.sit.as<int32_t>());
    UOI_CHECK_LAUNCH();
    count_launch(5);
    m.mM = make_map_bf16_blocks32(m.mp.ptr, (int64_t)P.G * m.RT * m.kst * XT_PIECES, XT_PIECES,
                                  CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
}

// The V pieces an x-update reads on even (parity 0) or odd steps, in boxes of NT chains.
CUtensorMap xt_map_v(const XtMember& m, int parity, int NT)
{
    return make_map_bf16_k32((parity ? m.v1 : m.v0).ptr, m.kpad, m.slots, XT_PIECES, NT,
                             CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
}

// Arguments of the x-update on even (parity 0) or odd steps: read V_t with its
// scale, write V_{t+1} into the other buffer.
XtArgs xt_args(const XtMember& m, int parity, int NT, int32_t* err)
{
    const AdmmProblem<float>& P = m.P;
    XtArgs a;
    a.G = P.G; a.q = P.q; a.r = (int32_t)P.r; a.p = m.p; a.nchains = m.nchains; a.NT = NT; a.kst = m.kst;
    a.RT = m.RT; a.warm = P.warm; a.ppad = m.ppad; a.kpad = m.kpad; a.slots = m.slots;
    a.c = P.c; a.lambdas = P.lambdas; a.rho = (float)P.rho;
    a.z = m.zb.as<float>(); a.u = m.ub.as<float>();
    a.vnext = (parity ? m.v0 : m.v1).as<__half>();
    a.row_inv = m.rinv.as<float>();
    a.vs_r = (parity ? m.vs1 : m.vs0).as<float>();
    a.vs_w = (parity ? m.vs0 : m.vs1).as<float>();
    a.slot_j = m.sj.as<int32_t>(); a.live = m.live.as<uint8_t>(); a.norms = m.nb.as<float>();
    a.err = err;
    a.tiles = nullptr;
    a.ntiles = nullptr;
    a.nct = (int32_t)ceil_div(m.nchains, NT);
    return a;
}

// Arguments of the convergence check after an even (parity 0) or odd step.
XtCheck xt_check_args(const XtMember& m, int parity, int32_t* live_count)
{
    const AdmmProblem<float>& P = m.P;
    XtCheck ca;
    ca.G = P.G; ca.q = P.q; ca.r = (int32_t)P.r; ca.p = m.p; ca.nchains = m.nchains; ca.RT = m.RT;
    ca.warm = P.warm; ca.max_iter = P.max_iter;
    ca.rho = (float)P.rho; ca.abs_tol = (float)P.abs_tol; ca.rel_tol = (float)P.rel_tol;
    ca.sqrtp = (float)sqrt((double)m.p);
    ca.z = m.zb.as<float>(); ca.norms = m.nb.as<float>();
    ca.slot_j = m.sj.as<int32_t>(); ca.slot_jend = m.sje.as<int32_t>(); ca.slot_it = m.sit.as<int32_t>();
    ca.live = m.live.as<uint8_t>(); ca.beta = P.beta; ca.iters = P.iters; ca.conv = P.conv;
    ca.family = P.family; ca.W = m.W; ca.live_count = live_count; ca.cn = m.cn.as<float>();
    ca.vs_next = (parity ? m.vs1 : m.vs0).as<float>(); ca.u = m.ub.as<float>(); ca.lambdas = P.lambdas;
    ca.near_count = P.near_count;
    return ca;
}

}  // namespace

// Streaming ADMM with the tensor-core x-update (FP32 state).  Same outputs as
// admm_solve<float>.
void admm_solve_tc(const AdmmProblem<float>& P, cudaStream_t s)
{
    XtMember m;
    xt_prepare(P, s, m);
    const int32_t nchains = m.nchains;
    const int NT = (int)std::min<int64_t>(XT_NT_MAX, ceil_div(nchains, 16) * 16);
    DevBuf cnt(sizeof(int32_t), s), err(sizeof(int32_t), s);
    UOI_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), s));
    const CUtensorMap mV0 = xt_map_v(m, 0, NT), mV1 = xt_map_v(m, 1, NT);
    UOI_CUDA(cudaFuncSetAttribute(k_xupdate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, XT_SMEM));
    XtArgs ae = xt_args(m, 0, NT, err.as<int32_t>()), ao = xt_args(m, 1, NT, err.as<int32_t>());
    const XtCheck ce = xt_check_args(m, 0, cnt.as<int32_t>()), co = xt_check_args(m, 1, cnt.as<int32_t>());
    const int32_t nct = ae.nct;
    // wide right-hand sides: launch only the tiles that still have a live chain
    const bool use_list = nct >= 4 && (int64_t)P.G * nct <= 65535;
    DevBuf tlist, tcount;
    int64_t tiles_bound = (int64_t)P.G * nct;
    if (use_list) {
        tlist.alloc(sizeof(int32_t) * (size_t)P.G * nct, s);
        tcount.alloc(sizeof(int32_t), s);
        UOI_CUDA(cudaMemsetAsync(tcount.ptr, 0, sizeof(int32_t), s));
        k_xt_tiles<<<(unsigned)ceil_div((int64_t)P.G * nct, 256), 256, 0, s>>>(
            P.G, nchains, NT, nct, m.live.as<uint8_t>(), tlist.as<int32_t>(), tcount.as<int32_t>());
        UOI_CHECK_LAUNCH();
        count_launch();
        ae.tiles = ao.tiles = tlist.as<int32_t>();
        ae.ntiles = ao.ntiles = tcount.as<int32_t>();
    }
    const dim3 gc((unsigned)ceil_div(m.slots * 32, 256));
    int32_t* host_cnt = pinned_scratch_i32();
    const int64_t bound = (int64_t)(P.warm ? P.q : 1) * P.max_iter + 2;
    bool done = false;
    for (int64_t it = 0; it < bound && !done; ++it) {
        const bool even = (it & 1) == 0;
        UOI_CUDA(cudaMemsetAsync(cnt.ptr, 0, sizeof(int32_t), s));
        ktimer_begin(TK_XUPDATE, s);
        const dim3 grid = use_list ? dim3((unsigned)m.RT, (unsigned)std::max<int64_t>(1, tiles_bound), 1u)
                                   : dim3((unsigned)m.RT, (unsigned)nct, (unsigned)P.G);
        k_xupdate_tc<<<grid, XT_THREADS, XT_SMEM, s>>>(m.mM, even ? mV0 : mV1, even ? ae : ao);
        UOI_CHECK_LAUNCH();
        ktimer_end(TK_XUPDATE, s, 0.0, 0.0);
        k_xt_check<<<gc, 256, 0, s>>>(even ? ce : co);
        UOI_CHECK_LAUNCH();
        count_launch(2);
        if (use_list) {
            UOI_CUDA(cudaMemsetAsync(tcount.ptr, 0, sizeof(int32_t), s));
            k_xt_tiles<<<(unsigned)ceil_div((int64_t)P.G * nct, 256), 256, 0, s>>>(
                P.G, nchains, NT, nct, m.live.as<uint8_t>(), tlist.as<int32_t>(), tcount.as<int32_t>());
            UOI_CHECK_LAUNCH();
            count_launch();
        }
        if ((it + 1) % 8 == 0 || it + 1 == bound) {
            int32_t herr = 0;
            UOI_CUDA(cudaMemcpyAsync(host_cnt, cnt.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            if (use_list)
                UOI_CUDA(cudaMemcpyAsync(host_cnt + 1, tcount.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            UOI_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            UOI_CUDA(cudaStreamSynchronize(s));
            if (herr) throw Error(herr, "tensor-core x-update: a bounded pipeline wait expired");
            done = *host_cnt == 0;
            if (use_list) tiles_bound = host_cnt[1];       // tiles only die: a bound for later steps
        }
    }
    if (!done) throw Error(UOI_ERR_TIMEOUT, "ADMM loop exceeded its iteration bound");
}

// ---- grouped solve of a batch of problems -------------------------------------------

namespace {

// Tile choices of the grouped solve, picked by timing: the chain tile NT (chains
// per CTA, hence how often a row tile of M is streamed per step) and the ring
// depth (4 stages at two CTAs per SM, or 6 at one).  Each candidate runs one
// replay of real iterations (every candidate gives the same iterates); the score
// is the replay's wall time per live item at its start.  The winner is kept per
// batch shape for the life of the process.
struct XtTileChoice {
    int NT = 32;
    int stages = 4;
};

std::mutex g_tune_mu;
std::map<std::string, XtTileChoice>& tune_cache()
{
    static std::map<std::string, XtTileChoice> c;
    return c;
}

constexpr int XT_CHUNK = 8;            // steps per graph replay (even: each replay starts on parity 0)

template <int STAGES>
constexpr int xt_smem() { return STAGES * XT_STAGE_MAX + 1024; }

}  // namespace

// A batch of problems whose tensor-core ADMM solves iterate together.  Members
// join from their own threads once their state is prepared; a solver thread,
// started by the first join, adds the members that have joined at every replay
// boundary, replays XT_CHUNK steps of all of them as one CUDA graph (grouped
// x-update and check launches), and releases each member as soon as none of its
// columns is still iterating, so that its thread goes on with the estimation while
// the others iterate.  Released members' device state stays in the table (their
// slots are no longer live, so no kernel touches their buffers) until the batch
// ends.
struct AdmmBatch {
    struct Slot {
        std::unique_ptr<XtMember> m;
        bool done = false;
        int32_t status = 0;
        std::string error;
        double ms = 0.0;            // replay time credited to this member
        int64_t launches = 0;       // launches credited to this member
    };

    AdmmBatch(int32_t expected, int device) : expected(expected), device(device) {}
    ~AdmmBatch()
    {
        if (solver.joinable()) solver.join();    // ends once every member has arrived and finished
    }

    std::mutex mu;
    std::condition_variable cv_members, cv_solver;
    int32_t expected, arrived = 0;
    int device;
    std::vector<Slot*> incoming;                 // joined, not yet in the solver's table
    std::vector<std::unique_ptr<Slot>> held;     // released members, kept until the batch ends
    std::thread solver;
    bool started = false;

    void hold(std::unique_ptr<Slot> sl)
    {
        std::lock_guard<std::mutex> lk(mu);
        held.push_back(std::move(sl));
    }

    void arrive_locked(Slot* slot)
    {
        ++arrived;
        if (slot) {
            incoming.push_back(slot);
            if (!started) {
                started = true;
                solver = std::thread([this] { run(); });
            }
        }
        cv_solver.notify_one();
    }

    void release(Slot* sl, int32_t st, const std::string& msg)
    {
        std::lock_guard<std::mutex> lk(mu);
        sl->status = st;
        sl->error = msg;
        sl->done = true;
        cv_members.notify_all();
    }

    void run();
};

namespace {

// The solver's device-side table of the members and their work items.  Counters
// (device, and their pinned copy): [0, cap) live slots per member, cap live items,
// cap + 1 live chain tiles, cap + 2 error.
struct GroupTable {
    std::vector<AdmmBatch::Slot*> slots;    // members in join order (index = table row)
    std::vector<bool> released;
    DevBuf d_mem, d_all, d_live, d_tiles, d_ctr;
    std::vector<XtMemberDev> hmem;
    int64_t nall = 0;
    int32_t cap = 0;
    int32_t* host = nullptr;
    int NT = 0;
    int32_t* ctr() const { return d_ctr.as<int32_t>(); }

    // Rebuilds the table and the item list for chain tile NT, then the live lists.
    void build(int nt, cudaStream_t s)
    {
        NT = nt;
        const int32_t n = (int32_t)slots.size();
        hmem.resize((size_t)n);
        std::vector<XtItem> items;
        for (int32_t i = 0; i < n; ++i) {
            const XtMember& m = *slots[(size_t)i]->m;
            const int t = (int)std::min<int64_t>(nt, ceil_div(m.nchains, 16) * 16);
            XtMemberDev& d = hmem[(size_t)i];
            d.mM = m.mM;
            for (int par = 0; par < 2; ++par) {
                d.mV[par] = xt_map_v(m, par, t);
                d.args[par] = xt_args(m, par, t, ctr() + cap + 2);
                d.check[par] = xt_check_args(m, par, ctr() + i);
            }
            if (released[(size_t)i]) continue;           // its items are all dead
            const int nct = (int)ceil_div(m.nchains, t);
            for (int g = 0; g < m.P.G; ++g)
                for (int ct = 0; ct < nct; ++ct)
                    for (int rt = 0; rt < m.RT; ++rt) items.push_back(XtItem{ i, g, rt, ct });
        }
        d_mem.alloc(sizeof(XtMemberDev) * (size_t)std::max(1, n), s);
        UOI_CUDA(cudaMemcpyAsync(d_mem.ptr, hmem.data(), sizeof(XtMemberDev) * (size_t)n, cudaMemcpyHostToDevice, s));
        nall = (int64_t)items.size();
        d_all.alloc(sizeof(XtItem) * (size_t)std::max<int64_t>(1, nall), s);
        d_live.alloc(sizeof(XtItem) * (size_t)std::max<int64_t>(1, nall), s);
        d_tiles.alloc(sizeof(XtItem) * (size_t)std::max<int64_t>(1, nall), s);
        if (nall > 0)
            UOI_CUDA(cudaMemcpyAsync(d_all.ptr, items.data(), sizeof(XtItem) * (size_t)nall, cudaMemcpyHostToDevice, s));
        UOI_CUDA(cudaMemsetAsync(ctr() + cap, 0, 2 * sizeof(int32_t), s));
        if (nall > 0) {
            k_xt_items<<<(unsigned)ceil_div(nall, 256), 256, 0, s>>>(d_mem.as<XtMemberDev>(), d_all.as<XtItem>(), nall,
                                                                      d_live.as<XtItem>(), ctr() + cap,
                                                                      d_tiles.as<XtItem>(), ctr() + cap + 1);
            UOI_CHECK_LAUNCH();
        }
        UOI_CUDA(cudaMemcpyAsync(host + cap, ctr() + cap, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        UOI_CUDA(cudaStreamSynchronize(s));
    }
};

struct GroupGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t grid = 0, tgrid = 0;
    XtTileChoice cfg;
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        grid = tgrid = 0;
    }
    ~GroupGraph() { reset(); }

    // XT_CHUNK steps of every member in the table (grids bounded by the live items
    // and tiles at capture; lists only shrink), then the next live lists and the
    // counters' copy to the host.
    void capture(GroupTable& T, const XtTileChoice& c, int64_t g, int64_t tg, cudaStream_t s)
    {
        reset();
        int32_t* ctr = T.ctr();
        UOI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < XT_CHUNK; ++k) {
            const int par = k & 1;
            cudaMemsetAsync(ctr, 0, sizeof(int32_t) * (size_t)T.cap, s);
            if (c.stages == 4)
                k_xupdate_tc_grouped<4><<<(unsigned)g, XT_THREADS, xt_smem<4>(), s>>>(
                    T.d_mem.as<XtMemberDev>(), T.d_live.as<XtItem>(), ctr + T.cap, par);
            else
                k_xupdate_tc_grouped<6><<<(unsigned)g, XT_THREADS, xt_smem<6>(), s>>>(
                    T.d_mem.as<XtMemberDev>(), T.d_live.as<XtItem>(), ctr + T.cap, par);
            k_xt_check_tiles<<<(unsigned)tg, 32 * XT_CHECK_WARPS, 0, s>>>(T.d_mem.as<XtMemberDev>(),
                                                                          T.d_tiles.as<XtItem>(), ctr + T.cap + 1, par);
        }
        cudaMemsetAsync(ctr + T.cap, 0, 2 * sizeof(int32_t), s);
        k_xt_items<<<(unsigned)std::max<int64_t>(1, ceil_div(T.nall, 256)), 256, 0, s>>>(
            T.d_mem.as<XtMemberDev>(), T.d_all.as<XtItem>(), T.nall, T.d_live.as<XtItem>(), ctr + T.cap,
            T.d_tiles.as<XtItem>(), ctr + T.cap + 1);
        cudaMemcpyAsync(T.host, ctr, sizeof(int32_t) * (size_t)(T.cap + 3), cudaMemcpyDeviceToHost, s);
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess)
            throw Error(UOI_ERR_CUDA, std::string("graph capture of the grouped ADMM: ") + cudaGetErrorString(e));
        UOI_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        grid = g;
        tgrid = tg;
        cfg = c;
    }
};

}  // namespace

void AdmmBatch::run()
{
    cudaSetDevice(device);
    cudaStream_t s = nullptr;
    int32_t fail = 0;
    std::string fail_msg;
    GroupTable T;
    GroupGraph gg;
    try {
        UOI_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        static std::once_flag once;
        std::call_once(once, [] {
            UOI_CUDA(cudaFuncSetAttribute(k_xupdate_tc_grouped<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          xt_smem<4>()));
            UOI_CUDA(cudaFuncSetAttribute(k_xupdate_tc_grouped<6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          xt_smem<6>()));
        });
        T.cap = expected;
        T.d_ctr.alloc(sizeof(int32_t) * (size_t)(T.cap + 3), s);
        UOI_CUDA(cudaMemsetAsync(T.d_ctr.ptr, 0, T.d_ctr.bytes, s));
        UOI_CUDA(cudaMallocHost(&T.host, sizeof(int32_t) * (size_t)(T.cap + 3)));
    } catch (const Error& e) {
        fail = e.status;
        fail_msg = e.what();
    }
    std::vector<XtTileChoice> cands;
    std::vector<double> score;
    size_t next_cand = 0;
    bool tuned = false;
    XtTileChoice best;
    std::string key;
    int active = 0;                    // members in the table not yet released
    for (;;) {
        std::vector<Slot*> fresh;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_solver.wait(lk, [&] { return !incoming.empty() || active > 0 || arrived == expected; });
            fresh.swap(incoming);
            if (fresh.empty() && active == 0 && arrived == expected) break;
        }
        if (fail) {
            for (Slot* sl : fresh) {
                T.slots.push_back(sl);             // its buffers are freed with the others below
                T.released.push_back(true);
                release(sl, fail, fail_msg);
            }
            continue;
        }
        try {
            if (!fresh.empty()) {
                for (Slot* sl : fresh) {
                    T.slots.push_back(sl);
                    T.released.push_back(false);
                }
                active += (int)fresh.size();
                if (key.empty()) {
                    // the batch shape as the first member gives it
                    const AdmmProblem<float>& P = T.slots[0]->m->P;
                    key = std::to_string(expected) + "/" + std::to_string(P.G) + "/" + std::to_string(P.q) + "/" +
                          std::to_string(P.r) + "/" + std::to_string(P.warm);
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    auto f = tune_cache().find(key);
                    if (f != tune_cache().end()) { best = f->second; tuned = true; }
                    const int ntmax = (int)std::min<int64_t>(XT_NT_MAX, ceil_div(T.slots[0]->m->nchains, 16) * 16);
                    for (int nt = 16; nt <= ntmax; nt *= 2)
                        for (int st : { 4, 6 }) cands.push_back(XtTileChoice{ nt, st });
                    if (cands.empty()) cands.push_back(XtTileChoice{ 16, 4 });
                    score.assign(cands.size(), 0.0);
                }
                T.NT = 0;                                   // table rebuilt below
            }
            const bool trial = !tuned && next_cand < cands.size();
            const XtTileChoice c = trial ? cands[next_cand] : best;
            if (T.NT != c.NT) {
                T.build(c.NT, s);
                gg.reset();
            }
            const int64_t grid = std::max<int32_t>(1, T.host[T.cap]), tgrid = std::max<int32_t>(1, T.host[T.cap + 1]);
            if (!gg.exec || gg.cfg.NT != c.NT || gg.cfg.stages != c.stages || grid > gg.grid || tgrid > gg.tgrid ||
                2 * grid < gg.grid)
                gg.capture(T, c, grid, tgrid, s);
            const int32_t at_start = T.host[T.cap];
            const auto t0 = std::chrono::steady_clock::now();
            UOI_CUDA(cudaGraphLaunch(gg.exec, s));
            UOI_CUDA(cudaStreamSynchronize(s));
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (T.host[T.cap + 2])
                throw Error(T.host[T.cap + 2], "tensor-core x-update: a bounded pipeline wait expired");
            if (trial) {
                score[next_cand] = ms / std::max(1, at_start);
                if (++next_cand == cands.size()) {
                    size_t bi = 0;
                    for (size_t k = 1; k < cands.size(); ++k)
                        if (score[k] < score[bi]) bi = k;
                    best = cands[bi];
                    tuned = true;
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    tune_cache()[key] = best;
                }
            }
            // credit the replay to the first member still iterating, then release the finished
            bool credited = false;
            for (size_t i = 0; i < T.slots.size(); ++i) {
                if (T.released[i]) continue;
                Slot* sl = T.slots[i];
                if (!credited) {
                    sl->ms += ms;
                    sl->launches += 2 * XT_CHUNK + 1;
                    credited = true;
                }
                if (T.host[i] == 0) {
                    T.released[i] = true;
                    --active;
                    release(sl, 0, std::string());
                }
            }
        } catch (const Error& e) {
            fail = e.status;
            fail_msg = e.what();
        } catch (const std::exception& e) {
            fail = UOI_ERR_CUDA;
            fail_msg = e.what();
        }
        if (fail) {
            // every member still waiting gets the error
            for (size_t i = 0; i < T.slots.size(); ++i)
                if (!T.released[i]) {
                    T.released[i] = true;
                    --active;
                    release(T.slots[i], fail, fail_msg);
                }
        }
    }
    gg.reset();
    if (s) cudaStreamSynchronize(s);
    // the members' ADMM state, freed on this thread's stream now that nothing reads it
    for (Slot* sl : T.slots) {
        XtMember& m = *sl->m;
        for (DevBuf* b : { &m.rs, &m.rinv, &m.mp, &m.zb, &m.ub, &m.v0, &m.v1, &m.vs0, &m.vs1, &m.cn, &m.nb, &m.sj,
                           &m.sje, &m.sit, &m.live }) {
            b->stream = s;
            b->release();
        }
    }
    for (DevBuf* b : { &T.d_mem, &T.d_all, &T.d_live, &T.d_tiles, &T.d_ctr }) b->release();
    if (T.host) cudaFreeHost(T.host);
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
}

namespace {
thread_local AdmmBatch* t_batch = nullptr;
thread_local bool t_batch_arrived = false;
}  // namespace

AdmmBatch* admm_batch_create(int32_t expected)
{
    int dev = 0;
    UOI_CUDA(cudaGetDevice(&dev));
    return new AdmmBatch(expected, dev);
}

void admm_batch_destroy(AdmmBatch* b) { delete b; }

void admm_batch_enter(AdmmBatch* b)
{
    t_batch = b;
    t_batch_arrived = false;
}

void admm_batch_leave()
{
    AdmmBatch* b = t_batch;
    t_batch = nullptr;
    if (!b || t_batch_arrived) return;
    t_batch_arrived = true;
    std::lock_guard<std::mutex> lk(b->mu);
    b->arrive_locked(nullptr);
}

bool admm_batch_try_join(const AdmmProblem<float>& P, cudaStream_t s)
{
    AdmmBatch* b = t_batch;
    if (!b || t_batch_arrived) return false;
    t_batch_arrived = true;
    auto slot = std::make_unique<AdmmBatch::Slot>();
    slot->m = std::make_unique<XtMember>();
    int32_t st = 0;
    std::string msg;
    try {
        xt_prepare(P, s, *slot->m);
        UOI_CUDA(cudaStreamSynchronize(s));
    } catch (const Error& e) {
        st = e.status;
        msg = e.what();
    }
    if (st != 0) {
        std::lock_guard<std::mutex> lk(b->mu);
        b->arrive_locked(nullptr);
        throw Error(st, msg);
    }
    AdmmBatch::Slot* sl = slot.get();
    {
        std::unique_lock<std::mutex> lk(b->mu);
        b->arrive_locked(sl);
        b->cv_members.wait(lk, [&] { return sl->done; });
    }
    // the solver keeps this member's state until the batch ends: hand the slot over
    b->hold(std::move(slot));
    ktimer_credit(TK_XUPDATE, sl->ms, sl->launches);
    count_launch(sl->launches);
    if (sl->status != 0) throw Error(sl->status, sl->error);
    return true;
}

}  // namespace uoi
