// gram_tc.cu -- G1 on the 5th-generation tensor cores (tcgen05, TMA, TMEM): the
// weighted moments of the mixed-precision form.
//
// For bootstrap k, G_k = X^T W_k X and B_k = X^T W_k Y are the lower triangle of
// Z_k^T Z_k with Z_k = diag(sqrt(w_k)) [X | Y] restricted to rows with w > 0.
// Each FP64 value v of Z_k is split into two bf16 pieces, hi = bf16(v) and
// lo = bf16(v - hi) (|v - hi - lo| <= 2^-17 |v|), and the product is
// hi'hi + hi'lo + lo'hi on bf16 tensor cores with FP32 accumulation in TMEM.
// The tensor cores' FP32 accumulation loses about a third of an ulp per K=16
// step (measured), so the accumulator is drained every 128 sample rows (24
// steps, <= 5e-7 relative) into FP32 running sums held in the epilogue warps'
// registers (the rounding of those few hundred additions is ~1e-7 relative),
// and the sum is written once in FP64 at the end.
// The lo'lo term (up to 2^-16 relative per product) is zero-mean off the
// diagonal; on the diagonal it is a positive bias and is added exactly
// (k_diag_lo).  Relative error of the Gram: ~5e-7 of the largest diagonal entry.
//
// Two kernels:
//  * k_split_transpose: gather rows (with weights), split, and write the two
//    bf16 pieces transposed (features x rows, rows contiguous = K-major).
//  * k_gram_tc: one cluster of two CTAs per (256 x 256 block of the lower
//    triangle, item): row tiles 2m and 2m+1 need the same column tiles, and the
//    pair computes both with M = 256 products (tcgen05 cta_group::2).  Each CTA
//    stages its own 128 rows of A and one half (128 columns) of B, so a stage
//    is 32 KB per SM instead of 48 and six fit in shared memory; the first CTA
//    issues the pair's MMAs and each CTA's TMEM receives its own 128 x 256
//    tile.  Warp 0 issues TMA loads of K-major SWIZZLE_64B tiles (completion
//    counted on the first CTA's barrier); warp 1 of the first CTA issues
//    tcgen05.mma (bf16 -> f32) into one of two TMEM accumulators; warps 2-9 of
//    both CTAs drain the other accumulator (tcgen05.ld) into their registers.
//    Every wait is bounded (about one second) and reports UOI_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "tc_common.cuh"

namespace uoi {

namespace {
using namespace tc;

constexpr int TM = 128;                 // tile rows per CTA (the pair's UMMA M is 256)
constexpr int TN = 256;                 // tile cols (UMMA N), 128 staged by each CTA
constexpr int TK = 32;                  // rows of the sample per stage (64 B of bf16, 64-byte swizzle)
constexpr int STAGES = 6;
constexpr int CHUNK_STAGES = 4;         // 128 sample rows per FP32 accumulation chunk
constexpr int A_BYTES = TM * TK * 2;    // 8 KB per piece
constexpr int BH_BYTES = (TN / 2) * TK * 2;              // this CTA's half of B: 8 KB per piece
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * BH_BYTES;  // 32 KB per CTA
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;  // + alignment slack
static_assert(TN == 2 * TM, "a pair of row tiles spans one column tile");
constexpr uint32_t TMEM_COLS = 512;     // two 256-column FP32 accumulators
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;   // producer, MMA, 8 epilogue warps

struct GramTcArgs {
    int64_t n_pad;            // K extent of the transposed pieces (multiple of TK)
    int32_t pz_pad;           // feature extent of the pieces (multiple of TN)
    int32_t pz;               // Z columns = pz_x + r
    int32_t pz_x;             // columns of Z that come from X (= p, or |U| with a subset)
    int32_t r;
    int32_t p_out;            // leading size of the G / Bm outputs
    int32_t ntiles;           // tile pairs (clusters per item)
    const int32_t* tiles;     // (m, tj): row tiles 2m (first CTA) and 2m+1, column tile tj
    const int32_t* nrows;     // per item: sample rows (K extent actually used)
    const int32_t* colmap;    // Z column (< pz_x) -> output feature index, or null
    double* G;                // items x p_out x p_out
    double* Bm;               // items x p_out x r
    int32_t* err;
    uint64_t wait_ns = tc::kWaitLimitNs;   // limit of every bounded mbarrier wait
};

__global__ void __launch_bounds__(THREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tmA, GramTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = blockIdx.x & 1;                 // 0: the CTA that issues the pair's MMAs
    const int pr = blockIdx.x >> 1;                  // the cluster (2 CTAs along x)
    const int item = blockIdx.y;
    const int ti = 2 * a.tiles[2 * pr] + rank, tj = a.tiles[2 * pr + 1];
    const int rows = a.nrows[item];
    const int kstages = (rows + TK - 1) / TK;
    const int nchunks = (kstages + CHUNK_STAGES - 1) / CHUNK_STAGES;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        // full: the first CTA's arrival plus the bytes of both CTAs' loads;
        // empty / accumulator ready / done: one arrival from the pair's commit;
        // accumulator drained: every epilogue thread of both CTAs
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&accf_bar[b], 1); mbar_init(&acce_bar[b], 2 * 32 * EPI_WARPS); }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        // the same TMEM columns in both CTAs (one warp of each allocates)
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();                  // both CTAs' barriers and TMEM exist before either uses the other's
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0 && kstages > 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        const int zA = item * 2;
        const int jb = tj * TN + rank * (TN / 2);    // this CTA's half of the column tile
        for (int g = 0; g < kstages; ++g) {
            const int s = g % STAGES;
            if (g >= STAGES && !mbar_wait(&empty_bar[s], ((g / STAGES) - 1) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            const uint32_t st = sbase + s * STAGE_BYTES;
            if (rank == 0) mbar_expect_tx(&full_bar[s], 2 * STAGE_BYTES);
            const uint32_t fb = cluster_addr(&full_bar[s], 0);
            const int k0 = g * TK;
            tma_load_3d_pair(st, &tmA, fb, k0, ti * TM, zA);                              // A hi
            tma_load_3d_pair(st + A_BYTES, &tmA, fb, k0, ti * TM, zA + 1);                // A lo
            tma_load_3d_pair(st + 2 * A_BYTES, &tmA, fb, k0, jb, zA);                     // B hi (half)
            tma_load_3d_pair(st + 2 * A_BYTES + BH_BYTES, &tmA, fb, k0, jb, zA + 1);      // B lo (half)
        }
        if (abort_flag && rank == 0) {
            // let the copies already issued land before the CTA releases its memory
            for (int g = max(0, kstages - STAGES); g < kstages; ++g)
                mbar_wait(&full_bar[g % STAGES], (g / STAGES) & 1, &abort_flag, a.wait_ns);
        }
    } else if (warp == 1 && lane == 0 && kstages > 0 && rank == 0) {
        // ---------------- MMA issuer (first CTA, for the pair) ----------------
        constexpr uint32_t idesc = idesc_bf16(2 * TM, TN);
        int g = 0;
        for (int c = 0; c < nchunks && !abort_flag; ++c) {
            const int b = c & 1;
            if (c >= 2 && !mbar_wait_cluster(&acce_bar[b], ((c >> 1) - 1) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(b * TN);
            const int gend = min(kstages, (c + 1) * CHUNK_STAGES);
            bool first = true;
            for (; g < gend; ++g) {
                const int s = g % STAGES;
                if (!mbar_wait(&full_bar[s], (g / STAGES) & 1, &abort_flag, a.wait_ns)) {
                    abort_flag = 1;
                    atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t st = sbase + s * STAGE_BYTES;
                const uint64_t ah = smem_desc_sw64(st), al = smem_desc_sw64(st + A_BYTES);
                const uint64_t bh = smem_desc_sw64(st + 2 * A_BYTES);
                const uint64_t bl = smem_desc_sw64(st + 2 * A_BYTES + BH_BYTES);
#pragma unroll
                for (int ks = 0; ks < TK / 16; ++ks) {
                    const uint64_t adv = (uint64_t)(ks * 32 >> 4);   // 16 bf16 = 32 B along K
                    mma_bf16_pair(d, ah + adv, bh + adv, idesc, first ? 0u : 1u);
                    mma_bf16_pair(d, ah + adv, bl + adv, idesc, 1u);
                    mma_bf16_pair(d, al + adv, bh + adv, idesc, 1u);
                    first = false;
                }
                mma_commit_pair(&empty_bar[s]);     // slot s of both CTAs free once these complete
            }
            if (abort_flag) break;
            mma_commit_pair(&accf_bar[b]);          // accumulator b ready in both CTAs
        }
        mma_commit_pair(&done_bar);                 // every MMA issued above has completed
        int dummy = 0;
        mbar_wait(&done_bar, 0, &dummy, a.wait_ns);
    } else if (warp == 1 && lane == 0 && kstages > 0) {
        // second CTA: its TMEM is written by the first CTA's MMAs until this arrives
        int dummy = 0;
        mbar_wait(&done_bar, 0, &dummy, a.wait_ns);
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> FP32 running sums (both CTAs) ----------------
        const int quad = warp & 3;                       // TMEM lanes 32*quad .. +31
        const int half = (warp - 2) >> 2;                // columns 128*half .. +127
        const int iz = ti * TM + quad * 32 + lane;       // Z row of this thread
        const uint32_t drained[2] = { cluster_addr(&acce_bar[0], 0), cluster_addr(&acce_bar[1], 0) };
        float acc[128];
#pragma unroll
        for (int t = 0; t < 128; ++t) acc[t] = 0.f;
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
            for (int cb = 0; cb < 8; ++cb) {
                float v[16];
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) +
                                       (uint32_t)(b * TN + half * 128 + cb * 16);
                tmem_ld16(taddr, v);
#pragma unroll
                for (int t = 0; t < 16; ++t) acc[cb * 16 + t] += v[t];
            }
            tc_fence_before();
            mbar_arrive_cluster(drained[b]);             // on the first CTA's barrier
        }
        if (iz < a.pz && !abort_flag) {
            const int jz0 = tj * TN + half * 128;
#pragma unroll
            for (int t = 0; t < 128; ++t) {
                const int jz = jz0 + t;
                if (jz > iz || jz >= a.pz_x) continue;           // lower triangle, X columns
                const double val = (double)acc[t];
                const int jo = a.colmap ? a.colmap[jz] : jz;
                if (iz < a.pz_x) {
                    const int io = a.colmap ? a.colmap[iz] : iz;
                    const int64_t gi = ((int64_t)item * a.p_out + io) * a.p_out + jo;
                    if (UOI_IN_BOUNDS(gi, (int64_t)gridDim.y * a.p_out * a.p_out, 101)) a.G[gi] = val;
                } else {
                    const int64_t bi = ((int64_t)item * a.p_out + jo) * a.r + (iz - a.pz_x);
                    if (UOI_IN_BOUNDS(bi, (int64_t)gridDim.y * a.p_out * a.r, 102)) a.Bm[bi] = val;
                }
            }
        }
    }
    // teardown: no MMA writes TMEM any more (done waited for above) and both
    // CTAs have finished reading their TMEM before the pair frees it; neither
    // CTA leaves while the other may still signal its barriers
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
    cluster_sync();
}

// Gather rows with positive weight, scale by sqrt(w), split into bf16 hi/lo and
// write transposed: out[((item*2 + piece) * pz_pad + col) * n_pad + t].  Values
// are taken to FP32 first (relative error 2^-23 after the scaling, below the
// 2^-17 residue of the two-piece split).  A block covers 128 sample rows x 32
// columns: warp w reads rows 16w .. 16w+15 (16 row segments of 128 B, all loads
// issued before any shared-memory store) and stores each column's 16 values as
// four 16-byte vectors into a column-major tile; with a row length of 132 floats
// both the vector stores and the vector reads of the second phase are free of
// bank conflicts.  Then each lane turns four consecutive rows of a column into
// 8-byte runs of bf16 hi and lo.  It also writes the FP32 sum of lo^2 of each
// column over each 64 rows (losq[(item*row_tiles + tile)*pz_x + col], a fixed
// order), from which the diagonal correction is reduced in a fixed order.
constexpr int SPLIT_ROWS = 128;
constexpr int SPLIT_COLS = 32;                  // columns of one half of a block
constexpr int SPLIT_HALVES = 2;                 // a block covers 64 columns: its loads of both halves in flight together
constexpr int SPLIT_LD = SPLIT_ROWS + 4;
__global__ void __launch_bounds__(256)
k_split_transpose(const double* X, int64_t ldx, const float* X32, int64_t ld32, int32_t x32_compact,
                  const double* Y, int64_t ldy, int32_t pz_x, int32_t r, const int32_t* colmap,
                  const int32_t* rowlist,
                  const float* rowscale, const int32_t* nrows, int64_t m, int64_t n_pad,
                  int32_t pz_pad, int32_t row_tiles, __nv_bfloat16* out, float* losq,
                  const float* zrow)
{
    __shared__ __align__(16) float tile[SPLIT_HALVES][SPLIT_COLS][SPLIT_LD];      // [half][column][row]
    __shared__ int64_t rowoff[SPLIT_ROWS];
    __shared__ const float* rowptr[SPLIT_ROWS];     // row of the FP32 copy, or a row of zeros
    __shared__ float rowsc[SPLIT_ROWS];
    // items vary fastest: the items' sorted row lists advance through X at nearly
    // the same pace, so CTAs launched together read the same rows (L2 hits)
    const int item = blockIdx.x;
    const int64_t t0 = (int64_t)blockIdx.y * SPLIT_ROWS;
    const int cb = blockIdx.z * SPLIT_COLS * SPLIT_HALVES;
    const int nr = nrows[item];
    const int pz = pz_x + r;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < SPLIT_ROWS) {
        const int64_t t = t0 + threadIdx.x;
        const int64_t row = t < nr ? (int64_t)rowlist[(int64_t)item * m + t] : -1;
        rowoff[threadIdx.x] = row;
        rowptr[threadIdx.x] = row >= 0 && X32 ? X32 + row * ld32 : zrow;
        rowsc[threadIdx.x] = t < nr ? rowscale[(int64_t)item * m + t] : 0.f;
    }
    __syncthreads();
    // four consecutive rows of one column, scaled, as one 16-byte vector of the tile
    auto put = [&](int h, const float (&q)[16]) {
#pragma unroll
        for (int i4 = 0; i4 < 4; ++i4) {
            const int tl = 16 * warp + 4 * i4;
            *reinterpret_cast<float4*>(&tile[h][lane][tl]) =
                make_float4(q[4 * i4] * rowsc[tl], q[4 * i4 + 1] * rowsc[tl + 1], q[4 * i4 + 2] * rowsc[tl + 2],
                            q[4 * i4 + 3] * rowsc[tl + 3]);
        }
    };
    // read: warp w takes rows 16w .. 16w + 15; lane = column of each half.  Blocks
    // whose columns all come from the FP32 copy without a column map (all but the
    // last block of a fit) take a path with no per-element branch, with the loads of
    // both halves issued before any store.
    const bool fast = X32 != nullptr && (colmap == nullptr || x32_compact) &&
                      cb + SPLIT_COLS * SPLIT_HALVES <= pz_x;
    if (fast) {
        float q[SPLIT_HALVES][16];
#pragma unroll
        for (int h = 0; h < SPLIT_HALVES; ++h)
#pragma unroll
            for (int i = 0; i < 16; ++i) q[h][i] = __ldg(rowptr[16 * warp + i] + cb + SPLIT_COLS * h + lane);
#pragma unroll
        for (int h = 0; h < SPLIT_HALVES; ++h) put(h, q[h]);
    } else {
#pragma unroll 1
        for (int h = 0; h < SPLIT_HALVES; ++h) {
            const int c = cb + SPLIT_COLS * h + lane;
            const int64_t col = colmap && c < pz_x ? colmap[c] : c;      // column of X
            const int64_t col32 = x32_compact ? c : col;                 // column of the FP32 copy
            float q[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int64_t row = rowoff[16 * warp + i];
                float v = 0.f;
                if (row >= 0 && c < pz) {
                    if (c < pz_x)
                        v = X32 ? __ldg(X32 + row * ld32 + col32) : f64_to_f32_int(__ldg(X + row * ldx + col));
                    else
                        v = f64_to_f32_int(__ldg(Y + row * ldy + (c - pz_x)));
                }
                q[i] = v;
            }
            put(h, q);
        }
    }
    __syncthreads();
    // write: warp w takes columns w, w + 8, w + 16, w + 24 of each half; lane covers
    // rows 4*lane .. 4*lane + 3 (lanes 0-15: the first 64 rows, 16-31: the second)
    const int64_t piece = (int64_t)pz_pad * n_pad;                 // elements per piece
#pragma unroll
    for (int h = 0; h < SPLIT_HALVES; ++h) {
        const int c0 = cb + SPLIT_COLS * h;
        __nv_bfloat16* out_hi = out + ((int64_t)item * 2 * pz_pad + c0 + warp) * n_pad + t0 + 4 * lane;
        float* losq_c = losq + ((int64_t)item * row_tiles + (t0 / 64) + (lane >> 4)) * pz_x + c0 + warp;
#pragma unroll
        for (int j = 0; j < SPLIT_COLS / 8; ++j) {
            const int cl = warp + 8 * j;
            const int cc = c0 + cl;
            if (cc >= pz_pad) break;
            const float4 v = *reinterpret_cast<const float4*>(&tile[h][cl][4 * lane]);
            // two values per conversion (round to nearest even, as one at a time)
            const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
            const float2 hf01 = __bfloat1622float2(h01), hf23 = __bfloat1622float2(h23);
            const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - hf01.x, v.y - hf01.y);   // exact differences
            const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - hf23.x, v.w - hf23.y);
            const float2 lf01 = __bfloat1622float2(l01), lf23 = __bfloat1622float2(l23);
            float sq = 0.f;
            sq += lf01.x * lf01.x;
            sq += lf01.y * lf01.y;
            sq += lf23.x * lf23.x;
            sq += lf23.y * lf23.y;
            __nv_bfloat16* base_hi = out_hi + (int64_t)(8 * j) * n_pad;
            *reinterpret_cast<uint2*>(base_hi) =
                make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
            *reinterpret_cast<uint2*>(base_hi + piece) =
                make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
            if (cc < pz_x) {
                // sum over the 16 lanes of each 64-row half (fixed order)
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
                if ((lane & 15) == 0) losq_c[8 * j] = sq;
            }
        }
    }
}

// Row list of each item: rows with positive weight (in increasing order) and
// their scale sqrt(w); nrows[item] = count.  One block per item.
__global__ void k_row_lists(const uint32_t* w, const uint8_t* mask, int64_t m, int32_t* rowlist,
                            float* rowscale, int32_t* nrows)
{
    const int item = blockIdx.x;
    __shared__ int warp_tot[32];
    __shared__ int carry, block_total;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < m; base += blockDim.x) {
        const int64_t t = base + threadIdx.x;
        uint32_t wt = 0;
        if (t < m) wt = w ? w[(int64_t)item * m + t] : (uint32_t)mask[(int64_t)item * m + t];
        const int flag = wt > 0;
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[wid] = __popc(bal);
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            int v = lane < nw ? warp_tot[lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += n;
            }
            if (lane < nw) warp_tot[lane] = incl - v;
            if (lane == nw - 1) block_total = incl;
        }
        __syncthreads();
        if (flag) {
            const int pos = carry + warp_tot[wid] + before;
            rowlist[(int64_t)item * m + pos] = (int32_t)t;
            rowscale[(int64_t)item * m + pos] = sqrtf((float)wt);
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += block_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) nrows[item] = carry;
}

// corr[item][c] = sum_t lo[c][t]^2: the lo'lo term of the diagonal, which the
// three-product split leaves out and which is biased (always positive).  The
// off-diagonal lo'lo terms are zero-mean and stay out.  Sums the per-64-row
// partials of k_split_transpose in a fixed order.
// Same for an output without a column map: 32 x 32 tiles through shared memory,
// so the lower triangle is read and the upper written along rows.  Block (32, 8).
__global__ void k_mirror_tiled(double* G, int64_t p_out, int32_t pz_x, const double* corr)
{
    __shared__ double tile[32][33];
    const int item = blockIdx.z;
    const int bx = blockIdx.x, by = blockIdx.y;       // target tile: rows by*32.., columns bx*32..
    if (bx < by) return;                              // lower tiles are the source
    double* g = G + (size_t)item * p_out * p_out;
    const int tx = threadIdx.x;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {    // source rows bx*32 + yy, columns by*32 + tx
        const int r = bx * 32 + yy, c = by * 32 + tx;
        tile[yy][tx] = (r < pz_x && c < pz_x) ? g[(size_t)r * p_out + c] : 0.0;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {    // target rows by*32 + yy, columns bx*32 + tx
        const int r = by * 32 + yy, c = bx * 32 + tx;
        if (r >= pz_x || c >= pz_x) continue;
        if (c > r) g[(size_t)r * p_out + c] = tile[tx][yy];
        else if (c == r) g[(size_t)r * p_out + c] += corr[(int64_t)item * pz_x + r];
    }
}

__global__ void k_diag_lo(const float* losq, int32_t row_tiles, int32_t pz_x,
                          const int32_t* nrows, double* corr)
{
    const int item = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= pz_x) return;
    const int tiles = min((nrows[item] + 63) / 64, row_tiles);
    const float* src = losq + (int64_t)item * row_tiles * pz_x + c;
    double s = 0.0;
    int t = 0;
    // eight loads in flight before their (in-order) additions
    for (; t + 8 <= tiles; t += 8) {
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = src[(int64_t)(t + u) * pz_x];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)x[u];
    }
    for (; t < tiles; ++t) s += (double)src[(int64_t)t * pz_x];
    corr[(int64_t)item * pz_x + c] = s;
}

// Add the diagonal correction only (the caller reads the lower triangle alone).
__global__ void k_add_diag(double* G, int64_t p_out, int32_t pz_x, const double* corr)
{
    const int item = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < pz_x) G[(size_t)item * p_out * p_out + (size_t)c * p_out + c] += corr[(int64_t)item * pz_x + c];
}

// Add the diagonal correction and fill the upper triangle from the lower one
// (over the used features only).
__global__ void k_mirror(double* G, int64_t p_out, const int32_t* colmap, int32_t pz_x,
                         const double* corr)
{
    const int item = blockIdx.y;
    double* g = G + (size_t)item * p_out * p_out;
    const int64_t total = (int64_t)pz_x * pz_x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / pz_x), j = (int)(t % pz_x);
        const int io = colmap ? colmap[i] : i, jo = colmap ? colmap[j] : j;
        if (j == i) g[(size_t)io * p_out + io] += corr[(int64_t)item * pz_x + i];
        if (j <= i) continue;
        g[(size_t)io * p_out + jo] = g[(size_t)jo * p_out + io];
    }
}

}  // namespace

bool gram_tc_available()
{
    // decided once per process; the initialisation of a function-local static is
    // thread-safe, so concurrent first callers (batch workers) all see one answer
    static const bool avail = [] {
        int dev = 0, major = 0, minor = 0;
        return cudaGetDevice(&dev) == cudaSuccess &&
               cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
               cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess &&
               major == 10 && minor == 3 && tc::encode_fn() != nullptr;
    }();
    return avail;
}

// Tensor-core moments for B items (weights w or 0/1 mask, or unweighted),
// optionally restricted to the X columns listed in colmap (pz_x of them).
void moments_tc_cols(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m,
                     int64_t p_out, int64_t r, int32_t pz_x, const int32_t* colmap,
                     const uint32_t* w, const uint8_t* mask, int32_t B, double* G, double* Bm,
                     cudaStream_t s, const float* X32, int64_t ld32, bool x32_compact, bool lower_only)
{
    if (ld32 == 0) ld32 = ldx;
    if (!gram_tc_available()) throw Error(UOI_ERR_UNSUPPORTED, "tcgen05 Gram needs sm_103a");
    const int32_t pz = pz_x + (int32_t)r;
    const int32_t pz_pad = (int32_t)ceil_div(pz, TN) * TN;
    // tile list of the lower triangle (rows of Z x X columns), by pairs of row tiles
    // 2m, 2m+1: both need the column tiles tj <= floor(min(256m + 255, pz_x - 1) / 256).
    // With an odd count the last pair's second tile lies past pz: it reads the zero
    // padding of the pieces (pz_pad is a multiple of TN) and writes nothing.
    std::vector<int32_t> tiles;
    const int nti = (int)ceil_div(pz, TM);
    for (int m2 = 0; 2 * m2 < nti; ++m2) {
        const int jmax = std::min(m2 * TN + TN - 1, pz_x - 1);
        for (int tj = 0; tj * TN <= jmax; ++tj) { tiles.push_back(m2); tiles.push_back(tj); }
    }
    const int ntiles = (int)tiles.size() / 2;
    DevBuf tl(sizeof(int32_t) * tiles.size(), s);
    UOI_CUDA(cudaMemcpyAsync(tl.ptr, tiles.data(), sizeof(int32_t) * tiles.size(),
                             cudaMemcpyHostToDevice, s));
    DevBuf rows(sizeof(int32_t) * (size_t)(m * B), s), scale(sizeof(float) * (size_t)(m * B), s);
    DevBuf nrows(sizeof(int32_t) * B, s), err(sizeof(int32_t), s);
    UOI_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), s));
    if (w || mask) {
        k_row_lists<<<B, 1024, 0, s>>>(w, mask, m, rows.as<int32_t>(), scale.as<float>(),
                                        nrows.as<int32_t>());
        UOI_CHECK_LAUNCH();
        count_launch();
    } else {
        throw Error(UOI_ERR_INVALID_ARG, "tensor-core moments need weights or a mask");
    }
    std::vector<int32_t> nr((size_t)B);
    UOI_CUDA(cudaMemcpyAsync(nr.data(), nrows.ptr, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    int32_t max_rows = 1;
    for (int32_t v : nr) max_rows = std::max(max_rows, v);
    const int64_t n_pad = ceil_div(max_rows, 128) * 128;      // K extent (whole split blocks)
    const int32_t row_tiles = (int32_t)(n_pad / 64);
    // items per pass bounded by the size of the split copies (<= 16 GB: the 48
    // selection items of a 50000 x 2000 fit in one pass, 22.7 waves of 152 CTAs
    // instead of 15 + 9 in two)
    const size_t per_item = (size_t)2 * pz_pad * n_pad * sizeof(__nv_bfloat16);
    const int group = (int)std::max<size_t>(1, std::min<size_t>((size_t)B, (16ull << 30) / per_item));
    DevBuf zt(per_item * group, s);
    DevBuf corr(sizeof(double) * (size_t)group * pz_x, s);
    DevBuf losq(sizeof(float) * (size_t)group * row_tiles * pz_x, s);
    DevBuf zrow(sizeof(float) * (size_t)pz_pad, s);               // read for the padding rows
    UOI_CUDA(cudaMemsetAsync(zrow.ptr, 0, sizeof(float) * (size_t)pz_pad, s));
    auto kern = k_gram_tc;
    UOI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    for (int b0 = 0; b0 < B; b0 += group) {
        const int nb = std::min(group, B - b0);
        dim3 gs((unsigned)nb, (unsigned)(n_pad / SPLIT_ROWS), (unsigned)ceil_div(pz_pad, SPLIT_COLS * SPLIT_HALVES));
        k_split_transpose<<<gs, 256, 0, s>>>(X, ldx, X32, ld32, x32_compact ? 1 : 0, Y, ldy, pz_x,
                                             (int32_t)r, colmap,
                                             rows.as<int32_t>() + (size_t)b0 * m,
                                             scale.as<float>() + (size_t)b0 * m,
                                             nrows.as<int32_t>() + b0, m, n_pad, pz_pad, row_tiles,
                                             zt.as<__nv_bfloat16>(), losq.as<float>(), zrow.as<float>());
        UOI_CHECK_LAUNCH();
        const CUtensorMap mA = tc::make_map_bf16_k32(zt.ptr, n_pad, pz_pad, 2 * nb, TM);   // 128-row boxes
        GramTcArgs a;
        a.n_pad = n_pad; a.pz_pad = pz_pad; a.pz = pz; a.pz_x = pz_x; a.r = (int32_t)r;
        a.p_out = (int32_t)p_out; a.ntiles = ntiles; a.tiles = tl.as<int32_t>();
        a.nrows = nrows.as<int32_t>() + b0; a.colmap = colmap;
        a.G = G + (size_t)b0 * p_out * p_out; a.Bm = Bm + (size_t)b0 * p_out * r;
        a.err = err.as<int32_t>();
        ktimer_begin(TK_GRAM_TC, s);
        {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(2 * ntiles), (unsigned)nb);
            cfg.blockDim = dim3(THREADS);
            cfg.dynamicSmemBytes = SMEM_BYTES;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            UOI_CUDA(cudaLaunchKernelEx(&cfg, k_gram_tc, mA, a));
        }
        UOI_CHECK_LAUNCH();
        ktimer_end(TK_GRAM_TC, s, 0.0, 0.0);
        dim3 gd((unsigned)ceil_div(pz_x, 256), (unsigned)nb);
        k_diag_lo<<<gd, 256, 0, s>>>(losq.as<float>(), row_tiles, pz_x, nrows.as<int32_t>() + b0,
                                     corr.as<double>());
        UOI_CHECK_LAUNCH();
        if (lower_only && !colmap) {
            k_add_diag<<<dim3((unsigned)ceil_div(pz_x, 256), (unsigned)nb), 256, 0, s>>>(
                G + (size_t)b0 * p_out * p_out, p_out, pz_x, corr.as<double>());
        } else if (colmap) {
            dim3 gm((unsigned)std::min<int64_t>(ceil_div((int64_t)pz_x * pz_x, 256), 2048), (unsigned)nb);
            k_mirror<<<gm, 256, 0, s>>>(G + (size_t)b0 * p_out * p_out, p_out, colmap, pz_x,
                                        corr.as<double>());
        } else {
            const unsigned tt = (unsigned)ceil_div(pz_x, 32);
            k_mirror_tiled<<<dim3(tt, tt, (unsigned)nb), dim3(32, 8), 0, s>>>(
                G + (size_t)b0 * p_out * p_out, p_out, pz_x, corr.as<double>());
        }
        UOI_CHECK_LAUNCH();
        count_launch(4);
    }
    int32_t h = 0;
    UOI_CUDA(cudaMemcpyAsync(&h, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    if (h) throw Error(h, "tensor-core Gram: a bounded pipeline wait expired");
    // algorithmic work: the lower triangle of X^T W X plus X^T W Y over the rows used
    double used_rows = 0.0;
    for (int32_t v : nr) used_rows += (double)v;
    ktimer_add_work(TK_GRAM_TC,
                    2.0 * used_rows * ((double)pz_x * (pz_x + 1) / 2.0 + (double)pz_x * r),
                    used_rows * (double)(pz_x + r) * 8.0);
}

void moments_tc(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p,
                int64_t r, const uint32_t* w, const uint8_t* mask, int32_t B, double* G,
                double* Bm, cudaStream_t s, const float* X32, bool lower_only)
{
    moments_tc_cols(X, ldx, Y, ldy, m, p, r, (int32_t)p, nullptr, w, mask, B, G, Bm, s, X32, 0, false,
                    lower_only);
}

namespace {
__global__ void k_gather_cols_f32(const float* X32, int64_t ld, int64_t m, const int32_t* cols, int64_t nu,
                                  float* out)
{
    const int64_t total = m * nu;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        out[t] = X32[(t / nu) * ld + cols[t % nu]];
}
}  // namespace

void gather_cols_f32(const float* X32, int64_t ld, int64_t m, const int32_t* cols, int64_t nu, float* out,
                     cudaStream_t s)
{
    k_gather_cols_f32<<<(unsigned)std::min<int64_t>(ceil_div(m * nu, 256), 152 * 32), 256, 0, s>>>(
        X32, ld, m, cols, nu, out);
    UOI_CHECK_LAUNCH();
    count_launch();
}

namespace {
// Contiguous rows (ldx == p): one flat loop; otherwise rows over blocks and
// columns over threads.  No division per element.  With a flag, each value's
// exponent field is also tested (all ones = Inf or NaN): one flag write per warp
// that saw a non-finite value.
__global__ void k_to_f32(const double* __restrict__ X, int64_t ldx, int64_t m, int64_t p,
                         float* __restrict__ out, int32_t* flag)
{
    bool bad = false;
    if (ldx == p) {
        const int64_t total = m * p;
#pragma unroll 4
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
             t += (int64_t)gridDim.x * blockDim.x) {
            const double x = __ldg(X + t);
            bad |= ((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF;
            out[t] = f64_to_f32_int(x);
        }
    } else {
        for (int64_t row = blockIdx.x; row < m; row += gridDim.x) {
            const double* xr = X + row * ldx;
            float* orow = out + row * ldx;
#pragma unroll 4
            for (int64_t j = threadIdx.x; j < p; j += blockDim.x) {
                const double x = __ldg(xr + j);
                bad |= ((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF;
                orow[j] = f64_to_f32_int(x);
            }
        }
    }
    if (flag && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}
}  // namespace

void to_f32(const double* X, int64_t ldx, int64_t m, int64_t p, float* out, cudaStream_t s, int32_t* flag)
{
    k_to_f32<<<(unsigned)std::min<int64_t>(ceil_div(m * p, 256), 152 * 64), 256, 0, s>>>(X, ldx, m, p, out,
                                                                                          flag);
    UOI_CHECK_LAUNCH();
    count_launch();
}

}  // namespace uoi
