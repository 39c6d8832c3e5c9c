// gemm_tc.cu -- FP32-accurate batched GEMM on the tensor cores, and the
// inverse of a batch of SPD matrices built on it (G3 of the mixed form: the
// cached inverse M = (G/n + rho I)^{-1} that the ADMM x-update multiplies by).
//
// GEMM: D_g = alpha * A_g B_g^T + beta * C_g with A_g (m x k) and B_g (n x k)
// given as two fp16 pieces each: every matrix scaled by an exact power of two
// that puts its largest entry just below 2^10, then v = h + l (residue <=
// 2^-22 |v|); the three products l.H, h.L, h.H (small first) accumulate into a
// double-buffered TMEM accumulator (2 x 256 columns) that 8 epilogue warps drain
// every 64 k into FP32 running sums; the epilogue undoes the two scales.  The
// largest entries come for free: an SPD matrix's largest entry is its largest
// diagonal entry, and the GEMM epilogue reports the largest |D| it writes.  Tiles 128 x 256 (the wide N keeps shared-memory operand traffic below the
// tensor rate), k = 32 per stage (64-byte swizzle), 4-stage TMA ring of 48 KB
// stages, one CTA per SM.  Operands are stored as contiguous 128 x 32 (A) or
// 256 x 32 (B) blocks, [g][row tile][k block][piece][rows][32], so every stage
// is one TMA copy per operand.
//
// Inverse: block (Schur complement) recursion on the SPD matrix
//   A = [A11 A21^T; A21 A22],  X = A11^{-1},  U = A21 X,  S = A22 - A21 U^T,
//   Y = S^{-1},  M21 = -Y U,  M11 = X - U^T M21,  M12 = M21^T,
// which is exact algebra (the block form of the Cholesky-based inverse) with
// every product a large GEMM; blocks of order <= 192 are inverted in shared
// memory by Gauss-Jordan elimination (no pivoting: the pivots are the Schur
// complements' diagonals, positive for SPD A).  S stays SPD for SPD A.
#include <cuda_fp16.h>

#include <algorithm>
#include <exception>
#include <future>
#include <mutex>

#include "kernels.h"
#include "tc_common.cuh"

namespace uoi {

namespace {
using namespace tc;

constexpr int GT_TM = 128;                             // A rows per tile
constexpr int GT_TN = 256;                             // B rows per tile (UMMA N)
constexpr int GT_TK = 32;
constexpr int GT_PIECES = 2;                           // fp16 pieces per operand
constexpr int GT_STAGES = 4;
constexpr int GT_A_BYTES = GT_TM * GT_TK * 2;          // 8 KB per piece
constexpr int GT_B_BYTES = GT_TN * GT_TK * 2;          // 16 KB per piece
constexpr int GT_STAGE = GT_PIECES * GT_A_BYTES + GT_PIECES * GT_B_BYTES;   // 48 KB
constexpr int GT_SMEM = GT_STAGES * GT_STAGE + 1024;
constexpr int GT_EPI_WARPS = 8;
constexpr int GT_THREADS = 64 + 32 * GT_EPI_WARPS;     // producer, MMA, 8 epilogue warps
constexpr uint32_t GT_TMEM_COLS = 512;                 // two 256-column accumulators
constexpr int GT_CHUNK_STAGES = 2;                     // drain every 64 k
constexpr int GT_STG = 132;                            // epilogue staging row (floats)
static_assert(GT_EPI_WARPS * 32 * GT_STG * 4 <= GT_STAGES * GT_STAGE, "staging fits the ring");
constexpr int64_t INV_BASE = 192;                      // shared-memory inverse at or below this order
constexpr int GT_SCALE_EXP = 10;                       // scaled magnitudes stay below 2^10

struct GemmArgs {
    int32_t m, n, kst, MT, NT;
    float alpha, beta;
    const float* C; int64_t ldc, gsc;                  // C may alias D
    float* D; int64_t ldd, gsd;
    const float* ainv;                                 // G: 1 / scale of A_g
    const float* binv;                                 // G: 1 / scale of B_g
    uint32_t* dmax;                                    // G: largest |D_g| (float bits), nullable
    int32_t* err;
    uint64_t wait_ns = tc::kWaitLimitNs;   // limit of every bounded mbarrier wait
};

__device__ __forceinline__ void split2(float x, __half& h, __half& l)
{
    h = __float2half_rn(x);
    l = __float2half_rn(x - __half2float(h));
}

// 2^(GT_SCALE_EXP - e) for m = f 2^e, f in [0.5, 1) (1 for m = 0).
__device__ __forceinline__ float pow2_scale(float m)
{
    if (!(m > 0.f) || !(m < 3.0e38f)) return 1.f;
    int e;
    frexpf(m, &e);
    return ldexpf(1.f, min(120, max(-120, GT_SCALE_EXP - e)));
}

__global__ void __launch_bounds__(GT_THREADS, 1)
k_gemm3_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[GT_STAGES], empty_bar[GT_STAGES], accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x, nt = blockIdx.y, g = blockIdx.z;
    const int nchunks = (a.kst + GT_CHUNK_STAGES - 1) / GT_CHUNK_STAGES;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GT_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&accf_bar[b], 1); mbar_init(&acce_bar[b], 32 * GT_EPI_WARPS); }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(GT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        const int blkA = ((g * a.MT + mt) * a.kst) * GT_PIECES;
        const int blkB = ((g * a.NT + nt) * a.kst) * GT_PIECES;
        for (int s_ = 0; s_ < a.kst; ++s_) {
            const int s = s_ % GT_STAGES;
            if (s_ >= GT_STAGES && !mbar_wait(&empty_bar[s], ((s_ / GT_STAGES) - 1) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            const uint32_t st = sbase + s * GT_STAGE;
            mbar_expect_tx(&full_bar[s], GT_STAGE);
            tma_load_3d(st, &tmA, &full_bar[s], 0, 0, blkA + GT_PIECES * s_);
            tma_load_3d(st + GT_PIECES * GT_A_BYTES, &tmB, &full_bar[s], 0, 0, blkB + GT_PIECES * s_);
        }
        if (abort_flag)
            for (int s_ = max(0, a.kst - GT_STAGES); s_ < a.kst; ++s_)
                mbar_wait(&full_bar[s_ % GT_STAGES], (s_ / GT_STAGES) & 1, &abort_flag, a.wait_ns);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer: all three products into accumulator b ----------------
        const uint32_t idesc = idesc_f16(GT_TM, GT_TN);
        int s_ = 0;
        for (int c = 0; c < nchunks && !abort_flag; ++c) {
            const int b = c & 1;
            if (c >= 2 && !mbar_wait(&acce_bar[b], ((c >> 1) - 1) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(b * GT_TN);
            const int send = min(a.kst, (c + 1) * GT_CHUNK_STAGES);
            bool first = true;
            for (; s_ < send; ++s_) {
                const int s = s_ % GT_STAGES;
                if (!mbar_wait(&full_bar[s], (s_ / GT_STAGES) & 1, &abort_flag, a.wait_ns)) {
                    abort_flag = 1;
                    atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t st = sbase + s * GT_STAGE;
                const uint64_t Ah = smem_desc_sw64(st), Al = smem_desc_sw64(st + GT_A_BYTES);
                const uint32_t bb = st + GT_PIECES * GT_A_BYTES;
                const uint64_t Bh = smem_desc_sw64(bb), Bl = smem_desc_sw64(bb + GT_B_BYTES);
#pragma unroll
                for (int ks = 0; ks < GT_TK / 16; ++ks) {
                    const uint64_t adv = (uint64_t)(ks * 32 >> 4);
                    // small products first, h.H last (adds the largest term to the smallest sum)
                    mma_bf16(d, Al + adv, Bh + adv, idesc, first ? 0u : 1u);
                    mma_bf16(d, Ah + adv, Bl + adv, idesc, 1u);
                    mma_bf16(d, Ah + adv, Bh + adv, idesc, 1u);
                    first = false;
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
        // ---------------- epilogue: TMEM -> FP32 running sums -> D ----------------
        const int quad = warp & 3;                       // TMEM lanes 32*quad .. +31
        const int half = (warp - 2) >> 2;                // columns 128*half .. +127
        const float ar = a.alpha * (a.ainv[g] * a.binv[g]);   // read while the products run
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
                tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * GT_TN + half * 128 + cb * 16), v);
#pragma unroll
                for (int t = 0; t < 16; ++t) acc[cb * 16 + t] += v[t];
            }
            tc_fence_before();
            mbar_arrive(&acce_bar[b]);
        }
        {
            int dummy = 0;
            if (!abort_flag) mbar_wait(&done_bar, 0, &dummy, a.wait_ns);   // the ring is idle from here
        }
        __syncwarp();
        // stage the warp's 32 x 128 block in shared memory, then write whole rows
        float* stage = reinterpret_cast<float*>(smem_raw + (sbase - smem_u32(smem_raw))) +
                       (warp - 2) * 32 * GT_STG;
#pragma unroll
        for (int c4 = 0; c4 < 32; ++c4)
            *reinterpret_cast<float4*>(stage + lane * GT_STG + 4 * c4) =
                make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
        __syncwarp();
        if (!abort_flag) {
            const int j = nt * GT_TN + half * 128 + 4 * lane;
            const int i0 = mt * GT_TM + quad * 32;
            const int nrow = max(0, min(32, a.m - i0));
            float dm = 0.f;
            for (int r0 = 0; r0 < nrow; r0 += 8) {
                // C of eight rows read before any of them is written (all loads in
                // flight at once; D may be C itself, element for element)
                float cv[8][4];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        cv[u][t] = (a.C && r0 + u < nrow && j + t < a.n)
                                       ? a.C[(int64_t)g * a.gsc + (int64_t)(i0 + r0 + u) * a.ldc + j + t]
                                       : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int rr = r0 + u;
                    if (rr >= nrow) break;
                    const float4 v = *reinterpret_cast<const float4*>(stage + rr * GT_STG + 4 * lane);
                    float r4[4] = { v.x, v.y, v.z, v.w };
                    float* drow = a.D + (int64_t)g * a.gsd + (int64_t)(i0 + rr) * a.ldd;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (j + t < a.n) {
                            float r = ar * r4[t];
                            if (a.C) r += a.beta * cv[u][t];
                            drow[j + t] = r;
                            dm = fmaxf(dm, fabsf(r));
                        }
                    }
                }
            }
            if (a.dmax) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
                if (lane == 0 && dm > 0.f) atomicMax(&a.dmax[g], __float_as_uint(dm));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GT_TMEM_COLS));
    }
}

// One operand split: the two fp16 pieces of op(S_g) (rows x K; op = transpose if
// trans), scaled by the power of two of S_g's largest magnitude smax[g] (float
// bits), in blocks of rt x 32, ordered [g][row tile][k block][piece][rt][32], zero
// padded to the tile multiples; sinv[g] = 1 / scale.  S_g element (i, k) is at
// src[g*gs + i*ld + k] (or src[g*gs + k*ld + i] transposed).
constexpr int SPLIT_KC = 4;                            // 32-k blocks per CTA
struct SplitJob {
    const float* src;
    int64_t ld, gs;
    int32_t rows, K, trans, rt;
    int64_t rpad, kpad;
    const uint32_t* smax;
    float* sinv;
    __half* out;
    int32_t nbx, nby;                                  // CTAs per group: rpad / 32 x ceil(kpad / (32 SPLIT_KC))
};
// Up to two independent splits in one launch: CTA b < first1 works on job 0, the
// rest on job 1 (each job's CTAs ordered [g][k group][row block]).
struct SplitJobs {
    SplitJob j[2];
    int64_t first1;
};

// 32 x 32 tiles through shared memory, so that both the read (along the source's
// contiguous index) and the write (along k) are coalesced.  Block (32, 8); a CTA
// covers 32 rows x SPLIT_KC blocks of 32 k, and every thread issues all of its
// 4 x SPLIT_KC loads before its first store, so more bytes are in flight per SM.
__global__ void k_split_blocks(const __grid_constant__ SplitJobs J, int32_t G)
{
    __shared__ float tile[SPLIT_KC][32][33];            // [k block][k local][i local]
    const int64_t b = blockIdx.x;
    const int jj = b < J.first1 ? 0 : 1;
    const SplitJob& P = J.j[jj];
    const int64_t local = b - (jj ? J.first1 : 0);
    const int64_t per_g = (int64_t)P.nbx * P.nby;
    const int64_t g = local / per_g, rem = local % per_g;
    const int64_t bx = rem % P.nbx, by = rem / P.nbx;
    const int64_t i0 = bx * 32, kb0 = by * SPLIT_KC;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int32_t rows = P.rows, K = P.K, rt = P.rt;
    const int64_t ld = P.ld, rpad = P.rpad, kpad = P.kpad;
    const float* sg = P.src + g * P.gs;
    const float sc = pow2_scale(__uint_as_float(P.smax[g]));
    if (bx == 0 && by == 0 && tx == 0 && ty == 0) P.sinv[g] = 1.f / sc;
    const int64_t kst = kpad / GT_TK;
    float v[SPLIT_KC][4];
#pragma unroll
    for (int c = 0; c < SPLIT_KC; ++c) {
        const int64_t k0 = (kb0 + c) * 32;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = ty + 8 * u;
            if (P.trans) {
                const int64_t i = i0 + tx, k = k0 + j;
                v[c][u] = (i < rows && k < K) ? sg[k * ld + i] : 0.f;
            } else {
                const int64_t i = i0 + j, k = k0 + tx;
                v[c][u] = (i < rows && k < K) ? sg[i * ld + k] : 0.f;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < SPLIT_KC; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = ty + 8 * u;
            if (P.trans) tile[c][j][tx] = v[c][u];
            else tile[c][tx][j] = v[c][u];
        }
    __syncthreads();
    // write: thread (row r, k quad kq) splits four consecutive k of one row and
    // stores 8-byte runs of each piece (conflict-free reads: bank = kq + u + r)
    const int64_t RT = rpad / rt;
    const int t = ty * 32 + tx, r = t >> 3, kq = (t & 7) << 2;
    const int64_t i = i0 + r;
#pragma unroll
    for (int c = 0; c < SPLIT_KC; ++c) {
        const int64_t kb = kb0 + c;
        if (kb >= kst) break;
        const int64_t k = kb * 32 + kq;
        __half h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) split2(tile[c][kq + u][r] * sc, h[u], l[u]);
        const int64_t blk = ((g * RT + i / rt) * kst + kb) * GT_PIECES;
        const int64_t o = (blk * rt + i % rt) * GT_TK + k % GT_TK;             // multiple of 4
        if (!UOI_IN_BOUNDS(o + rt * GT_TK + 3, (int64_t)G * rpad * kpad * GT_PIECES, 401)) return;
        const __half2 h01 = __halves2half2(h[0], h[1]), h23 = __halves2half2(h[2], h[3]);
        const __half2 l01 = __halves2half2(l[0], l[1]), l23 = __halves2half2(l[2], l[3]);
        *reinterpret_cast<uint2*>(P.out + o) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
        *reinterpret_cast<uint2*>(P.out + o + rt * GT_TK) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
    }
}

// out[g] = largest diagonal entry of the SPD block A_g (n x n), as float bits:
// the largest magnitude of an SPD matrix (|a_ij| <= sqrt(a_ii a_jj)).
__global__ void k_diag_max(const float* A, int64_t lda, int64_t gsa, int64_t n, uint32_t* out)
{
    __shared__ float red[32];
    const int64_t g = blockIdx.x;
    float m = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(A[g * gsa + i * lda + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        out[g] = __float_as_uint(fmaxf(m, red[0]));
    }
}

// dst block (n1 x n2) = src block^T (n2 x n1), per group.
__global__ void k_transpose_block(const float* src, int64_t lds, float* dst, int64_t ldd, int64_t gs,
                                  int32_t n1, int32_t n2)
{
    __shared__ float tile[32][33];
    const int g = blockIdx.z;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;    // bx over n1 (dst rows), by over n2
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int r = by + yy, c = bx + threadIdx.x;           // src row r (< n2), col c (< n1)
        if (r < n2 && c < n1) tile[yy][threadIdx.x] = src[(int64_t)g * gs + (int64_t)r * lds + c];
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        const int r = bx + yy, c = by + threadIdx.x;           // dst row r (< n1), col c (< n2)
        if (r < n1 && c < n2) dst[(int64_t)g * gs + (int64_t)r * ldd + c] = tile[threadIdx.x][yy];
    }
}

// Device scratch of one run of the recursion, taken in last-in-first-out order
// from one allocation sized beforehand by inv_scratch_bytes: nothing is allocated
// or freed inside the recursion.  Taking more than the capacity throws.
struct InvScratch {
    char* base = nullptr;
    size_t cap = 0, top = 0;
    template <typename T> T* take(int64_t count)
    {
        const size_t bytes = ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
        if (top + bytes > cap) throw Error(UOI_ERR_OOM, "tensor-core inverse: scratch plan exceeded");
        T* q = reinterpret_cast<T*>(base + top);
        top += bytes;
        return q;
    }
};

size_t scratch_round(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

struct Pieces {
    __half* buf = nullptr;
    float* sinv = nullptr;         // G: 1 / scale
    CUtensorMap map;
    int32_t tiles = 0, kst = 0;
};

// Scratch bytes of one operand's pieces (the fp16 pieces and the G inverse scales).
size_t pieces_bytes(int64_t rows, int64_t K, int32_t rt, int32_t G)
{
    const int64_t rpad = ceil_div(rows, rt) * rt, kpad = ceil_div(K, GT_TK) * GT_TK;
    return scratch_round(sizeof(__half) * GT_PIECES * (size_t)G * rpad * kpad) +
           scratch_round(sizeof(float) * (size_t)G);
}

// Plan the split of op(S) into scaled pieces for a GEMM operand with row tiles of
// rt: scratch for the pieces and scales, the launch job (smax: G, float bits, each
// S_g's largest magnitude) and the tensor map.  split_pieces launches the jobs.
void plan_pieces(Pieces& P, SplitJob& J, InvScratch& W, const float* src, int64_t ld, int64_t gs, int32_t rows,
                 int32_t K, bool trans, int32_t rt, int32_t G, const uint32_t* smax)
{
    const int64_t rpad = ceil_div(rows, rt) * rt, kpad = ceil_div(K, GT_TK) * GT_TK;
    P.tiles = (int32_t)(rpad / rt);
    P.kst = (int32_t)(kpad / GT_TK);
    P.buf = W.take<__half>(GT_PIECES * (int64_t)G * rpad * kpad);
    P.sinv = W.take<float>(G);
    J.src = src; J.ld = ld; J.gs = gs;
    J.rows = rows; J.K = K; J.trans = trans ? 1 : 0; J.rt = rt;
    J.rpad = rpad; J.kpad = kpad;
    J.smax = smax; J.sinv = P.sinv; J.out = P.buf;
    J.nbx = (int32_t)(rpad / 32);
    J.nby = (int32_t)ceil_div(kpad / 32, SPLIT_KC);
    // blocks of rt x 32 fp16 (64-byte rows); two consecutive blocks per stage
    CUtensorMap m;
    cuuint64_t dims[3] = { 32u, (cuuint64_t)rt, (cuuint64_t)((int64_t)G * P.tiles * P.kst * GT_PIECES) };
    cuuint64_t strides[2] = { 64u, (cuuint64_t)rt * 64u };
    cuuint32_t box[3] = { 32u, (cuuint32_t)rt, (cuuint32_t)GT_PIECES };
    cuuint32_t estr[3] = { 1, 1, 1 };
    CUresult res = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, P.buf, dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (res != CUDA_SUCCESS) throw Error(UOI_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    P.map = m;
}

// One launch for one or two planned splits (independent of each other).
void split_pieces(const SplitJob& a, const SplitJob* b, int32_t G, cudaStream_t s)
{
    SplitJobs J;
    J.j[0] = a;
    J.j[1] = b ? *b : a;
    J.first1 = (int64_t)G * a.nbx * a.nby;
    const int64_t total = J.first1 + (b ? (int64_t)G * b->nbx * b->nby : 0);
    k_split_blocks<<<(unsigned)total, dim3(32, 8), 0, s>>>(J, G);
    UOI_CHECK_LAUNCH();
    count_launch();
}

// D = alpha A B^T + beta C with A (m x k) and B (n x k) in pieces; dmax (G,
// nullable, zeroed by the caller) receives the largest |D_g| as float bits.
void gemm3(const Pieces& A, const Pieces& B, int32_t m, int32_t n, int32_t G, float alpha, float beta,
           const float* C, int64_t ldc, int64_t gsc, float* D, int64_t ldd, int64_t gsd, int32_t* err,
           cudaStream_t s, uint32_t* dmax = nullptr)
{
    if (A.kst != B.kst) throw Error(UOI_ERR_INVALID_ARG, "gemm3: operand k extents differ");
    static std::once_flag once;
    std::call_once(once, [] {
        UOI_CUDA(cudaFuncSetAttribute(k_gemm3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM));
    });
    GemmArgs a;
    a.m = m; a.n = n; a.kst = A.kst; a.MT = A.tiles; a.NT = B.tiles;
    a.alpha = alpha; a.beta = beta;
    a.C = C; a.ldc = ldc; a.gsc = gsc;
    a.D = D; a.ldd = ldd; a.gsd = gsd;
    a.ainv = A.sinv;
    a.binv = B.sinv;
    a.dmax = dmax;
    a.err = err;
    const dim3 grid((unsigned)ceil_div(m, GT_TM), (unsigned)ceil_div(n, GT_TN), (unsigned)G);
    k_gemm3_tc<<<grid, GT_THREADS, GT_SMEM, s>>>(A.map, B.map, a);
    UOI_CHECK_LAUNCH();
    count_launch();
}

// In-place blocked Gauss-Jordan inverse of one SPD block per CTA (n <= INV_BASE =
// 192), in steps of 32 pivots (no pivoting: the pivots are Schur-complement
// diagonals, positive for SPD A).  1024 threads; thread (ty, tx) owns the
// elements (ty + 32u, tx + 32w), u, w < R, in registers.  Step K works on row and
// column block K (indices 32K .. 32K + 31):
//   P = A_KK^{-1}                        (one warp, in registers, by shuffles)
//   A_KJ <- P A_KJ             (J != K)  (block row K; each warp one of its rows)
//   A_IJ <- A_IJ - A_IK A_KJ   (I, J != K; A_IK before the step, A_KJ after it)
//   A_IK <- -A_IK P            (I != K)
//   A_KK <- P
// which leaves A^{-1} after the last step (the block form of the pivot-by-pivot
// Gauss-Jordan elimination: the same products, four barriers per 32 pivots
// instead of one per pivot).  Rows and columns past n hold zeros and the padded
// part of the last diagonal block is inverted as the identity, so they never
// reach the n x n result.  A pivot <= 0 sets status UOI_ERR_NOT_PD (where = g0 + group).
constexpr int GJ_LD = 33;                              // shared rows: conflict-free columns
template <int R>
constexpr size_t gj_smem_bytes() { return sizeof(float) * (size_t)(3 * 32 * R * GJ_LD + 32 * GJ_LD); }

// P = inverse of the bk x bk diagonal block whose row k, column l is at
// D[k * GJ_LD + l] (identity past bk), by one warp: lane l holds column l in
// registers and each of the 32 pivots is one round of shuffles.  Returns false
// when a pivot is not positive.  Not inlined, so that the caller's register tile
// is saved around it by the one warp that calls it instead of being squeezed.
__device__ __noinline__ bool gj_invert_diag(const float* D, float* P, int bk)
{
    const int tx = threadIdx.x & 31;
    float d[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) d[k] = (k < bk && tx < bk) ? D[k * GJ_LD + tx] : (k == tx ? 1.f : 0.f);
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float piv = __shfl_sync(0xffffffffu, d[k], k);
        ok = ok && piv > 0.f;
        const float inv = 1.f / piv;
        const float r = (tx == k) ? inv : d[k] * inv;           // row k / pivot
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float c = __shfl_sync(0xffffffffu, d[i], k);   // column k
            d[i] = (i == k) ? r : fmaf(-c, r, tx == k ? 0.f : d[i]);
        }
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) P[k * GJ_LD + tx] = d[k];
    return ok;
}

template <int R>
__global__ void __launch_bounds__(1024) k_spd_inverse_blocked(const float* A, int64_t lda, int64_t gsa,
                                                              float* M, int64_t ldm, int64_t gsm, int n,
                                                              int g0, DevStatus* st)
{
    extern __shared__ float sm[];
    float* colK = sm;                           // [32R][LD]: colK[i][k] = A(i, 32K + k) before step K
    float* rowT = colK + 32 * R * GJ_LD;        // [32R][LD]: rowT[j][k] = A(32K + k, j) before step K
    float* rowN = rowT + 32 * R * GJ_LD;        // [32R][LD]: rowN[j][k] = (P A_K.)(k, j)
    float* P = rowN + 32 * R * GJ_LD;           // [32][LD]:  P[k][l] = (A_KK^{-1})(k, l)
    __shared__ int bad;
    const int g = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const float* a = A + (int64_t)g * gsa;
    float v[R][R];
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int w = 0; w < R; ++w) {
            const int i = ty + 32 * u, j = tx + 32 * w;
            v[u][w] = (i < n && j < n) ? a[(int64_t)i * lda + j] : 0.f;
        }
    if (threadIdx.x == 0) bad = 0;
    const int nblk = (n + 31) / 32;
#pragma unroll
    for (int K = 0; K < R; ++K) {
        if (K >= nblk) break;
        __syncthreads();                        // the last step's readers are done
#pragma unroll
        for (int u = 0; u < R; ++u) colK[(ty + 32 * u) * GJ_LD + tx] = v[u][K];
#pragma unroll
        for (int w = 0; w < R; ++w) rowT[(tx + 32 * w) * GJ_LD + ty] = v[K][w];
        __syncthreads();
        if (ty == 0) {
            const bool ok = gj_invert_diag(colK + 32 * K * GJ_LD, P, min(32, n - 32 * K));
            if (!ok && tx == 0) bad = 1;
        }
        __syncthreads();
        if (bad) {
            if (threadIdx.x == 0) dev_fail(st, UOI_ERR_NOT_PD, g0 + g);
            return;                             // same decision in every thread
        }
        // block row K: this warp's row 32K + ty becomes row ty of P A_K.
#pragma unroll
        for (int w = 0; w < R; ++w)
            if (w != K) v[K][w] = 0.f;
#pragma unroll 2
        for (int k = 0; k < 32; ++k) {
            const float pk = P[ty * GJ_LD + k];
#pragma unroll
            for (int w = 0; w < R; ++w)
                if (w != K) v[K][w] = fmaf(pk, rowT[(tx + 32 * w) * GJ_LD + k], v[K][w]);
        }
#pragma unroll
        for (int w = 0; w < R; ++w)
            if (w != K) rowN[(tx + 32 * w) * GJ_LD + ty] = v[K][w];
        v[K][K] = P[ty * GJ_LD + tx];
        __syncthreads();
        // every other block row: A_IJ -= A_IK (P A_KJ), A_IK = -A_IK P
#pragma unroll
        for (int u = 0; u < R; ++u)
            if (u != K) v[u][K] = 0.f;
#pragma unroll 1
        for (int k = 0; k < 32; ++k) {
            float r[R];
#pragma unroll
            for (int w = 0; w < R; ++w)
                r[w] = (w == K) ? P[k * GJ_LD + tx] : rowN[(tx + 32 * w) * GJ_LD + k];
#pragma unroll
            for (int u = 0; u < R; ++u) {
                if (u == K) continue;
                const float c = colK[(ty + 32 * u) * GJ_LD + k];
#pragma unroll
                for (int w = 0; w < R; ++w) v[u][w] = fmaf(-c, r[w], v[u][w]);
            }
        }
    }
    float* mo = M + (int64_t)g * gsm;
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int w = 0; w < R; ++w) {
            const int i = ty + 32 * u, j = tx + 32 * w;
            if (i < n && j < n) mo[(int64_t)i * ldm + j] = v[u][w];
        }
}

template <int R>
void launch_inverse_blocked(const float* A, int64_t ldA, int64_t gsA, float* Mout, int64_t ldM, int64_t gsM,
                            int64_t n, int32_t G, int32_t g0, DevStatus* st, cudaStream_t s)
{
    static std::once_flag once;
    std::call_once(once, [] {
        UOI_CUDA(cudaFuncSetAttribute(k_spd_inverse_blocked<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)gj_smem_bytes<R>()));
    });
    k_spd_inverse_blocked<R><<<(unsigned)G, 1024, gj_smem_bytes<R>(), s>>>(A, ldA, gsA, Mout, ldM, gsM,
                                                                           (int)n, g0, st);
}

void inv_base(const float* A, int64_t ldA, int64_t gsA, float* Mout, int64_t ldM, int64_t gsM,
              int64_t n, int32_t G, int32_t g0, DevStatus* st, cudaStream_t s)
{
    if (n <= 64)
        launch_inverse_blocked<2>(A, ldA, gsA, Mout, ldM, gsM, n, G, g0, st, s);
    else if (n <= 128)
        launch_inverse_blocked<4>(A, ldA, gsA, Mout, ldM, gsM, n, G, g0, st, s);
    else
        launch_inverse_blocked<6>(A, ldA, gsA, Mout, ldM, gsM, n, G, g0, st, s);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void diag_max(const float* A, int64_t lda, int64_t gsa, int64_t n, int32_t G, uint32_t* out, cudaStream_t s)
{
    k_diag_max<<<(unsigned)G, 256, 0, s>>>(A, lda, gsa, n, out);
    UOI_CHECK_LAUNCH();
    count_launch();
}

// Split point of the recursion: the leading block, a multiple of the GEMM's row tile.
int64_t inv_split(int64_t n) { return ceil_div(n / 2, GT_TM) * GT_TM; }

// Peak scratch of inv_rec(n, G): the same takes in the same order as inv_rec.
size_t inv_scratch_bytes(int64_t n, int32_t G)
{
    if (n <= INV_BASE) return 0;
    const int64_t p1 = inv_split(n), p2 = n - p1;
    const size_t mx = scratch_round(sizeof(uint32_t) * 5 * (size_t)G);
    const size_t U = scratch_round(sizeof(float) * (size_t)G * p2 * p1);
    const size_t S = scratch_round(sizeof(float) * (size_t)G * p2 * p2);
    const size_t prod_u_s = pieces_bytes(p2, p1, GT_TM, G) + pieces_bytes(p1, p1, GT_TN, G) +
                            pieces_bytes(p2, p1, GT_TN, G);                       // pa, pb, pu
    const size_t prod_m21 = pieces_bytes(p2, p2, GT_TM, G) + pieces_bytes(p1, p2, GT_TN, G);   // py, put
    const size_t prod_m11 = pieces_bytes(p1, p2, GT_TM, G) + pieces_bytes(p1, p2, GT_TN, G);   // pua, pmt
    size_t peak = inv_scratch_bytes(p1, G);                                     // X = A11^{-1}
    peak = std::max(peak, U + S + std::max(prod_u_s, inv_scratch_bytes(p2, G)));  // U, S, then Y = S^{-1}
    peak = std::max(peak, U + std::max(prod_m21, prod_m11));
    return mx + peak;
}

// g0: index of the first of the G systems in the caller's batch (for error reports).
void inv_rec(const float* A, int64_t ldA, int64_t gsA, float* M, int64_t ldM, int64_t gsM, int64_t n,
             int32_t G, int32_t g0, DevStatus* st, int32_t* err, InvScratch& W, cudaStream_t s)
{
    if (n <= INV_BASE) {
        inv_base(A, ldA, gsA, M, ldM, gsM, n, G, g0, st, s);
        return;
    }
    const size_t top0 = W.top;
    const int64_t p1 = inv_split(n), p2 = n - p1;
    const float* A21 = A + p1 * ldA;
    const float* A22 = A + p1 * ldA + p1;
    float* X = M;                                  // M11 block, holds X = A11^{-1} first
    float* M21 = M + p1 * ldM;
    float* M12 = M + p1;
    float* Y = M + p1 * ldM + p1;
    // largest magnitudes of the split operands (float bits per group): A, X, Y are
    // SPD (their largest diagonal entry), U and M21 come from the GEMM epilogues
    uint32_t* mA = W.take<uint32_t>(5 * (int64_t)G);
    UOI_CUDA(cudaMemsetAsync(mA, 0, sizeof(uint32_t) * 5 * (size_t)G, s));
    uint32_t* mX = mA + G;
    uint32_t* mU = mA + 2 * G;
    uint32_t* mY = mA + 3 * G;
    uint32_t* mM21 = mA + 4 * G;
    diag_max(A, ldA, gsA, n, G, mA, s);
    // X = A11^{-1}
    inv_rec(A, ldA, gsA, X, ldM, gsM, p1, G, g0, st, err, W, s);
    diag_max(X, ldM, gsM, p1, G, mX, s);
    // U = A21 X   (p2 x p1)
    float* U = W.take<float>((int64_t)G * p2 * p1);
    const size_t top_u = W.top;
    float* S = W.take<float>((int64_t)G * p2 * p2);
    const size_t top_s = W.top;
    {
        Pieces pa, pb;
        SplitJob ja, jb;
        plan_pieces(pa, ja, W, A21, ldA, gsA, (int32_t)p2, (int32_t)p1, false, GT_TM, G, mA);
        plan_pieces(pb, jb, W, X, ldM, gsM, (int32_t)p1, (int32_t)p1, false, GT_TN, G, mX);
        split_pieces(ja, &jb, G, s);
        gemm3(pa, pb, (int32_t)p2, (int32_t)p1, G, 1.f, 0.f, nullptr, 0, 0, U, p1, p2 * p1, err, s, mU);
        // S = A22 - A21 U^T   (p2 x p2)
        Pieces pu;
        SplitJob ju;
        plan_pieces(pu, ju, W, U, p1, p2 * p1, (int32_t)p2, (int32_t)p1, false, GT_TN, G, mU);
        split_pieces(ju, nullptr, G, s);
        gemm3(pa, pu, (int32_t)p2, (int32_t)p2, G, -1.f, 1.f, A22, ldA, gsA, S, p2, p2 * p2, err, s);
    }
    W.top = top_s;
    // Y = S^{-1}
    inv_rec(S, p2, p2 * p2, Y, ldM, gsM, p2, G, g0, st, err, W, s);
    W.top = top_u;                                 // S is no longer needed
    diag_max(Y, ldM, gsM, p2, G, mY, s);
    {
        // M21 = -Y U   (p2 x p1): A = Y (p2 x p2), B rows = columns of U
        Pieces py, put;
        SplitJob jy, jut;
        plan_pieces(py, jy, W, Y, ldM, gsM, (int32_t)p2, (int32_t)p2, false, GT_TM, G, mY);
        plan_pieces(put, jut, W, U, p1, p2 * p1, (int32_t)p1, (int32_t)p2, true, GT_TN, G, mU);
        split_pieces(jy, &jut, G, s);
        gemm3(py, put, (int32_t)p2, (int32_t)p1, G, -1.f, 0.f, nullptr, 0, 0, M21, ldM, gsM, err, s, mM21);
    }
    W.top = top_u;
    {
        // M11 = X - U^T M21   (p1 x p1): A rows = columns of U, B rows = columns of M21
        Pieces pua, pmt;
        SplitJob jua, jmt;
        plan_pieces(pua, jua, W, U, p1, p2 * p1, (int32_t)p1, (int32_t)p2, true, GT_TM, G, mU);
        plan_pieces(pmt, jmt, W, M21, ldM, gsM, (int32_t)p1, (int32_t)p2, true, GT_TN, G, mM21);
        split_pieces(jua, &jmt, G, s);
        gemm3(pua, pmt, (int32_t)p1, (int32_t)p1, G, -1.f, 1.f, X, ldM, gsM, X, ldM, gsM, err, s);
    }
    W.top = top0;
    // M12 = M21^T
    k_transpose_block<<<dim3((unsigned)ceil_div(p1, 32), (unsigned)ceil_div(p2, 32), (unsigned)G),
                        dim3(32, 8), 0, s>>>(M21, ldM, M12, ldM, gsM, (int32_t)p1, (int32_t)p2);
    UOI_CHECK_LAUNCH();
    count_launch();
}

// The recursion for G systems on stream s, with its scratch taken from one
// allocation on s.
void inv_chain(const float* A, int64_t p, int32_t G, int32_t g0, float* M, DevStatus* st, int32_t* err,
               cudaStream_t s)
{
    InvScratch W;
    W.cap = inv_scratch_bytes(p, G);
    DevBuf ws(W.cap, s);
    W.base = ws.as<char>();
    inv_rec(A, p, p * p, M, p, p * p, p, G, g0, st, err, W, s);
}

}  // namespace

bool inverse_tc_available() { return gram_tc_available(); }

void spd_inverse_tc(const float* A, int64_t p, int32_t G, float* M, DevStatus* st, cudaStream_t s)
{
    DevBuf err(sizeof(int32_t), s);
    UOI_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), s));
    // Below the top levels the recursion is a chain of short launches (leaves of one
    // CTA per system, GEMMs of one tile per system) whose time does not shrink with
    // the batch.  Two halves of a batch of 8 or more therefore run as two chains side
    // by side, each enqueued by its own host thread: the short launches of one fill
    // the SMs the other leaves idle.  Each system's arithmetic is unchanged.  Not on
    // the workers of a batch of fits, which already share the device.
    const int32_t G2 = (G >= 8 && p > INV_BASE && !g_fit_in_batch) ? G / 2 : 0, G1 = G - G2;
    if (G2 == 0) {
        inv_chain(A, p, G, 0, M, st, err.as<int32_t>(), s);
    } else {
        const int64_t pp = p * p;
        cudaStream_t side = side_stream();
        int dev = 0;
        UOI_CUDA(cudaGetDevice(&dev));
        cudaEvent_t ready = nullptr, done = nullptr;
        UOI_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        UOI_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        UOI_CUDA(cudaEventRecord(ready, s));
        UOI_CUDA(cudaStreamWaitEvent(side, ready, 0));
        int32_t* e = err.as<int32_t>();
        std::future<int64_t> second = std::async(std::launch::async, [=]() -> int64_t {
            UOI_CUDA(cudaSetDevice(dev));
            const int64_t l0 = g_launches;               // this thread's own counter
            inv_chain(A + G1 * pp, p, G2, G1, M + G1 * pp, st, e, side);
            return g_launches - l0;
        });
        std::exception_ptr first_err;
        try {
            inv_chain(A, p, G1, 0, M, st, e, s);
        } catch (...) {
            first_err = std::current_exception();
        }
        std::exception_ptr second_err;
        try {
            count_launch(second.get());
        } catch (...) {
            second_err = std::current_exception();
        }
        UOI_CUDA(cudaEventRecord(done, side));
        UOI_CUDA(cudaStreamWaitEvent(s, done, 0));
        cudaEventDestroy(ready);
        cudaEventDestroy(done);
        if (first_err) std::rethrow_exception(first_err);
        if (second_err) std::rethrow_exception(second_err);
    }
    int32_t herr = 0;
    UOI_CUDA(cudaMemcpyAsync(&herr, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error(herr, "tensor-core inverse: a bounded pipeline wait expired");
}

}  // namespace uoi
