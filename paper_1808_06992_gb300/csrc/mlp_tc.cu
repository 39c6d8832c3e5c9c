// mlp_tc.cu -- the warm-start network's 512 x 512 hidden-layer products on the
// 5th-generation tensor cores (tcgen05, TMA, TMEM).
//
// C = A B^T with A (M x K) and B (N x K) bf16 row-major (K contiguous), FP32
// accumulation in TMEM, and an epilogue fused per use:
//   forward   pre = acc + b_n, h = gelu(pre): h (bf16, row-major: the next layer's A),
//             h^T (bf16: the weight gradient's B) and pre (FP32, for the backward);
//   backward  da = acc * gelu'(pre): da (bf16, row-major: the next backward
//             product's A) and da^T (bf16: the weight gradient's A);
//   gradient  the FP32 partial sums of one slice of K (rows of the batch), reduced
//             over slices afterwards in a fixed order;
//   forward + head (inference, last hidden layer)  h = gelu(acc + b_n) rounded to
//             bf16 as the forward stores it, then its products with the head's
//             weights, one partial sum per (row, 128 columns): h is never written.
// Tile 128 x 256 (UMMA M = 128, N = 256), k = 32 per stage (64 B of bf16 per row,
// 64-byte swizzle), a 3-stage TMA ring (K is 512: sixteen stages), one CTA per
// tile (cta_group::1) with 256 TMEM columns, two CTAs per SM.  Warp 0 issues the
// TMA loads, warp 1 the MMAs, warps 2-9 drain the accumulator (one tile row and
// half of its columns per thread) and apply the epilogue -- the GELU and the
// stores are the bulk of a layer's time, so eight warps take them.  Rows past M
// are read as zeros (the tensor maps' out-of-range fill) and not written.  Every
// wait is bounded (wait_ns) and reports UOI_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "gelu.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace uoi {

namespace {
using namespace tc;

constexpr int MT_TM = 128;
constexpr int MT_TN = 256;
constexpr int MT_TK = 32;
constexpr int MT_STAGES = 3;
constexpr int MT_A_BYTES = MT_TM * MT_TK * 2;             // 8 KB
constexpr int MT_B_BYTES = MT_TN * MT_TK * 2;             // 16 KB
constexpr int MT_STAGE = MT_A_BYTES + MT_B_BYTES;         // 24 KB
constexpr int MT_SMEM = MT_STAGES * MT_STAGE + 1024;
constexpr int MT_THREADS = 64 + 256;                      // TMA, MMA, 8 epilogue warps
constexpr uint32_t MT_TMEM_COLS = 256;
constexpr int WS_OUT = 3;                                 // outputs of the head (forward + head mode)

enum MlpEpilogue : int32_t { MLP_FORWARD = 0, MLP_BACKWARD = 1, MLP_GRAD_PARTIAL = 2, MLP_FORWARD_HEAD = 3 };

struct MlpGemmArgs {
    int32_t M, N;                 // rows of A / C, columns of C (rows of B)
    int32_t kst_total;            // k stages over the whole K extent
    int32_t kst_slice;            // k stages per CTA along blockIdx.z (gradient slices)
    int32_t mode;                 // MlpEpilogue
    const float* bias;            // forward: N
    float* pre;                   // forward: M x N written (nullable); backward: M x N read
    __nv_bfloat16* out;           // forward / backward: M x N
    __nv_bfloat16* outT;          // forward / backward: N x ldT (nullable)
    int64_t ldT;
    float* part;                  // gradient: slices x M x N
    const __nv_bfloat16* w4;      // forward + head: head weights, WS_OUT rows of N
    float* head;                  // forward + head: (N / 128) slots x M x WS_OUT partial sums
    int32_t* err;
    uint64_t wait_ns = tc::kWaitLimitNs;   // limit of every bounded mbarrier wait
};

__global__ void __launch_bounds__(MT_THREADS, 2)
k_mlp_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, MlpGemmArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[MT_STAGES], empty_bar[MT_STAGES], acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, epi_ok;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * MT_TM, n0 = blockIdx.x * MT_TN;   // N tiles adjacent: they share A
    const int g0 = blockIdx.z * a.kst_slice;
    const int g1 = min(a.kst_total, g0 + a.kst_slice);
    const int nst = max(0, g1 - g0);
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MT_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&acc_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(MT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0 && nst > 0) {
        // ---------------- TMA producer ----------------
        for (int i = 0; i < nst; ++i) {
            const int s = i % MT_STAGES;
            if (i >= MT_STAGES && !mbar_wait(&empty_bar[s], ((i / MT_STAGES) - 1) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            const uint32_t st = sbase + s * MT_STAGE;
            mbar_expect_tx(&full_bar[s], MT_STAGE);
            const int k0 = (g0 + i) * MT_TK;
            tma_load_3d(st, &tmA, &full_bar[s], k0, m0, 0);
            tma_load_3d(st + MT_A_BYTES, &tmB, &full_bar[s], k0, n0, 0);
        }
        if (abort_flag) {
            // let the copies already issued land before the CTA releases its memory
            for (int i = max(0, nst - MT_STAGES); i < nst; ++i)
                mbar_wait(&full_bar[i % MT_STAGES], (i / MT_STAGES) & 1, &abort_flag, a.wait_ns);
        }
    } else if (warp == 1 && lane == 0 && nst > 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = idesc_bf16(MT_TM, MT_TN);
        for (int i = 0; i < nst; ++i) {
            const int s = i % MT_STAGES;
            if (!mbar_wait(&full_bar[s], (i / MT_STAGES) & 1, &abort_flag, a.wait_ns)) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t st = sbase + s * MT_STAGE;
            const uint64_t ad = smem_desc_sw64(st), bd = smem_desc_sw64(st + MT_A_BYTES);
#pragma unroll
            for (int ks = 0; ks < MT_TK / 16; ++ks) {
                const uint64_t adv = (uint64_t)(ks * 32 >> 4);       // 16 bf16 = 32 B along K
                mma_bf16(tmem, ad + adv, bd + adv, idesc, (i | ks) ? 1u : 0u);
            }
            mma_commit(&empty_bar[s]);
        }
        mma_commit(&acc_bar);             // arrives once every MMA issued above has completed
    } else if (warp >= 2) {
        // ---------------- epilogue: one tile row per thread ----------------
        const int quad = warp & 3;                        // TMEM lanes 32*quad .. +31
        const int half = (warp - 2) >> 2;                 // columns 128*half .. +127
        const int m = m0 + quad * 32 + lane;
        // One thread waits for the accumulator while the other epilogue warps sleep
        // on a named barrier: warps that poll take issue slots from the epilogue of
        // the SM's other CTA.
        if (warp == 2 && lane == 0) epi_ok = (nst == 0 || mbar_wait(&acc_bar, 0, &abort_flag, a.wait_ns)) ? 1 : 0;
        named_barrier_sync(1, MT_THREADS - 64);
        if (!epi_ok) {
            if (warp == 2 && lane == 0) {
                abort_flag = 1;
                atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
            }
        } else {
            tc_fence_after();
            float hsum[WS_OUT] = {};
            // one chunk of 16 columns, its accumulators in rv
            auto chunk = [&](const uint32_t (&rv)[16], int cb) {
                if (m >= a.M) return;
                float v[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(rv[t]);
                const int nb = n0 + cb * 16;
                if (a.mode == MLP_GRAD_PARTIAL) {
                    float* dst = a.part + ((int64_t)blockIdx.z * a.M + m) * a.N + nb;
#pragma unroll
                    for (int t = 0; t < 16; t += 4)
                        if (nb + t + 3 < a.N)
                            *reinterpret_cast<float4*>(dst + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
                    return;
                }
                // 16-byte vector loads and stores: a thread owns 16 consecutive columns
                // of one row, so each bf16 row segment is one full 32-byte sector and
                // each FP32 one two.
                float r[16];
                const int64_t off = (int64_t)m * a.N + nb;
                if (a.mode == MLP_FORWARD || a.mode == MLP_FORWARD_HEAD) {
                    const float4* bias4 = reinterpret_cast<const float4*>(a.bias + nb);
#pragma unroll
                    for (int t = 0; t < 16; t += 4) {
                        const float4 b = __ldg(bias4 + t / 4);
                        const float4 pre = make_float4(v[t] + b.x, v[t + 1] + b.y, v[t + 2] + b.z, v[t + 3] + b.w);
                        if (a.pre) *reinterpret_cast<float4*>(a.pre + off + t) = pre;
                        r[t] = gelu_f(pre.x);
                        r[t + 1] = gelu_f(pre.y);
                        r[t + 2] = gelu_f(pre.z);
                        r[t + 3] = gelu_f(pre.w);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 16; t += 4) {
                        const float4 pre = *reinterpret_cast<const float4*>(a.pre + off + t);
                        r[t] = v[t] * gelu_grad_f(pre.x);
                        r[t + 1] = v[t + 1] * gelu_grad_f(pre.y);
                        r[t + 2] = v[t + 2] * gelu_grad_f(pre.z);
                        r[t + 3] = v[t + 3] * gelu_grad_f(pre.w);
                    }
                }
                uint32_t packed[8];
#pragma unroll
                for (int t = 0; t < 16; t += 2) {
                    const __nv_bfloat162 hb = __floats2bfloat162_rn(r[t], r[t + 1]);
                    packed[t / 2] = *reinterpret_cast<const uint32_t*>(&hb);
                }
                if (a.mode == MLP_FORWARD_HEAD) {
                    // the head reads the activations as stored (BF16), so it takes them
                    // after the rounding; h itself is not written
#pragma unroll
                    for (int t = 0; t < 16; t += 2) {
                        const float2 hv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&packed[t / 2]));
#pragma unroll
                        for (int j = 0; j < WS_OUT; ++j) {
                            const float2 wv = __bfloat1622float2(
                                __ldg(reinterpret_cast<const __nv_bfloat162*>(a.w4 + (int64_t)j * a.N + nb + t)));
                            hsum[j] = fmaf(hv.y, wv.y, fmaf(hv.x, wv.x, hsum[j]));
                        }
                    }
                    return;
                }
                uint4* orow = reinterpret_cast<uint4*>(a.out + off);
                orow[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                orow[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                if (a.outT) {
                    // column-major copy: the warp's 32 consecutive rows are adjacent
#pragma unroll
                    for (int t = 0; t < 16; ++t) a.outT[(int64_t)(nb + t) * a.ldT + m] = __float2bfloat16_rn(r[t]);
                }
            };
            // TMEM loads double-buffered: chunk cb + 1 is in flight while cb is computed
            const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
            auto issue = [&](int cb, uint32_t (&rv)[16]) {
                if (nst > 0) {
                    tmem_ld16_issue(trow + (uint32_t)(cb * 16), rv);
                } else {
#pragma unroll
                    for (int t = 0; t < 16; ++t) rv[t] = 0u;
                }
            };
            const int cb0 = half * 8;
            uint32_t ra[16], rb[16];
            issue(cb0, ra);
            tmem_wait16(ra);
            for (int cb = cb0; cb < cb0 + 8; cb += 2) {
                issue(cb + 1, rb);
                chunk(ra, cb);
                tmem_wait16(rb);
                if (cb + 2 < cb0 + 8) issue(cb + 2, ra);
                chunk(rb, cb + 1);
                if (cb + 2 < cb0 + 8) tmem_wait16(ra);
            }
            if (a.mode == MLP_FORWARD_HEAD && m < a.M) {
                float* dst = a.head + (((int64_t)blockIdx.x * 2 + half) * a.M + m) * WS_OUT;
#pragma unroll
                for (int j = 0; j < WS_OUT; ++j) dst[j] = hsum[j];
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MT_TMEM_COLS));
    }
}

// Tensor map over a rows x K bf16 row-major matrix (K contiguous, row stride ld
// elements, a multiple of 8), boxes of 32 x box_rows with the 64-byte swizzle.
CUtensorMap map_rows(const __nv_bfloat16* base, int64_t K, int64_t rows, int64_t ld, int box_rows)
{
    CUtensorMap m;
    cuuint64_t dims[3] = { (cuuint64_t)K, (cuuint64_t)rows, 1u };
    cuuint64_t strides[2] = { (cuuint64_t)(ld * 2), (cuuint64_t)(ld * 2 * rows) };
    cuuint32_t box[3] = { 32u, (cuuint32_t)box_rows, 1u };
    cuuint32_t estr[3] = { 1, 1, 1 };
    CUresult res = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(base), dims,
                               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (res != CUDA_SUCCESS) throw Error(UOI_ERR_CUDA, "cuTensorMapEncodeTiled failed (MLP operand)");
    return m;
}

void launch(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int32_t M, int32_t N,
            int32_t K, int32_t slices, MlpGemmArgs a, cudaStream_t s)
{
    if (K % MT_TK != 0 || N % MT_TN != 0 || lda % 8 != 0 || ldb % 8 != 0)
        throw Error(UOI_ERR_INVALID_ARG, "tensor-core MLP product: K % 32, N % 256, strides % 8 must be 0");
    static std::once_flag once;
    std::call_once(once, [] {
        UOI_CUDA(cudaFuncSetAttribute(k_mlp_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, MT_SMEM));
    });
    const CUtensorMap mA = map_rows(A, K, M, lda, MT_TM);
    const CUtensorMap mB = map_rows(B, K, N, ldb, MT_TN);
    a.M = M;
    a.N = N;
    a.kst_total = K / MT_TK;
    a.kst_slice = (int32_t)ceil_div(a.kst_total, slices);
    if (ceil_div(M, MT_TM) > 65535)
        throw Error(UOI_ERR_INVALID_ARG, "tensor-core MLP product: at most 65535 row tiles per launch");
    const dim3 grid((unsigned)(N / MT_TN), (unsigned)ceil_div(M, MT_TM), (unsigned)slices);
    k_mlp_gemm_tc<<<grid, MT_THREADS, MT_SMEM, s>>>(mA, mB, a);
    UOI_CHECK_LAUNCH();
    count_launch();
}

}  // namespace

bool mlp_tc_available() { return gram_tc_available(); }

void mlp_forward_tc(const __nv_bfloat16* H, int64_t M, const __nv_bfloat16* W, int32_t width,
                    const float* bias, float* pre, __nv_bfloat16* Hn, __nv_bfloat16* HnT, int64_t ldT,
                    int32_t* err, cudaStream_t s)
{
    MlpGemmArgs a;
    a.mode = MLP_FORWARD;
    a.bias = bias; a.pre = pre; a.out = Hn; a.outT = HnT; a.ldT = ldT; a.part = nullptr; a.err = err;
    a.w4 = nullptr; a.head = nullptr;
    launch(H, width, W, width, (int32_t)M, width, width, 1, a, s);
}

void mlp_forward_head_tc(const __nv_bfloat16* H, int64_t M, const __nv_bfloat16* W, int32_t width,
                         const float* bias, const __nv_bfloat16* w4, float* head_part, int32_t* err, cudaStream_t s)
{
    MlpGemmArgs a;
    a.mode = MLP_FORWARD_HEAD;
    a.bias = bias; a.pre = nullptr; a.out = nullptr; a.outT = nullptr; a.ldT = 0; a.part = nullptr; a.err = err;
    a.w4 = w4; a.head = head_part;
    launch(H, width, W, width, (int32_t)M, width, width, 1, a, s);
}

void mlp_backward_tc(const __nv_bfloat16* dA, int64_t M, const __nv_bfloat16* WT, int32_t width,
                     const float* pre_prev, __nv_bfloat16* dAp, __nv_bfloat16* dApT, int64_t ldT, int32_t* err,
                     cudaStream_t s)
{
    MlpGemmArgs a;
    a.mode = MLP_BACKWARD;
    a.bias = nullptr; a.pre = const_cast<float*>(pre_prev); a.out = dAp; a.outT = dApT; a.ldT = ldT;
    a.part = nullptr; a.err = err; a.w4 = nullptr; a.head = nullptr;
    launch(dA, width, WT, width, (int32_t)M, width, width, 1, a, s);
}

void mlp_weight_grad_tc(const __nv_bfloat16* dAT, const __nv_bfloat16* HT, int64_t ld, int64_t rows, int32_t width,
                        int32_t slices, float* part, int32_t* err, cudaStream_t s)
{
    MlpGemmArgs a;
    a.mode = MLP_GRAD_PARTIAL;
    a.bias = nullptr; a.pre = nullptr; a.out = nullptr; a.outT = nullptr; a.ldT = 0; a.part = part; a.err = err;
    a.w4 = nullptr; a.head = nullptr;
    launch(dAT, ld, HT, ld, width, width, (int32_t)ceil_div(rows, MT_TK) * MT_TK, slices, a, s);
}

}  // namespace uoi
