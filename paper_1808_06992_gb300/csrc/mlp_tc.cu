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
//             over slices afterwards in a fixed order.
// Tile 128 x 256 (UMMA M = 128, N = 256), k = 32 per stage (64 B of bf16 per row,
// 64-byte swizzle), a 6-stage TMA ring, one CTA per tile (cta_group::1) with 256
// TMEM columns.  Warp 0 issues the TMA loads, warp 1 the MMAs, warps 2-5 drain
// the accumulator (one tile row per thread) and apply the epilogue.  Rows past M
// are read as zeros (the tensor maps' out-of-range fill) and not written.  Every
// wait is bounded (wait_ns) and reports UOI_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "kernels.h"
#include "tc_common.cuh"

namespace uoi {

namespace {
using namespace tc;

constexpr int MT_TM = 128;
constexpr int MT_TN = 256;
constexpr int MT_TK = 32;
constexpr int MT_STAGES = 6;
constexpr int MT_A_BYTES = MT_TM * MT_TK * 2;             // 8 KB
constexpr int MT_B_BYTES = MT_TN * MT_TK * 2;             // 16 KB
constexpr int MT_STAGE = MT_A_BYTES + MT_B_BYTES;         // 24 KB
constexpr int MT_SMEM = MT_STAGES * MT_STAGE + 1024;
constexpr int MT_THREADS = 64 + 128;                      // TMA, MMA, 4 epilogue warps
constexpr uint32_t MT_TMEM_COLS = 256;

enum MlpEpilogue : int32_t { MLP_FORWARD = 0, MLP_BACKWARD = 1, MLP_GRAD_PARTIAL = 2 };

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
    int32_t* err;
    uint64_t wait_ns = tc::kWaitLimitNs;   // limit of every bounded mbarrier wait
};

__device__ __forceinline__ float gelu_t(float x)
{
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_t(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__global__ void __launch_bounds__(MT_THREADS, 1)
k_mlp_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, MlpGemmArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[MT_STAGES], empty_bar[MT_STAGES], acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * MT_TM, n0 = blockIdx.y * MT_TN;
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
        const int m = m0 + quad * 32 + lane;
        bool ok = true;
        if (nst > 0) ok = mbar_wait(&acc_bar, 0, &abort_flag, a.wait_ns);
        if (!__all_sync(0xffffffffu, ok)) {
            abort_flag = 1;
            atomicCAS(a.err, 0, UOI_ERR_TIMEOUT);
        } else {
            tc_fence_after();
            for (int cb = 0; cb < MT_TN / 16; ++cb) {
                float v[16];
                if (nst > 0) {
                    tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cb * 16), v);
                } else {
#pragma unroll
                    for (int t = 0; t < 16; ++t) v[t] = 0.f;
                }
                if (m >= a.M) continue;
                const int nb = n0 + cb * 16;
                if (a.mode == MLP_GRAD_PARTIAL) {
                    float* dst = a.part + ((int64_t)blockIdx.z * a.M + m) * a.N + nb;
#pragma unroll
                    for (int t = 0; t < 16; t += 4)
                        if (nb + t + 3 < a.N)
                            *reinterpret_cast<float4*>(dst + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
                    continue;
                }
                float r[16];
                if (a.mode == MLP_FORWARD) {
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const float pre = v[t] + a.bias[nb + t];
                        if (a.pre) a.pre[(int64_t)m * a.N + nb + t] = pre;
                        r[t] = gelu_t(pre);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 16; ++t) r[t] = v[t] * gelu_grad_t(a.pre[(int64_t)m * a.N + nb + t]);
                }
                __nv_bfloat16* orow = a.out + (int64_t)m * a.N + nb;
#pragma unroll
                for (int t = 0; t < 16; t += 2)
                    *reinterpret_cast<__nv_bfloat162*>(orow + t) = __floats2bfloat162_rn(r[t], r[t + 1]);
                if (a.outT) {
                    // column-major copy: the warp's 32 consecutive rows are adjacent
#pragma unroll
                    for (int t = 0; t < 16; ++t) a.outT[(int64_t)(nb + t) * a.ldT + m] = __float2bfloat16_rn(r[t]);
                }
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
    const dim3 grid((unsigned)ceil_div(M, MT_TM), (unsigned)(N / MT_TN), (unsigned)slices);
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
    launch(H, width, W, width, (int32_t)M, width, width, 1, a, s);
}

void mlp_backward_tc(const __nv_bfloat16* dA, int64_t M, const __nv_bfloat16* WT, int32_t width,
                     const float* pre_prev, __nv_bfloat16* dAp, __nv_bfloat16* dApT, int64_t ldT, int32_t* err,
                     cudaStream_t s)
{
    MlpGemmArgs a;
    a.mode = MLP_BACKWARD;
    a.bias = nullptr; a.pre = const_cast<float*>(pre_prev); a.out = dAp; a.outT = dApT; a.ldT = ldT;
    a.part = nullptr; a.err = err;
    launch(dA, width, WT, width, (int32_t)M, width, width, 1, a, s);
}

void mlp_weight_grad_tc(const __nv_bfloat16* dAT, const __nv_bfloat16* HT, int64_t ld, int64_t rows, int32_t width,
                        int32_t slices, float* part, int32_t* err, cudaStream_t s)
{
    MlpGemmArgs a;
    a.mode = MLP_GRAD_PARTIAL;
    a.bias = nullptr; a.pre = nullptr; a.out = nullptr; a.outT = nullptr; a.ldT = 0; a.part = part; a.err = err;
    launch(dAT, ld, HT, ld, width, width, (int32_t)ceil_div(rows, MT_TK) * MT_TK, slices, a, s);
}

}  // namespace uoi
