// tile.cuh -- a 64x64 CUDA-core tile product shared by the FP64/FP32 kernels.
#pragma once

#include "common.cuh"

namespace uoi {

// acc[u][v] += sum_{k in [k0,k1)} A(i0 + ty + 16u, k) * B(k, j0 + tx + 16v)
// for a 256-thread block (tx = tid % 16, ty = tid / 16).  fa(il, k) and fb(k, jl)
// return operand values for local row il / column jl in [0, 64) (zero outside).
// AK / BK: the operand is contiguous along k in memory (rows of K values), so
// consecutive threads load consecutive k; otherwise consecutive rows/columns.
template <typename T, bool AK = false, bool BK = false, typename FA, typename FB>
__device__ __forceinline__ void tile64_acc(T (&acc)[4][4], const FA& fa, const FB& fb, int64_t k0,
                                           int64_t k1)
{
    constexpr int TK = sizeof(T) == 8 ? 8 : 16;   // keeps FP64 users under 48 KB static smem
    __shared__ T As[TK][65];
    __shared__ T Bs[TK][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int64_t kb = k0; kb < k1; kb += TK) {
        for (int e = threadIdx.x; e < TK * 64; e += 256) {
            const int kka = AK ? e % TK : e / 64, ca = AK ? e / TK : e % 64;
            const int kkb = BK ? e % TK : e / 64, cb = BK ? e / TK : e % 64;
            As[kka][ca] = kb + kka < k1 ? fa(ca, kb + kka) : T(0);
            Bs[kkb][cb] = kb + kkb < k1 ? fb(kb + kkb, cb) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty + 16 * u]; b[u] = Bs[kk][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
}

// Triangular tile index t -> (ti, tj) with tj <= ti.
__device__ __forceinline__ void tri_index(int64_t t, int64_t& ti, int64_t& tj)
{
    ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    tj = t - ti * (ti + 1) / 2;
}

}  // namespace uoi
