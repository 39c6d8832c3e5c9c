// bootstrap.cu -- G0: Philox bootstrap and block-bootstrap index generation.
//
// Alg. 1/2 "Generate bootstrap sample T^k" (selection: draws with replacement
// from all units), and the estimation loop's training/evaluation samples
// (Fig. 1(c): reshuffle, then resample the training pool).  A unit is a row
// (UoI_LASSO) or a block of block_len consecutive lagged rows (UoI_VAR block
// bootstrap, Sec. III-A-2).  Results are integer counts built with atomics,
// so they are bit-exact and independent of thread order.
#include "kernels.h"

namespace uoi {

namespace {

__device__ __forceinline__ void add_unit(uint32_t* w, int64_t m, int64_t L, uint64_t unit)
{
    int64_t r0 = (int64_t)unit * L;
    int64_t r1 = r0 + L < m ? r0 + L : m;
    for (int64_t row = r0; row < r1; ++row) atomicAdd(&w[row], 1u);
}

// One thread per group of 4 draws (one Philox block); grid-stride over B x blocks.
__global__ void k_selection(int64_t m, int64_t L, int64_t units, PhiloxKey key, int32_t B,
                            uint32_t* w)
{
    const int64_t blocks = (units + 3) / 4;
    const int64_t total = blocks * B;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / blocks, blk = t % blocks;
        uint64_t c[4] = { (uint64_t)blk, (uint64_t)k, TAG_SELECTION, 0 };
        philox4x64_10(c, key.seed, key.problem);
        uint32_t* wk = w + k * m;
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) {
            const int64_t i = blk * 4 + lane;
            if (i < units) add_unit(wk, m, L, range_map(c[lane], (uint64_t)units));
        }
    }
}

// Moving blocks: draw i of bootstrap k starts a run of L rows at
// floor(r_i (m - L + 1) / 2^64); one thread per Philox block of 4 draws.
__global__ void k_selection_moving(int64_t m, int64_t L, int64_t units, PhiloxKey key, int32_t B,
                                   uint32_t* w)
{
    const int64_t blocks = (units + 3) / 4;
    const int64_t total = blocks * B;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / blocks, blk = t % blocks;
        uint64_t c[4] = { (uint64_t)blk, (uint64_t)k, TAG_SELECTION, 0 };
        philox4x64_10(c, key.seed, key.problem);
        uint32_t* wk = w + k * m;
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) {
            const int64_t i = blk * 4 + lane;
            if (i >= units) continue;
            const int64_t start = (int64_t)range_map(c[lane], (uint64_t)(m - L + 1));
            for (int64_t row = start; row < start + L; ++row) atomicAdd(&wk[row], 1u);
        }
    }
}

// Reshuffle keys: key[k][u] and bucket counts (bucket = floor(key * units / 2^64)).
__global__ void k_split_keys(int64_t units, PhiloxKey key, int32_t Bk, int split_fixed,
                             uint64_t* keys, uint32_t* counts)
{
    const int64_t total = units * Bk;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / units, u = t % units;
        const uint64_t kk = split_fixed ? 0u : (uint64_t)k;
        const uint64_t r = philox_draw(key, kk, TAG_SPLIT, (uint64_t)u);
        keys[t] = r;
        atomicAdd(&counts[k * units + range_map(r, (uint64_t)units)], 1u);
    }
}

// Exclusive scan of bucket counts per k (one block per k).
__global__ void k_bucket_scan(int64_t units, const uint32_t* counts, uint32_t* starts)
{
    const int64_t k = blockIdx.x;
    const uint32_t* c = counts + k * units;
    uint32_t* s = starts + k * units;
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < units; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        uint32_t v = i < units ? c[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += n;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            uint32_t t = lane < nw ? warp_tot[lane] : 0u;
            uint32_t ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t n = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o) ti += n;
            }
            if (lane < nw) warp_tot[lane] = ti - t;   // exclusive warp offsets
        }
        __syncthreads();
        if (i < units) s[i] = carry + warp_tot[wid] + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += warp_tot[wid] + incl;
        __syncthreads();
    }
}

__global__ void k_bucket_scatter(int64_t units, int32_t Bk, const uint64_t* keys,
                                 const uint32_t* starts, uint32_t* cursor, uint32_t* slots)
{
    const int64_t total = units * Bk;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / units, u = t % units;
        const uint64_t b = range_map(keys[t], (uint64_t)units);
        const uint32_t pos = atomicAdd(&cursor[k * units + b], 1u);
        slots[k * units + starts[k * units + b] + pos] = (uint32_t)u;
    }
}

// rank of unit u = bucket start + number of smaller (key, index) pairs in its bucket.
__global__ void k_bucket_rank(int64_t units, int32_t Bk, const uint64_t* keys,
                              const uint32_t* counts, const uint32_t* starts,
                              const uint32_t* slots, uint32_t* perm)
{
    const int64_t total = units * Bk;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / units, u = t % units;
        const uint64_t ku = keys[t];
        const uint64_t b = range_map(ku, (uint64_t)units);
        const uint32_t s0 = starts[k * units + b], n = counts[k * units + b];
        uint32_t rank = s0;
        for (uint32_t j = 0; j < n; ++j) {
            const uint32_t v = slots[k * units + s0 + j];
            const uint64_t kv = keys[k * units + v];
            if (kv < ku || (kv == ku && (int64_t)v < u)) ++rank;
        }
        perm[k * units + rank] = (uint32_t)u;
    }
}

__global__ void k_eval_mask(int64_t m, int64_t L, int64_t units, int64_t pool, int32_t B,
                            int split_fixed, const uint32_t* perm, uint8_t* eval)
{
    const int64_t ne = units - pool;
    const int64_t total = ne * B;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / ne, pos = pool + t % ne;
        const uint32_t* pk = perm + (split_fixed ? 0 : k) * units;
        const int64_t unit = pk[pos];
        const int64_t r0 = unit * L, r1 = r0 + L < m ? r0 + L : m;
        for (int64_t row = r0; row < r1; ++row) eval[k * m + row] = 1;
    }
}

__global__ void k_train_draws(int64_t m, int64_t L, int64_t units, int64_t pool, PhiloxKey key,
                              int32_t B, int split_fixed, const uint32_t* perm, uint32_t* w)
{
    const int64_t blocks = (pool + 3) / 4;
    const int64_t total = blocks * B;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / blocks, blk = t % blocks;
        uint64_t c[4] = { (uint64_t)blk, (uint64_t)k, TAG_RESAMPLE, 0 };
        philox4x64_10(c, key.seed, key.problem);
        const uint32_t* pk = perm + (split_fixed ? 0 : k) * units;
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) {
            const int64_t i = blk * 4 + lane;
            if (i < pool) add_unit(w + k * m, m, L, pk[range_map(c[lane], (uint64_t)pool)]);
        }
    }
}

__global__ void k_weight_sums(const uint32_t* w, const uint8_t* mask, int64_t m, double* nk)
{
    const int64_t k = blockIdx.x;
    uint64_t s = 0;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x)
        s += w ? (uint64_t)w[k * m + t] : (uint64_t)mask[k * m + t];
    s = warp_sum(s);
    __shared__ uint64_t part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t tot = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += part[i];
        nk[k] = (double)tot;
    }
}

int grid_for(int64_t work, int threads)
{
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

void selection_weights(int64_t m, int64_t block_len, PhiloxKey key, int32_t B, uint32_t* w,
                       cudaStream_t s, int32_t block_mode)
{
    const int64_t L = block_len > 1 ? block_len : 1;
    const int64_t units = (m + L - 1) / L;
    UOI_CUDA(cudaMemsetAsync(w, 0, sizeof(uint32_t) * (size_t)(m * B), s));
    const int64_t work = ((units + 3) / 4) * B;
    if (block_mode == 1 && L > 1)
        k_selection_moving<<<grid_for(work, 256), 256, 0, s>>>(m, L, units, key, B, w);
    else
        k_selection<<<grid_for(work, 256), 256, 0, s>>>(m, L, units, key, B, w);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void estimation_weights(int64_t m, int64_t block_len, double train_frac, int split_fixed,
                        PhiloxKey key, int32_t B, uint32_t* w_train, uint8_t* eval,
                        cudaStream_t s)
{
    const int64_t L = block_len > 1 ? block_len : 1;
    const int64_t units = (m + L - 1) / L;
    const int64_t pool = (int64_t)floor(train_frac * (double)units);
    if (pool < 1 || pool >= units)
        throw Error(UOI_ERR_INVALID_ARG, "estimation split leaves the pool or E^k empty");
    const int32_t Bk = split_fixed ? 1 : B;       // reshuffles needed
    DevBuf keys(sizeof(uint64_t) * units * Bk, s);
    DevBuf counts(sizeof(uint32_t) * units * Bk, s);
    DevBuf starts(sizeof(uint32_t) * units * Bk, s);
    DevBuf cursor(sizeof(uint32_t) * units * Bk, s);
    DevBuf slots(sizeof(uint32_t) * units * Bk, s);
    DevBuf perm(sizeof(uint32_t) * units * Bk, s);
    UOI_CUDA(cudaMemsetAsync(counts.ptr, 0, counts.bytes, s));
    UOI_CUDA(cudaMemsetAsync(cursor.ptr, 0, cursor.bytes, s));
    const int64_t work = units * Bk;
    k_split_keys<<<grid_for(work, 256), 256, 0, s>>>(units, key, Bk, split_fixed,
                                                     keys.as<uint64_t>(), counts.as<uint32_t>());
    UOI_CHECK_LAUNCH();
    k_bucket_scan<<<Bk, 1024, 0, s>>>(units, counts.as<uint32_t>(), starts.as<uint32_t>());
    UOI_CHECK_LAUNCH();
    k_bucket_scatter<<<grid_for(work, 256), 256, 0, s>>>(units, Bk, keys.as<uint64_t>(),
                                                         starts.as<uint32_t>(),
                                                         cursor.as<uint32_t>(),
                                                         slots.as<uint32_t>());
    UOI_CHECK_LAUNCH();
    k_bucket_rank<<<grid_for(work, 256), 256, 0, s>>>(units, Bk, keys.as<uint64_t>(),
                                                      counts.as<uint32_t>(),
                                                      starts.as<uint32_t>(),
                                                      slots.as<uint32_t>(), perm.as<uint32_t>());
    UOI_CHECK_LAUNCH();
    UOI_CUDA(cudaMemsetAsync(eval, 0, (size_t)(m * B), s));
    UOI_CUDA(cudaMemsetAsync(w_train, 0, sizeof(uint32_t) * (size_t)(m * B), s));
    k_eval_mask<<<grid_for((units - pool) * B, 256), 256, 0, s>>>(m, L, units, pool, B,
                                                                   split_fixed,
                                                                   perm.as<uint32_t>(), eval);
    UOI_CHECK_LAUNCH();
    k_train_draws<<<grid_for(((pool + 3) / 4) * B, 256), 256, 0, s>>>(
        m, L, units, pool, key, B, split_fixed, perm.as<uint32_t>(), w_train);
    UOI_CHECK_LAUNCH();
    count_launch(6);
}

void weight_sums(const uint32_t* w, const uint8_t* mask, int64_t m, int32_t B, double* nk,
                 cudaStream_t s)
{
    k_weight_sums<<<B, 256, 0, s>>>(w, mask, m, nk);
    UOI_CHECK_LAUNCH();
    count_launch();
}

}  // namespace uoi
