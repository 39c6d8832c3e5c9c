// common.cuh -- shared device helpers of the GB300 UoI library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "../../include/uoi.h"

namespace uoi {

// ---------------------------------------------------------------------------
// Errors: host code throws uoi::Error, the C-ABI layer turns it into a status.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
    int status;
    Error(int s, const std::string& msg) : std::runtime_error(msg), status(s) {}
};

#define UOI_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t err__ = (call);                                                     \
        if (err__ != cudaSuccess)                                                       \
            throw ::uoi::Error(err__ == cudaErrorMemoryAllocation ? UOI_ERR_OOM         \
                                                                 : UOI_ERR_CUDA,        \
                               std::string(#call) + ": " + cudaGetErrorString(err__));  \
    } while (0)

#define UOI_CHECK_LAUNCH() UOI_CUDA(cudaGetLastError())

// Count of kernels this library launched on the calling host thread (reported in
// uoi_diag.gpu_launches; one fit runs on one thread).
extern thread_local int64_t g_launches;
inline void count_launch(int64_t n = 1) { g_launches += n; }
// True on the worker threads of a batch of fits, whose fits share the device with
// one another (a fit then adds no concurrency of its own).
extern thread_local bool g_fit_in_batch;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11), written for the device.  The i-th draw
// of stream (k, tag) is lane i%4 of Philox(counter=(i/4, k, tag, 0),
// key=(seed, problem)); index maps use floor(r * n / 2^64).
// ---------------------------------------------------------------------------
struct PhiloxKey { uint64_t seed, problem; };

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__device__ __forceinline__ uint64_t philox_draw(PhiloxKey key, uint64_t k, uint64_t tag, uint64_t i)
{
    uint64_t c[4] = { i >> 2, k, tag, 0 };
    philox4x64_10(c, key.seed, key.problem);
    const uint32_t lane = (uint32_t)(i & 3u);
    return lane == 0 ? c[0] : lane == 1 ? c[1] : lane == 2 ? c[2] : c[3];
}

__device__ __forceinline__ uint64_t range_map(uint64_t r, uint64_t n) { return __umul64hi(r, n); }

enum : uint32_t { TAG_SELECTION = 1, TAG_SPLIT = 2, TAG_RESAMPLE = 3 };

// ---------------------------------------------------------------------------
// Small device utilities
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T soft_threshold(T v, T kappa)
{
    return v > kappa ? v - kappa : (v < -kappa ? v + kappa : T(0));
}

// FP64 -> FP32 with round-to-nearest-even using integer operations only (the
// FP64 pipe of this part is ~1/64 of its FP32 rate, and conversions from FP64
// run on it).  Magnitudes below 2^-126 flush to signed zero.
__device__ __forceinline__ float f64_to_f32_int(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FFull);
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (mant ? 0x400000u : 0u));
    int e32 = e - 1023 + 127;
    if (e32 <= 0) return __uint_as_float(sign);
    unsigned int m = (unsigned int)(mant >> 29);
    const unsigned long long rem = mant & ((1ull << 29) - 1ull);
    const unsigned long long half = 1ull << 28;
    if (rem > half || (rem == half && (m & 1u))) {
        if (++m == (1u << 23)) { m = 0; ++e32; }
    }
    if (e32 >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned int)e32 << 23) | m);
}

// Warp-wide count of near-threshold features at column completion: lane i holds the
// final z_i, u_i of a column with threshold kappa = lambda/rho (v = z + u, so the
// margin |v_i| - kappa is |z_i| where z_i != 0 and |u_i| - kappa where z_i = 0).
// Lane 0 adds the count to *out.  Every lane of the warp must call it.
template <typename T>
__device__ __forceinline__ void count_near_threshold(bool valid, T zi, T ui, T kappa, T band,
                                                     unsigned long long* out)
{
    const T az = zi < T(0) ? -zi : zi;
    const T au = ui < T(0) ? -ui : ui;
    const T gap = au > kappa ? au - kappa : kappa - au;
    const bool near = valid && (zi != T(0) ? az <= band : gap <= band);
    const unsigned bal = __ballot_sync(0xffffffffu, near);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(out, (unsigned long long)__popc(bal));
}

// Device-side error word: kernels record the first error here and return.
struct DevStatus {
    int32_t code;      // 0 = ok, else a UOI_ERR_* value
    int32_t where;     // kernel-specific detail (index)
};

__device__ __forceinline__ void dev_fail(DevStatus* st, int code, int where)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

// ---------------------------------------------------------------------------
// Index checks.  check_index records UOI_ERR_BOUNDS and the site in *st and
// returns false when i is outside [0, n), so the caller skips the access:
// nothing traps and nothing outside a buffer is touched.  UOI_IN_BOUNDS(i, n,
// site) is such a check in the checked build (compiled with UOI_BOUNDS_CHECK=1),
// on a status word of its own translation unit, and `true` in the release build.
// Every fit of the checked build reads and clears the status words of all
// translation units when it ends and fails with UOI_ERR_BOUNDS if one was set.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool check_index(DevStatus* st, int64_t i, int64_t n, int site)
{
    if (i >= 0 && i < n) return true;
    if (atomicCAS(&st->code, 0, UOI_ERR_BOUNDS) == 0) st->where = site;
    return false;
}

#if defined(UOI_BOUNDS_CHECK) && UOI_BOUNDS_CHECK
static __device__ DevStatus g_bounds_status;     // one per translation unit
#define UOI_IN_BOUNDS(i, n, site) ::uoi::check_index(&::uoi::g_bounds_status, (int64_t)(i), (int64_t)(n), (site))
// Registers a reader of one translation unit's status word (defined in api.cu).
void register_bounds_reader(DevStatus (*reader)());
namespace {
DevStatus read_bounds_status_tu()
{
    DevStatus h{}, z{};
    cudaMemcpyFromSymbol(&h, g_bounds_status, sizeof(h));
    cudaMemcpyToSymbol(g_bounds_status, &z, sizeof(z));
    return h;
}
struct BoundsReaderRegistration {
    BoundsReaderRegistration() { register_bounds_reader(&read_bounds_status_tu); }
};
static BoundsReaderRegistration g_bounds_reader_registration;
}  // namespace
#else
#define UOI_IN_BOUNDS(i, n, site) true
#endif

}  // namespace uoi
