// noalloc.cu -- lasso_admm_batch_noalloc: the batched LASSO-ADMM solver for callers
// that must not allocate device memory.
//
// Some callers cannot let a library allocate device memory: applications that
// reserve all of the device's memory at start-up for their own allocator (so a
// library allocation fails or steals from a budget the application manages),
// hosts that run under a fixed device-memory quota, and latency-critical loops
// where an allocation may block and a free synchronises the device.  This entry
// point takes its working memory from one file-scope device array instead, so it
// allocates nothing.
//
// The array lives in every GPU that loads the library, for the life of the
// process.  In host code its name is only a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and that pointer is handed to the kernels.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "kernels.h"

namespace uoi {
namespace {

constexpr size_t kScratchBytes = UOI_NOALLOC_SCRATCH_BYTES;   // per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

void* g_scratch_dev[kMaxDevices] = {};
std::once_flag g_scratch_once[kMaxDevices];

// Device address of the scratch array on the current device, looked up once per
// device (std::call_once: concurrent first calls wait for one lookup; a failed
// lookup throws and leaves the flag unset, so the next call tries again).
void* scratch_for_current_device()
{
    int dev = 0;
    UOI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw Error(UOI_ERR_UNSUPPORTED, "device index out of range");
    std::call_once(g_scratch_once[dev], [dev] {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            throw Error(UOI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_dev[dev] = ptr;
    });
    return g_scratch_dev[dev];
}

// True for device memory of the current device, or managed memory.
bool on_device(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return at.device == dev;
}

__global__ void k_fill(double* out, int n, double v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

__global__ void k_count_nonconverged(const uint8_t* conv, int64_t n, int32_t* out)
{
    int c = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) c += conv[i] ? 0 : 1;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

// Carves aligned pieces out of the scratch array.
struct Carver {
    unsigned char* base;
    size_t used = 0;
    template <typename T>
    T* take(size_t count)
    {
        used = (used + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + used);
        used += count * sizeof(T);
        return p;
    }
};

}  // namespace
}  // namespace uoi

using namespace uoi;

extern "C" int lasso_admm_batch_noalloc(const double* X, const double* Y, int64_t n, int64_t p,
                                        int64_t r, const uint32_t* weights, int32_t B,
                                        const double* lambdas, int32_t q, double rho,
                                        double abs_tol, double rel_tol, int32_t max_iter,
                                        int32_t warm_start, double* beta_out, int32_t* iters_out,
                                        uint8_t* converged_out, void* stream)
{
    try {
        g_last_error.clear();
        if (!X || !Y || !lambdas || !beta_out)
            throw Error(UOI_ERR_INVALID_ARG, "NULL pointer");
        if (n <= 0 || p <= 0 || r <= 0 || q <= 0 || B <= 0 || max_iter <= 0)
            throw Error(UOI_ERR_INVALID_ARG, "sizes must be positive");
        if (!weights && B != 1) throw Error(UOI_ERR_INVALID_ARG, "unweighted call needs B == 1");
        if (!(rho > 0.0)) throw Error(UOI_ERR_INVALID_ARG, "rho must be positive");
        if (warm_start != UOI_WARM_NONE && warm_start != UOI_WARM_PATH)
            throw Error(UOI_ERR_INVALID_ARG, "warm_start must be NONE or PATH");
        if (p > UOI_NOALLOC_MAX_P)
            throw Error(UOI_ERR_INVALID_ARG, "p exceeds UOI_NOALLOC_MAX_P");
        const void* ptrs[] = { X, Y, lambdas, beta_out };
        for (const void* ptr : ptrs)
            if (!on_device(ptr)) throw Error(UOI_ERR_INVALID_ARG, "every buffer must be device memory");
        if ((weights && !on_device(weights)) || (iters_out && !on_device(iters_out)) ||
            (converged_out && !on_device(converged_out)))
            throw Error(UOI_ERR_INVALID_ARG, "every buffer must be device memory");
        const int64_t ncol = (int64_t)B * q * r;
        // working set: G (B p p; reused for L^-1 once the system is built), A and M
        // (B p p each), moments and right-hand sides (B p r each), b_k / n_k for
        // r = 1 (B p), n_k, chain counters, status, convergence flags and a counter
        const size_t need = 3 * (sizeof(double) * (size_t)(B * p * p) + 256) +
                            2 * (sizeof(double) * (size_t)(B * p * r) + 256) +
                            sizeof(double) * (size_t)(B * p) + 256 +
                            sizeof(double) * B + sizeof(int32_t) * B + sizeof(DevStatus) +
                            (size_t)ncol + sizeof(int32_t) + 6 * 256;
        if (need > kScratchBytes)
            throw Error(UOI_ERR_INVALID_ARG, "problem needs more than the 16 MiB no-allocation scratch");

        cudaStream_t s = (cudaStream_t)stream;
        Carver cv{ static_cast<unsigned char*>(scratch_for_current_device()) };
        double* G = cv.take<double>((size_t)(B * p * p));
        double* A = cv.take<double>((size_t)(B * p * p));
        double* M = cv.take<double>((size_t)(B * p * p));
        double* Bm = cv.take<double>((size_t)(B * p * r));
        double* c = cv.take<double>((size_t)(B * p * r));
        double* bs = cv.take<double>((size_t)(B * p));
        double* nk = cv.take<double>((size_t)B);
        int32_t* chains = cv.take<int32_t>((size_t)B);
        DevStatus* st = cv.take<DevStatus>(1);
        uint8_t* conv = cv.take<uint8_t>((size_t)ncol);
        int32_t* noncon = cv.take<int32_t>(1);
        if (cv.used > kScratchBytes)
            throw Error(UOI_ERR_INVALID_ARG, "problem needs more than the 16 MiB no-allocation scratch");

        // the array keeps the previous call's contents: clear what must start at zero
        UOI_CUDA(cudaMemsetAsync(chains, 0, sizeof(int32_t) * B, s));
        UOI_CUDA(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
        UOI_CUDA(cudaMemsetAsync(noncon, 0, sizeof(int32_t), s));

        moments_fp64(X, p, Y, r, n, p, r, weights, nullptr, B, G, Bm, 0, s);
        if (weights) {
            weight_sums(weights, nullptr, n, B, nk, s);
        } else {
            k_fill<<<1, 32, 0, s>>>(nk, 1, (double)n);
            UOI_CHECK_LAUNCH();
        }
        build_and_factor<double>(G, nk, rho, p, B, A, st, s);
        DevStatus hs{};
        UOI_CUDA(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        UOI_CUDA(cudaStreamSynchronize(s));
        if (hs.code != 0) throw Error(hs.code, "Cholesky of G/n + rho I failed");
        // G is no longer read: its space holds L^-1
        inverse_and_rhs<double>(A, Bm, nk, p, r, B, G, M, c, s, bs);

        AdmmProblem<double> P;
        P.G = B; P.p = p; P.r = r; P.q = q;
        P.M = M; P.c = c; P.lambdas = lambdas;
        P.rho = rho; P.abs_tol = abs_tol; P.rel_tol = rel_tol; P.max_iter = max_iter;
        P.warm = warm_start;
        P.beta = beta_out; P.iters = iters_out; P.conv = converged_out ? converged_out : conv;
        if (!admm_solve_resident_with<double>(P, chains, s))
            throw Error(UOI_ERR_INVALID_ARG, "p too large for the no-allocation schedule");
        k_count_nonconverged<<<1, 256, 0, s>>>(P.conv, ncol, noncon);
        UOI_CHECK_LAUNCH();
        int32_t h = 0;
        UOI_CUDA(cudaMemcpyAsync(&h, noncon, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        UOI_CUDA(cudaStreamSynchronize(s));
        return h > 0 ? UOI_OK_WITH_WARNINGS : UOI_OK;
    } catch (const Error& e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return UOI_ERR_CUDA;
    }
}
