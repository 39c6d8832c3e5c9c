// selftest.cu -- test support: a bounded mbarrier wait that runs out, and the
// device index check.
//
// Every tensor-core kernel of the library waits on mbarriers with a limit
// (tc::mbar_wait, kernel argument wait_ns, one second by default).  When a limit
// runs out the kernel records UOI_ERR_TIMEOUT in its error word, leaves its
// pipeline and returns, so the context stays usable and the call returns
// UOI_ERR_TIMEOUT.  uoi_selftest_wait runs that wait on its own: one thread
// initialises an mbarrier that expects one arrival and waits for phase 0 with the
// caller's limit.  With arrive = 0 nothing arrives, so the wait must run out;
// with arrive = 1 the thread arrives first, so the wait must succeed at once.
#include <cuda_runtime.h>

#include "kernels.h"
#include "tc_common.cuh"

namespace uoi {
namespace {

__global__ void k_selftest_wait(uint64_t limit_ns, int32_t arrive, int32_t* err,
                                unsigned long long* waited_ns)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) tc::mbar_arrive(&bar);
        const uint64_t t0 = tc::now_ns();
        const bool ok = tc::mbar_wait(&bar, 0, &abort_flag, limit_ns);
        *waited_ns = (unsigned long long)(tc::now_ns() - t0);
        if (!ok) atomicCAS(err, 0, UOI_ERR_TIMEOUT);
    }
}

// One thread stores into buf[index] if the index check passes (buf has extent
// elements): the check of the checked build, run explicitly.
__global__ void k_selftest_index(int64_t index, int64_t extent, float* buf, DevStatus* st)
{
    if (threadIdx.x == 0 && check_index(st, index, extent, 901)) buf[index] = 1.f;
}

}  // namespace
}  // namespace uoi

using namespace uoi;

extern "C" int uoi_selftest_index_check(int64_t index, int64_t extent, void* stream)
{
    try {
        g_last_error.clear();
        if (extent <= 0 || extent > 4096) throw Error(UOI_ERR_INVALID_ARG, "extent must lie in (0, 4096]");
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf buf(sizeof(float) * (size_t)extent, s), st(sizeof(DevStatus), s);
        UOI_CUDA(cudaMemsetAsync(st.ptr, 0, st.bytes, s));
        k_selftest_index<<<1, 32, 0, s>>>(index, extent, buf.as<float>(), st.as<DevStatus>());
        UOI_CHECK_LAUNCH();
        count_launch();
        DevStatus h{};
        UOI_CUDA(cudaMemcpyAsync(&h, st.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
        UOI_CUDA(cudaStreamSynchronize(s));
        if (h.code != 0)
            throw Error(h.code, "index " + std::to_string(index) + " outside [0, " + std::to_string(extent) +
                                    ") at site " + std::to_string(h.where) + ": access skipped");
        return UOI_OK;
    } catch (const Error& e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return UOI_ERR_CUDA;
    }
}

extern "C" int uoi_selftest_wait(uint64_t limit_ns, int32_t arrive, double* waited_ms, void* stream)
{
    try {
        g_last_error.clear();
        if (limit_ns == 0 || limit_ns > 10000000000ull)
            throw Error(UOI_ERR_INVALID_ARG, "limit_ns must lie in (0, 10 s]");
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf err(sizeof(int32_t), s), waited(sizeof(unsigned long long), s);
        UOI_CUDA(cudaMemsetAsync(err.ptr, 0, err.bytes, s));
        UOI_CUDA(cudaMemsetAsync(waited.ptr, 0, waited.bytes, s));
        k_selftest_wait<<<1, 32, 0, s>>>(limit_ns, arrive ? 1 : 0, err.as<int32_t>(),
                                         waited.as<unsigned long long>());
        UOI_CHECK_LAUNCH();
        count_launch();
        int32_t h_err = 0;
        unsigned long long h_ns = 0;
        UOI_CUDA(cudaMemcpyAsync(&h_err, err.ptr, sizeof(h_err), cudaMemcpyDeviceToHost, s));
        UOI_CUDA(cudaMemcpyAsync(&h_ns, waited.ptr, sizeof(h_ns), cudaMemcpyDeviceToHost, s));
        UOI_CUDA(cudaStreamSynchronize(s));
        if (waited_ms) *waited_ms = (double)h_ns * 1e-6;
        if (h_err != 0)
            throw Error(h_err, "mbarrier wait ran out after " + std::to_string((double)h_ns * 1e-6) +
                                   " ms (limit " + std::to_string((double)limit_ns * 1e-6) + " ms)");
        return UOI_OK;
    } catch (const Error& e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return UOI_ERR_CUDA;
    }
}
