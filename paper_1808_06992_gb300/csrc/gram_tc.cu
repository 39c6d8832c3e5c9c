// gram_tc.cu -- G1 on tcgen05 tensor cores (mixed form).  Placeholder until the
// split-bf16 kernel lands: reports unavailable, so the FP64 kernel is used.
#include "kernels.h"

namespace uoi {

bool gram_tc_available() { return false; }

void moments_tc(const double*, int64_t, const double*, int64_t, int64_t, int64_t, int64_t,
                const uint32_t*, const uint8_t*, int32_t, double*, double*, cudaStream_t)
{
    throw Error(UOI_ERR_UNSUPPORTED, "tensor-core Gram not built");
}

}  // namespace uoi
