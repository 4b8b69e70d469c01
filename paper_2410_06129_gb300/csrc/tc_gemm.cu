// Mixed-precision tensor-core kernels (placeholder until the tcgen05 path lands).
#include "pinv_internal.h"

namespace pinv {

bool tc_available() { return false; }

cudaError_t launch_gram_tc(const EncodeDev&, double, int, double2*, int64_t, DevStatus*, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_recon_tc(const EncodeDev&, const double2*, int64_t, int, float2*, DevStatus*,
                            cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_apply32(const float2*, int64_t, int64_t, const float2*, int64_t, float2*,
                           cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace pinv
