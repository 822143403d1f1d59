// Correlation on the tcgen05 tensor cores (placeholder until the FP8 kernel lands).
#include "blink_internal.cuh"

namespace blink {

blink_status launch_corr_fp8(int, const uint8_t*, int64_t, const Plan&, int, int, int, void*, int64_t, int*, int,
                             cudaStream_t) {
    return set_error(BLINK_ERR_UNSUPPORTED, "FP8 tensor-core correlation is not built yet");
}

}  // namespace blink
