// Quality metrics (Section 3.7). Placeholder until the FP64 kernels land.
#include "bl_internal.cuh"

namespace bl {
bl_status quality_run(bl_layout*, int32_t, int32_t, uint64_t, double*, cudaStream_t) {
    return set_error(BL_EINVAL, "quality metrics are not built yet");
}
}  // namespace bl
