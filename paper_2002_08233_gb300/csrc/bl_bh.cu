// Barnes-Hut engine (Section 3.5, Algorithms S3-S5). Placeholder until the
// Morton sort, tree build and walk kernels land.
#include "bl_internal.cuh"

namespace bl {
struct BHState {};
void bh_state_free(BHState* s) { delete s; }
bl_status bh_run(bl_layout*, int, int, float, cudaStream_t) {
    return set_error(BL_EINVAL, "Barnes-Hut mode is not built yet");
}
bl_status bh_debug_forces(bl_layout*, float, float2*, cudaStream_t) {
    return set_error(BL_EINVAL, "Barnes-Hut mode is not built yet");
}
bl_status bh_debug_tree(bl_layout*, uint32_t*, int32_t*, int32_t*, int32_t*, int32_t*, int32_t*,
                        float*, float*, int64_t, int64_t*, float*, cudaStream_t) {
    return set_error(BL_EINVAL, "Barnes-Hut mode is not built yet");
}
}  // namespace bl
