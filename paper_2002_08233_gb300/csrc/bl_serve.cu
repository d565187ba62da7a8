// Batched layouts and the continuous-batching server. Placeholder until the
// persistent batched engine lands.
#include "bl_internal.cuh"

using namespace bl;

extern "C" {
bl_status bl_server_create(size_t, bl_server**) {
    return set_error(BL_EINVAL, "the server is not built yet");
}
bl_status bl_serve_submit(bl_server*, const bl_graph*, uint64_t, int32_t, int32_t, bl_mode, float,
                          uint64_t*) {
    return set_error(BL_EINVAL, "the server is not built yet");
}
bl_status bl_serve_poll(bl_server*, uint64_t, float*, int64_t, double*) {
    return set_error(BL_EINVAL, "the server is not built yet");
}
bl_status bl_serve_cancel(bl_server*, uint64_t) { return set_error(BL_EINVAL, "not built yet"); }
bl_status bl_server_stats(bl_server*, double*, int64_t) { return set_error(BL_EINVAL, "not built yet"); }
void bl_server_free(bl_server*) {}
}
