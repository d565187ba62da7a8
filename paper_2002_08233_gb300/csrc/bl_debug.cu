// Test hook for failure detection: a grid barrier that can never complete.
//
// The kernel runs the same bounded GridBarrier the engines use, launched
// cooperatively with 2 CTAs but told to expect 3, so no CTA ever sees the barrier
// complete. Each CTA's wait gives up after `limit_ms`, records BL_ETIMEOUT in the
// status word and leaves; nothing faults and the context stays usable. Tests use
// it to check that a wait that runs out reaches the host as BL_ETIMEOUT.
#include <cuda_runtime.h>

#include "bl_internal.cuh"

namespace bl {
namespace {

__global__ void barrier_timeout_kernel(unsigned* ctr, int* status, unsigned long long limit_ns) {
    GridBarrier gb{ctr, status, gridDim.x + 1u, 0u};
    gb.limit_ns = limit_ns;
    gb.sync();
}

}  // namespace
}  // namespace bl

using namespace bl;

extern "C" bl_status bl_debug_barrier_timeout(int32_t limit_ms) {
    if (limit_ms < 1 || limit_ms > 2000) return set_error(BL_EINVAL, "bl_debug_barrier_timeout: limit_ms in [1, 2000]");
    cudaStream_t st = current_stream();
    DevBuf words;
    BL_TRY(words.ensure(current_allocator(), 256));
    unsigned* ctr = reinterpret_cast<unsigned*>(static_cast<char*>(words.p) + 64);
    int* status = static_cast<int*>(words.p);
    bl_status s = BL_OK;
    cudaError_t e = cudaMemsetAsync(words.p, 0, 256, st);
    unsigned long long lim = (unsigned long long)limit_ms * 1000000ull;
    void* args[] = {&ctr, &status, &lim};
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void*)barrier_timeout_kernel, dim3(2), dim3(32), args, 0, st);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_error(e, "bl_debug_barrier_timeout");
    words.release();
    if (s != BL_OK) return s;
    if (h != 0) return set_error((bl_status)h, "a bounded device-side wait timed out");
    return BL_OK;
}
