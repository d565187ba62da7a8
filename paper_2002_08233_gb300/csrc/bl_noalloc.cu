// Exact-mode layout run that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an engine that owns every byte of device
// memory through its own pool, a serving loop that must not hit the implicit
// device synchronisation of an allocation, or a process running under a hard
// device-memory quota. bl_layout_run_noalloc takes the graph and the positions as
// device buffers the caller already owns and keeps the engine's own working memory
// (second position buffer, per-CTA energies, status word and step counter) in one
// file-scope device array instead of allocating it. Every GPU that loads the
// library holds that array (about 2 MiB) until the process exits.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "bl_internal.cuh"

namespace bl {
namespace {

constexpr int kNoAllocMaxN = 131072;              // vertices (second position buffer)
constexpr int kNoAllocMaxEnergySlots = 131072;    // iterations x CTAs of per-CTA energies
constexpr size_t kNoAllocHeader = 256;            // status word (+0), step counter (+64)
constexpr size_t kNoAllocPosBytes = (size_t)kNoAllocMaxN * sizeof(float2);
constexpr size_t kNoAllocBytes =
    kNoAllocHeader + kNoAllocPosBytes + (size_t)kNoAllocMaxEnergySlots * sizeof(double);

// The scratch array. Host code must not use this name as an address: it is a
// host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
struct ScratchEntry {
    void* addr = nullptr;
    unsigned long long ctx = 0;   // id of the context the address belongs to
};
std::mutex g_scratch_mu;
ScratchEntry g_scratch[kMaxDevices];

// Unique id of the calling thread's current context (cuCtxGetCurrent +
// cuCtxGetId, reached through the runtime's driver entry points so the library
// does not link the driver library), or 0 when there is none or it is unknown.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return 0;
    unsigned long long id = 0;
    return get_id(c, &id) == CUDA_SUCCESS ? id : 0;
}

// Device address of the scratch array on the current device. It is looked up
// with the device current on the first call, and again whenever the device's
// context has changed since (after a cudaDeviceReset the old address is stale).
bl_status scratch_address(void** out) {
    int dev = 0;
    BL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: device index out of range");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchEntry& ent = g_scratch[dev];
    if (ent.addr == nullptr || ctx == 0 || ctx != ent.ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
        ent.addr = p;
        ent.ctx = current_context_id();   // the lookup made the context current if it was not
    }
    *out = ent.addr;
    return BL_OK;
}

}  // namespace
}  // namespace bl

using namespace bl;

extern "C" bl_status bl_layout_run_noalloc(int32_t n, const int32_t* d_rowptr, const int32_t* d_colids,
                                           float* d_xy, int32_t iters, int32_t batch,
                                           const bl_force_params* params, int64_t start_iter,
                                           double* d_energy, void* stream) {
    if (n < 1 || !d_rowptr || !d_colids || !d_xy)
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: n must be >= 1 and buffers non-NULL");
    if (n > kNoAllocMaxN)
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: n exceeds the scratch limit of 131072 vertices");
    if (iters < 0 || start_iter < 0) return set_error(BL_EINVAL, "bl_layout_run_noalloc: negative count");
    if (batch < 1 || batch > kMaxBatch)
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: batch must be in [1, 8192]");
    bl_force_params p{1.0f, 1.0f, 0, -1, BL_MODEL_FR};
    if (params) p = *params;
    if (!(p.K > 0.0f) || !(p.R > 0.0f) || !std::isfinite(p.K) || !std::isfinite(p.R))
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: K and R must be positive and finite");
    if (p.energy_model < 0 || p.energy_model > 3)
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: energy_model must be 0..3");
    if (p.kahan < -1 || p.kahan > 1)
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: kahan must be -1, 0 or 1");
    if (iters == 0) return BL_OK;
    ExactPlan plan;
    BL_TRY(exact_plan(n, batch, 0, 0, &plan));
    if ((int64_t)iters * plan.G > kNoAllocMaxEnergySlots)
        return set_error(BL_EINVAL, "bl_layout_run_noalloc: iterations x CTAs exceed the scratch "
                                    "limit of 131072 energy slots (run fewer iterations per call)");
    void* base = nullptr;
    BL_TRY(scratch_address(&base));
    unsigned char* sc = static_cast<unsigned char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the status word and the step counter must start at zero; the rest is
    // written before it is read
    BL_CUDA_TRY(cudaMemsetAsync(sc, 0, kNoAllocHeader, st));
    ExactTask tk{};
    tk.n = n;
    tk.BS = batch;
    tk.B = div_up(n, batch);
    tk.rowptr = d_rowptr;
    tk.colids = d_colids;
    tk.pos = reinterpret_cast<float2*>(d_xy);
    tk.pos_alt = reinterpret_cast<float2*>(sc + kNoAllocHeader);
    tk.e_iter = reinterpret_cast<double*>(sc + kNoAllocHeader + kNoAllocPosBytes);
    tk.iters = iters;
    double step = 1.0;
    for (int64_t k = 0; k < start_iter; k++) step *= 0.999;
    tk.step0 = step;
    tk.crit_cap = plan.crit_cap;
    tk.nbr_cap = plan.nbr_cap;
    ExactParams prm{};
    prm.invK = 1.0f / p.K;
    prm.negRK2 = -p.R * p.K * p.K;
    prm.repulse_neighbors = p.repulse_neighbors;
    prm.am = model_exponent(p.energy_model);
    prm.kahan = kahan_on(p.kahan, n) ? 1 : 0;
    prm.status = reinterpret_cast<int*>(sc);
    prm.bar = reinterpret_cast<unsigned*>(sc + 64);
    BL_TRY(exact_launch(plan, tk, prm, st));
    if (d_energy) BL_TRY(energy_reduce(tk.e_iter, iters, plan.G, d_energy, st));
    if (iters & 1)   // an odd number of iterations ends in the second buffer
        BL_CUDA_TRY(cudaMemcpyAsync(d_xy, tk.pos_alt, (size_t)n * sizeof(float2),
                                    cudaMemcpyDeviceToDevice, st));
    int status = 0;
    BL_CUDA_TRY(cudaMemcpyAsync(&status, sc, sizeof(int), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    if (status != 0)
        return set_error((bl_status)status, "bl_layout_run_noalloc: a bounded device-side wait timed out");
    return BL_OK;
}
