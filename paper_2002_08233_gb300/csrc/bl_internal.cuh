// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the public C ABI (include/batchlayout.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/batchlayout.h"

namespace bl {

// ---------------------------------------------------------------------------
// host-side error plumbing
// ---------------------------------------------------------------------------

bl_status set_error(bl_status st, const std::string& msg);
bl_status cuda_error(cudaError_t e, const char* what);

#define BL_CUDA_TRY(expr)                                                  \
    do {                                                                   \
        cudaError_t e__ = (expr);                                          \
        if (e__ != cudaSuccess) return ::bl::cuda_error(e__, #expr);       \
    } while (0)

#define BL_TRY(expr)                                                       \
    do {                                                                   \
        bl_status s__ = (expr);                                            \
        if (s__ != BL_OK) return s__;                                      \
    } while (0)

cudaStream_t current_stream();

// device memory through the configured allocator
struct Allocator {
    void* (*alloc)(size_t, void*) = nullptr;
    void (*dealloc)(void*, void*) = nullptr;
    void* ctx = nullptr;
};
Allocator current_allocator();
bl_status dev_alloc(const Allocator& a, size_t bytes, void** p);
void dev_free(const Allocator& a, void* p);

// A device buffer owned by a library object.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    Allocator a;
    bl_status ensure(const Allocator& al, size_t need) {
        if (need <= bytes && p) return BL_OK;
        release();
        a = al;
        bl_status s = dev_alloc(a, need ? need : 16, &p);
        if (s == BL_OK) bytes = need ? need : 16;
        return s;
    }
    void release() {
        if (p) dev_free(a, p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Two timing events, destroyed when the scope ends (early error returns included).
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t create() {
        const cudaError_t e = cudaEventCreate(&e0);
        return e == cudaSuccess ? cudaEventCreate(&e1) : e;
    }
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

int device_sm_count();

// ---------------------------------------------------------------------------
// library objects
// ---------------------------------------------------------------------------

}  // namespace bl

struct bl_graph {
    int32_t n = 0;
    int64_t nnz = 0;
    std::vector<int32_t> h_rowptr, h_colids;   // host copy (CSR, cleaned)
    bl::DevBuf rowptr, colids;                 // device copy
};

namespace bl {
struct BHState;       // Barnes-Hut buffers (bl_bh.cu)
void bh_state_free(BHState* s);
}  // namespace bl

struct bl_layout {
    const bl_graph* g = nullptr;
    bl_force_params prm{1.0f, 1.0f, 0, -1, BL_MODEL_FR};
    int64_t t = 0;                      // iterations done
    bl::DevBuf pos;                     // float2[n] live positions
    bl::DevBuf pos2;                    // float2[n] second buffer (BH sweep)
    bl::DevBuf energy;                  // double[iters] of the last run
    bl::DevBuf epart;                   // double energy partials
    bl::DevBuf status;                  // int device status word + barrier counters
    bl::DevBuf scratch;                 // forces for debug hooks
    bl::DevBuf carry;                   // exact engine: row sums a launch leaves for the next
    mutable uint64_t carry_key = 0;     // launch shape those sums belong to (0: none valid)
    const void* carry_pos = nullptr;    // positions buffer they continue from
    int64_t last_iters = 0;
    double last_energy = 0.0;
    double pairs = 0.0, vupd = 0.0;
    double far_nodes = 0.0, near_pairs = 0.0;
    double last_ms = 0.0;
    bl::BHState* bh = nullptr;
    bl::Allocator alloc;
    int trace_steps = 0;                // phase trace of the next run (0 = off)
    bl::DevBuf trace;                   // uint64 timestamps
    int64_t trace_count = 0;            // entries written by the last traced run
    int phase_timing = 0;               // Barnes-Hut phase events on (bl_set_phase_timing)
    double phase_ms[9] = {};            // phase times of the last timed BH run (bl_get_phase_times)
    double phase_nodes = 0.0, phase_visits = 0.0;
    int64_t phase_iters = 0;
};

namespace bl {

// device status word values are bl_status codes
constexpr int kMaxBatch = 8192;
constexpr int kPhaseSlots = 9;    // Barnes-Hut phase times (bl_get_phase_times)
constexpr int kTraceSlots = 12;   // timestamps per CTA and step in a phase trace
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s per bounded wait

// ---------------------------------------------------------------------------
// exact engine (bl_exact.cu)
// ---------------------------------------------------------------------------

struct ExactTask {
    int n, BS, B;
    const int* rowptr;
    const int* colids;
    float2* pos;         // positions at launch start (iteration parity 0 buffer)
    float2* pos_alt;     // second position buffer (parity 1)
    double* e_iter;      // [iters * G] per-CTA energies per iteration, or null
    float2* f_out;       // snapshot mode: forces of all n vertices
    int iters;           // iterations in this launch (0 = snapshot mode)
    double step0;        // Step of the first iteration
    int crit_cap;        // most rows of one batch a CTA owns
    int nbr_cap;         // neighbour positions staged in shared memory
    unsigned long long* trace;   // optional phase timestamps [G][trace_steps][kTraceSlots]
    int trace_steps;
    int piece[16];       // one row per thread: bulk warp w's rows (see exact_plan)
    float4* carry;       // optional [G * ceil(n/G) * 2] row sums at the end of the launch
    int carry_in;        // 1: start from the sums in carry instead of the prologue
};

struct ExactParams {
    float invK;          // 1/K
    float negRK2;        // -R K^2
    int repulse_neighbors;
    int am;              // attraction exponent a of the (a,-1) model
    int kahan;           // 1: compensated repulsion sums across column tiles, 0: plain
    int* status;         // device status word
    unsigned* bar;       // step counter (one arrival per CTA per step)
};

// Launch shape of the grid engine: G co-resident CTAs of T threads, rpt rows per
// thread (row i lives on CTA i mod G).
struct ExactPlan {
    int G, T, rpt;
    int crit_cap, nbr_cap;   // see ExactTask
    int piece[16];           // one row per thread: block | halves << 16 | fold << 18
};
bl_status exact_plan(int n, int BS, int ctas_hint, int threads_hint, ExactPlan* out);

// Runs task.iters iterations (or the one-snapshot forces when iters == 0) of one
// graph on the grid engine. After an odd number of iterations the final
// positions are in task.pos_alt. Returns after queuing.
bl_status exact_launch(const ExactPlan& plan, const ExactTask& task, const ExactParams& prm,
                       cudaStream_t st);

// Ceiling probes of the pair loop and of rcp.approx (bl_measure_pair_rate).
bl_status exact_pair_rate(int threads, int skip_sp0, double* pairs_per_clk, double* rcp_per_clk,
                          double* pair_ms);

// Status word, grid-barrier counter and their reset (bl_runtime.cu).
bl_status layout_reset_sync_words(bl_layout* L, cudaStream_t st);
unsigned* layout_barrier_word(bl_layout* L);

// Per-iteration energies: energy[t] = sum over CTAs of e_iter[t][cta], in order.
bl_status energy_reduce(const double* e_iter, int iters, int G, double* energy, cudaStream_t st);

// Barnes-Hut iterations of one layout (bl_bh.cu); the caller updates L's counters.
// With sync, waits for the iterations and reads back the last walk's interaction
// counts (and phase times); without, returns once everything is queued on st.
bl_status bh_run(bl_layout* L, int iters, int BS, float theta, cudaStream_t st, bool sync = true);

// Compensated (Kahan) FP32 repulsion sums: bl_force_params.kahan = 1 always, 0
// never, < 0 from kKahanAutoN vertices on.
constexpr int64_t kKahanAutoN = 1000000;
inline bool kahan_on(int kahan, int64_t n) { return kahan > 0 || (kahan < 0 && n >= kKahanAutoN); }

// Attraction exponent a of an energy model (bl_energy_model): FR 2, FA 1, LinLog 0, A3 3.
inline int model_exponent(int energy_model) {
    static const int kA[4] = {2, 1, 0, 3};
    return (energy_model >= 0 && energy_model < 4) ? kA[energy_model] : 2;
}

// Exact mode on one thread-block cluster for small graphs (bl_exact_cluster.cu).
constexpr int kClusterMaxN = 8192;
constexpr int kClusterAutoN = 3072;   // measured crossover to the whole-GPU engine (n ~ 3,000)
bool cluster_engine_fits(int n, int BS, int64_t nnz);
// `iters` iterations of positions pos (updated in place); e_iter_buf holds
// iters x 16 doubles; energy (may be null) receives the per-iteration energies.
bl_status cluster_run(const int* rowptr, const int* colids, int64_t nnz, int n, float2* pos, int iters, int BS,
                      double step0, float invK, float negRK2, int rn, int am, int kahan, double* e_iter_buf,
                      double* energy, cudaStream_t st, int* C_out);

// Whole-GPU exact run of one layout (bl_runtime.cu); the caller updates L's counters.
bl_status exact_run(bl_layout* L, int iters, int BS, bool snapshot, float2* f_out, cudaStream_t st);

// SplitMix64-seeded positions uniform in [-1, 1), as bl_layout_init draws them.
void seeded_positions(int32_t n, uint64_t seed, float* xy);

// Frees a layout without synchronising: the caller has drained the stream its
// work ran on (bl_runtime.cu).
void layout_destroy(bl_layout* L);

// A layout whose positions are uploaded from xy (2n floats) or drawn from seed,
// without waiting for the upload (bl_runtime.cu). xy must stay valid until the
// stream reaches the copy.
bl_status layout_create(const bl_graph* g, const float* xy, uint64_t seed, int64_t start_iter,
                        const bl_force_params* params, bool sync, cudaStream_t st, bl_layout** out);

// ---------------------------------------------------------------------------
// batched engine (bl_batch.cu)
// ---------------------------------------------------------------------------

constexpr int kBatchMaxN = 16384;   // largest graph one CTA holds in shared memory
// Barnes-Hut: the quadtree reserves 17 n + 1 nodes (at most one per level and
// sorted position, plus the root) and indexes them with int32
constexpr int64_t kBHMaxN = (0x7fffffffLL - 1) / 17;
constexpr int kBatchMaxBS = 256;    // largest minibatch of the batched kernel

// Exact iterations of many layouts: graphs within the limits above go into one
// persistent launch per chunk of iterations (chunk <= 0: all at once), the rest
// through exact_run one at a time. Updates the layouts' counters; synchronises.
bl_status batch_run(bl_layout* const* Ls, int count, int iters, int BS, int chunk, cudaStream_t st,
                    double* elapsed_ms);

// One layout's share of a batched launch.
struct BatchJob {
    bl_layout* L;
    int iters;
    int BS;   // <= kBatchMaxBS
};
// Runs every job (each must satisfy n <= kBatchMaxN) in persistent launches of at
// most `chunk` iterations (chunk <= 0: one launch), captured into one CUDA graph.
// Updates the layouts' counters; synchronises.
bl_status batch_launch(const BatchJob* jobs, int count, int chunk, cudaStream_t st);

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace bl

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace bl {

// Squared distance floor for coincident pairs: a pair at distance 0 contributes
// (0,0) * (1/eps) = 0 exactly, which is the zero contribution the model gives
// coincident vertices; for any pair farther than ~1e-15 the term is unchanged.
#define BL_EPS2 1e-30f

__device__ __forceinline__ float rcp_sfu(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_sfu(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Repulsion of j on i before scaling by -R K^2: accumulates (c_j - c_i)/|c_j - c_i|^2.
__device__ __forceinline__ void rep_pair(float xi, float yi, float xj, float yj, float& ax,
                                         float& ay) {
    const float dx = xj - xi;
    const float dy = yj - yi;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, BL_EPS2));
    const float inv = rcp_sfu(d2);
    ax = fmaf(dx, inv, ax);
    ay = fmaf(dy, inv, ay);
}

// Kahan-compensated accumulation of v into (s, c); the sum is s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide barrier over a monotonically increasing counter, for cooperative
// launches (all CTAs co-resident). Every wait is bounded: after kWaitLimitNs the
// waiting CTA writes BL_ETIMEOUT to *status and every CTA leaves at its next check.
struct GridBarrier {
    unsigned* ctr;
    int* status;
    unsigned nblocks;
    unsigned phase;
    unsigned long long limit_ns = kWaitLimitNs;   // give up (BL_ETIMEOUT) after this long
    __device__ bool sync() {
        __syncthreads();
        __shared__ int s_ok;
        phase += 1;
        if (threadIdx.x == 0) {
            const unsigned target = phase * nblocks;
            __threadfence();
            red_release_add_u32(ctr, 1u);
            const unsigned long long t0 = global_ns();
            int ok = 1;
            for (unsigned spin = 0;; ++spin) {
                const unsigned v = ld_acquire_u32(ctr);
                if ((int)(v - target) >= 0) break;
                if ((spin & 255u) == 255u) {
                    if (ld_volatile_i32(status) != 0) { ok = 0; break; }
                    if (global_ns() - t0 > limit_ns) {
                        atomicCAS(status, 0, (int)BL_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

// The attraction of the (a,-1)-energy model along c_j - c_i: |d|^a / K times the
// unit vector = d^(a-1) / K (c_j - c_i). attr_scale(d2, a) = d^(a-1) from the
// squared distance (BL_EPS2 included, so a coincident pair gives 0).
__device__ __forceinline__ float attr_scale(float d2, int am) {
    switch (am) {
        case 2: return d2 * rsqrt_sfu(d2);   // d (Fruchterman-Reingold)
        case 1: return 1.0f;                 // ForceAtlas
        case 0: return rsqrt_sfu(d2);        // 1/d (LinLog)
        default: return d2;                  // a = 3: d^2
    }
}

// CSR terms of one neighbour: attraction d^(a-1)/K (c_j - c_i) (a = 2: (d/K)(c_j - c_i)),
// and, unless repulse_neighbors, the repulsion term the all-pairs sum gave this
// neighbour, computed with exactly rep_pair's expressions so that it cancels.
__device__ __forceinline__ void edge_terms(float xi, float yi, float2 p, float invK, int am, bool rn,
                                           float& ax, float& ay, float& qx, float& qy) {
    const float dx = p.x - xi;
    const float dy = p.y - yi;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, BL_EPS2));
    const float a = attr_scale(d2, am) * invK;
    ax = fmaf(dx, a, ax);
    ay = fmaf(dy, a, ay);
    if (!rn) {
        const float inv = rcp_sfu(d2);
        qx = fmaf(dx, inv, qx);
        qy = fmaf(dy, inv, qy);
    }
}

// ---- packed FP32x2 arithmetic (two columns per instruction) -----------------------
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

}  // namespace bl
#endif  // __CUDACC__
