// C ABI entry points and host runtime: error plumbing, allocator and stream
// hooks, CSR validation (Section 2.1), layout objects, dispatch to the engines.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bl_internal.cuh"

namespace bl {

static thread_local std::string g_last_error;
static std::mutex g_cfg_mu;
static cudaStream_t g_stream = nullptr;
static Allocator g_alloc;

bl_status set_error(bl_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

bl_status cuda_error(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return set_error(BL_ENOMEM, m);
    return set_error(BL_ECUDA, m);
}

cudaStream_t current_stream() {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    return g_stream;
}

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    return g_alloc;
}

bl_status dev_alloc(const Allocator& a, size_t bytes, void** p) {
    *p = nullptr;
    if (a.alloc) {
        *p = a.alloc(bytes, a.ctx);
        if (!*p) return set_error(BL_ENOMEM, "device allocation hook returned NULL");
        return BL_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_error(e, "cudaMalloc");
    }
    return BL_OK;
}

void dev_free(const Allocator& a, void* p) {
    if (!p) return;
    if (a.dealloc)
        a.dealloc(p, a.ctx);
    else
        cudaFree(p);
}

int device_sm_count() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev != cached_dev) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
        cached_dev = dev;
    }
    return cached;
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator: output k of
// the stream whose state starts at `seed`.
static inline uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void seeded_positions(int32_t n, uint64_t seed, float* xy) {
    for (int64_t k = 0; k < 2 * (int64_t)n; k++) {
        const uint64_t z = splitmix64_at(seed, (uint64_t)k);
        const double u = (double)(z >> 40) * (1.0 / 16777216.0);
        xy[k] = (float)(u * 2.0 - 1.0);
    }
}

static bl_status check_stream_status(bl_layout* L) {
    int st = 0;
    BL_CUDA_TRY(cudaMemcpy(&st, L->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        L->carry_key = 0;   // a failed run leaves no sums to continue from
        cudaMemset(L->status.p, 0, sizeof(int));
        return set_error((bl_status)st, st == BL_ETIMEOUT
                                            ? "a bounded device-side wait timed out"
                                            : "device-side error status");
    }
    return BL_OK;
}

bl_status layout_sync_status(bl_layout* L) {
    BL_CUDA_TRY(cudaStreamSynchronize(current_stream()));
    return check_stream_status(L);
}

// status word (int) + barrier counter (unsigned) + padding
static constexpr size_t kStatusBytes = 256;

bl_status layout_reset_sync_words(bl_layout* L, cudaStream_t st) {
    BL_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(L->status.p) + 64, 0, kStatusBytes - 64, st));
    return BL_OK;
}
unsigned* layout_barrier_word(bl_layout* L) {
    return reinterpret_cast<unsigned*>(static_cast<char*>(L->status.p) + 64);
}

// BH engine entry points (bl_bh.cu)

bl_status bh_debug_forces(bl_layout* L, float theta, float2* f_out, cudaStream_t st);
bl_status bh_debug_counts(bl_layout* L, float theta, int2* qcounts, cudaStream_t st);
bl_status bh_debug_tree(bl_layout* L, uint32_t* codes, int32_t* perm, int32_t* first,
                        int32_t* count, int32_t* level, int32_t* skip, float* sumx, float* sumy,
                        int64_t cap, int64_t* nnodes, float* box, cudaStream_t st);
// quality (bl_quality.cu)
bl_status quality_run(bl_layout* L, int32_t nsources, int32_t nqueries, uint64_t seed,
                      double* out, int64_t cap, cudaStream_t st);

// Identifies the launch shape and parameters a set of carried row sums belongs to
// (FNV-1a over the fields; never 0, which marks "none").
static uint64_t carry_key_of(const ExactPlan& pl, int BS, const bl_force_params& p) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* d, size_t len) {
        const unsigned char* b = static_cast<const unsigned char*>(d);
        for (size_t q = 0; q < len; q++) {
            h ^= b[q];
            h *= 1099511628211ull;
        }
    };
    const int shape[6] = {pl.G, pl.T, pl.rpt, pl.crit_cap, pl.nbr_cap, BS};
    mix(shape, sizeof(shape));
    mix(pl.piece, sizeof(pl.piece));
    const float kr[2] = {p.K, p.R};
    const int flags[3] = {p.repulse_neighbors, p.kahan, p.energy_model};
    mix(kr, sizeof(kr));
    mix(flags, sizeof(flags));
    return h | 1ull;
}

// Small graphs whose minibatch chain dominates run on one thread-block cluster
// (BL_EXACT_ENGINE=grid|cluster forces an engine).
static bool use_cluster_engine(const bl_layout* L, int BS) {
    const int n = L->g->n;
    if (!cluster_engine_fits(n, BS, L->g->nnz)) return false;
    if (const char* e = std::getenv("BL_EXACT_ENGINE")) return e[0] == 'c';
    return n <= kClusterAutoN;
}

bl_status exact_run(bl_layout* L, int iters, int BS, bool snapshot, float2* f_out,
                    cudaStream_t st) {
    const int n = L->g->n;
    if (!snapshot && iters > 0 && use_cluster_engine(L, BS)) {
        L->carry_key = 0;   // the positions move without the grid engine's sums
        double s = 1.0;
        for (int64_t k = 0; k < L->t; k++) s *= 0.999;
        BL_TRY(L->epart.ensure(L->alloc, (size_t)iters * 16 * sizeof(double)));
        BL_TRY(L->energy.ensure(L->alloc, (size_t)std::max(iters, 1) * sizeof(double)));
        return cluster_run(L->g->rowptr.as<int>(), L->g->colids.as<int>(), L->g->nnz, n, L->pos.as<float2>(),
                           iters, BS, s, 1.0f / L->prm.K, -L->prm.R * L->prm.K * L->prm.K,
                           L->prm.repulse_neighbors, model_exponent(L->prm.energy_model),
                           kahan_on(L->prm.kahan, n) ? 1 : 0, L->epart.as<double>(), L->energy.as<double>(),
                           st, nullptr);
    }
    ExactPlan plan;
    BL_TRY(exact_plan(n, BS, 0, 0, &plan));
    ExactTask tk{};
    tk.n = n;
    tk.BS = BS;
    tk.B = div_up(n, BS);
    tk.rowptr = L->g->rowptr.as<int>();
    tk.colids = L->g->colids.as<int>();
    BL_TRY(L->pos2.ensure(L->alloc, (size_t)n * sizeof(float2)));
    tk.pos = L->pos.as<float2>();
    tk.pos_alt = L->pos2.as<float2>();
    tk.crit_cap = plan.crit_cap;
    tk.nbr_cap = plan.nbr_cap;
    tk.iters = snapshot ? 0 : iters;
    {   // Step_t by repeated multiplication, as Algorithm 2 schedules it
        double s = 1.0;
        for (int64_t k = 0; k < L->t; k++) s *= 0.999;
        tk.step0 = s;
    }
    tk.f_out = f_out;
    if (!snapshot && L->trace_steps > 0) {
        const size_t tb = (size_t)plan.G * L->trace_steps * kTraceSlots * sizeof(unsigned long long);
        BL_TRY(L->trace.ensure(L->alloc, tb));
        BL_CUDA_TRY(cudaMemsetAsync(L->trace.p, 0, tb, st));
        tk.trace = L->trace.as<unsigned long long>();
        tk.trace_steps = L->trace_steps;
        L->trace_count = (int64_t)plan.G * L->trace_steps * kTraceSlots;
    }
    uint64_t key = 0;
    if (!snapshot) {
        BL_TRY(L->epart.ensure(L->alloc, (size_t)iters * plan.G * sizeof(double)));
        tk.e_iter = L->epart.as<double>();
        // Row sums carried between launches: a launch that continues the previous
        // one (same launch shape and parameters, positions untouched since) starts
        // from the sums that launch left instead of re-adding the columns after
        // each row's batch at the start positions.
        key = carry_key_of(plan, BS, L->prm);
        const bool cont = L->carry_key == key && L->carry_pos == L->pos.p;
        L->carry_key = 0;
        BL_TRY(L->carry.ensure(L->alloc, (size_t)plan.G * div_up(n, plan.G) * 2 * sizeof(float4)));
        tk.carry = L->carry.as<float4>();
        tk.carry_in = cont ? 1 : 0;
    }
    ExactParams prm{};
    prm.invK = 1.0f / L->prm.K;
    prm.negRK2 = -L->prm.R * L->prm.K * L->prm.K;
    prm.repulse_neighbors = L->prm.repulse_neighbors;
    prm.am = model_exponent(L->prm.energy_model);
    prm.kahan = kahan_on(L->prm.kahan, n) ? 1 : 0;
    prm.status = static_cast<int*>(L->status.p);
    prm.bar = layout_barrier_word(L);
    BL_TRY(layout_reset_sync_words(L, st));
    BL_TRY(exact_launch(plan, tk, prm, st));
    if (!snapshot) {
        BL_TRY(L->energy.ensure(L->alloc, (size_t)std::max(iters, 1) * sizeof(double)));
        BL_TRY(energy_reduce(L->epart.as<double>(), iters, plan.G, L->energy.as<double>(), st));
        if (iters & 1) std::swap(L->pos, L->pos2);   // final positions are in the other buffer
        L->carry_key = key;
        L->carry_pos = L->pos.p;
    }
    return BL_OK;
}

}  // namespace bl

namespace bl {
// Frees a layout's device memory; the caller has drained the stream its work ran on.
void layout_destroy(bl_layout* L) {
    if (!L) return;
    if (L->bh) bh_state_free(L->bh);
    L->pos.release();
    L->pos2.release();
    L->energy.release();
    L->epart.release();
    L->status.release();
    L->scratch.release();
    L->carry.release();
    L->trace.release();
    delete L;
}

bl_status layout_create(const bl_graph* g, const float* xy, uint64_t seed, int64_t start_iter,
                        const bl_force_params* params, bool sync, cudaStream_t st, bl_layout** out) {
    if (!out) return set_error(BL_EINVAL, "bl_layout_init: out is NULL");
    *out = nullptr;
    if (!g) return set_error(BL_EINVAL, "bl_layout_init: NULL graph");
    if (start_iter < 0) return set_error(BL_EINVAL, "bl_layout_init: start_iter < 0");
    bl_force_params p{1.0f, 1.0f, 0, -1, BL_MODEL_FR};
    if (params) p = *params;
    if (!(p.K > 0.0f) || !(p.R > 0.0f) || !std::isfinite(p.K) || !std::isfinite(p.R))
        return set_error(BL_EINVAL, "bl_layout_init: K and R must be positive and finite");
    if (p.energy_model < 0 || p.energy_model > 3)
        return set_error(BL_EINVAL, "bl_layout_init: energy_model must be 0..3");
    if (p.kahan < -1 || p.kahan > 1) return set_error(BL_EINVAL, "bl_layout_init: kahan must be -1, 0 or 1");
    bl_layout* L = new bl_layout();
    L->g = g;
    L->prm = p;
    L->t = start_iter;
    L->alloc = current_allocator();
    bl_status s = L->pos.ensure(L->alloc, (size_t)g->n * sizeof(float2));
    if (s == BL_OK) s = L->status.ensure(L->alloc, kStatusBytes);
    if (s == BL_OK) {
        std::vector<float> h;
        const float* src = xy;
        if (!src) {
            h.resize((size_t)2 * g->n);
            seeded_positions(g->n, seed, h.data());
            src = h.data();
        }
        cudaError_t e = cudaMemcpyAsync(L->pos.p, src, (size_t)g->n * sizeof(float2),
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(L->status.p, 0, kStatusBytes, st);
        if (e == cudaSuccess && (sync || !xy)) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "bl_layout_init: upload");
    }
    if (s != BL_OK) {
        cudaStreamSynchronize(st);
        layout_destroy(L);
        return s;
    }
    *out = L;
    return BL_OK;
}
}  // namespace bl

using namespace bl;

extern "C" {

bl_status bl_set_stream(void* stream) {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_stream = static_cast<cudaStream_t>(stream);
    return BL_OK;
}

bl_status bl_set_allocator(void* (*alloc)(size_t, void*), void (*dealloc)(void*, void*), void* ctx) {
    if ((alloc == nullptr) != (dealloc == nullptr))
        return set_error(BL_EINVAL, "bl_set_allocator: give both hooks or neither");
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_alloc.alloc = alloc;
    g_alloc.dealloc = dealloc;
    g_alloc.ctx = ctx;
    return BL_OK;
}

const char* bl_last_error(void) { return g_last_error.c_str(); }

const char* bl_version(void) { return "batchlayout-gb300 0.1 (sm_103a)"; }

bl_status bl_graph_load_csr(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colids,
                            uint32_t flags, bl_graph** out) {
    if (!out) return set_error(BL_EINVAL, "bl_graph_load_csr: out is NULL");
    *out = nullptr;
    if (n < 1) return set_error(BL_EINVAL, "bl_graph_load_csr: n must be >= 1");
    if (nnz < 0 || nnz > 0x7fffffffLL) return set_error(BL_EINVAL, "bl_graph_load_csr: nnz out of range");
    if (!rowptr || (nnz > 0 && !colids)) return set_error(BL_EINVAL, "bl_graph_load_csr: NULL array");
    if (rowptr[0] != 0 || rowptr[n] != nnz)
        return set_error(BL_EINVAL, "bl_graph_load_csr: rowptr[0] must be 0 and rowptr[n] = nnz");
    for (int32_t i = 0; i < n; i++)
        if (rowptr[i + 1] < rowptr[i]) return set_error(BL_EINVAL, "bl_graph_load_csr: rowptr decreases");
    for (int64_t k = 0; k < nnz; k++)
        if (colids[k] < 0 || colids[k] >= n)
            return set_error(BL_EINVAL, "bl_graph_load_csr: column id out of range");

    const bool sym = flags & BL_CSR_SYMMETRIZE, dedup = flags & BL_CSR_DEDUP;
    const bool sort = (flags & BL_CSR_SORT) || sym || dedup;
    std::vector<int32_t> rp(rowptr, rowptr + n + 1), ci(colids, colids + nnz);
    if (sym || sort || dedup) {
        std::vector<std::vector<int32_t>> rows(n);
        for (int32_t i = 0; i < n; i++)
            for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
                rows[i].push_back(ci[k]);
                if (sym) rows[ci[k]].push_back(i);
            }
        int64_t total = 0;
        for (int32_t i = 0; i < n; i++) {
            auto& r = rows[i];
            std::sort(r.begin(), r.end());
            if (dedup) {
                r.erase(std::unique(r.begin(), r.end()), r.end());
                r.erase(std::remove(r.begin(), r.end(), i), r.end());
            }
            total += (int64_t)r.size();
        }
        if (total > 0x7fffffffLL) return set_error(BL_EINVAL, "bl_graph_load_csr: graph too large");
        rp.assign(n + 1, 0);
        ci.clear();
        ci.reserve(total);
        for (int32_t i = 0; i < n; i++) {
            ci.insert(ci.end(), rows[i].begin(), rows[i].end());
            rp[i + 1] = (int32_t)ci.size();
        }
    }
    // validate the cleaned CSR: sorted, unique, no self-loops, symmetric
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            if (k > rp[i] && ci[k] <= ci[k - 1])
                return set_error(BL_EINVAL, "bl_graph_load_csr: row not strictly increasing (duplicates or unsorted)");
            if (ci[k] == i) return set_error(BL_EINVAL, "bl_graph_load_csr: self-loop");
        }
    for (int32_t i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            const int32_t j = ci[k];
            if (!std::binary_search(ci.begin() + rp[j], ci.begin() + rp[j + 1], i))
                return set_error(BL_EINVAL, "bl_graph_load_csr: graph is not symmetric");
        }
    bl_graph* g = new bl_graph();
    g->n = n;
    g->nnz = (int64_t)ci.size();
    g->h_rowptr.swap(rp);
    g->h_colids.swap(ci);
    const Allocator al = current_allocator();
    cudaStream_t st = current_stream();
    bl_status s = g->rowptr.ensure(al, (size_t)(n + 1) * sizeof(int32_t));
    if (s == BL_OK) s = g->colids.ensure(al, (size_t)std::max<int64_t>(g->nnz, 1) * sizeof(int32_t));
    if (s == BL_OK) {
        cudaError_t e = cudaMemcpyAsync(g->rowptr.p, g->h_rowptr.data(), (size_t)(n + 1) * sizeof(int32_t),
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && g->nnz > 0)
            e = cudaMemcpyAsync(g->colids.p, g->h_colids.data(), (size_t)g->nnz * sizeof(int32_t),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "bl_graph_load_csr: upload");
    }
    if (s != BL_OK) {
        g->rowptr.release();
        g->colids.release();
        delete g;
        return s;
    }
    *out = g;
    return BL_OK;
}

bl_status bl_graph_info(const bl_graph* g, int32_t* n, int64_t* nnz) {
    if (!g) return set_error(BL_EINVAL, "bl_graph_info: NULL graph");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return BL_OK;
}

void bl_graph_free(bl_graph* g) {
    if (!g) return;
    g->rowptr.release();
    g->colids.release();
    delete g;
}

bl_status bl_layout_init(const bl_graph* g, const float* xy, uint64_t seed, int64_t start_iter,
                         const bl_force_params* params, bl_layout** out) {
    return layout_create(g, xy, seed, start_iter, params, true, current_stream(), out);
}


// Greedy initialisation (Algorithm 3): a depth-first placement from v0 at (0, 0);
// a vertex U taken from the stack puts each of its not yet placed neighbours on
// the unit circle around U, the angle advancing by 360/deg(U) degrees after each,
// with the paper's PI = 3.1416. Positions are formed in double and stored as FP32.
// Vertices that v0 does not reach keep the seeded random positions. The walk is
// inherently sequential (its order defines the layout), O(n + m) on the host.
static void greedy_positions(const bl_graph* g, int v0, float* xy) {
    const int n = g->n;
    const int* rp = g->h_rowptr.data();
    const int* ci = g->h_colids.data();
    const double kPi = 3.1416;
    std::vector<double> px(n), py(n);
    std::vector<char> placed(n, 0);
    std::vector<int> stack;
    stack.reserve(n);
    px[v0] = 0.0;
    py[v0] = 0.0;
    placed[v0] = 1;
    stack.push_back(v0);
    while (!stack.empty()) {
        const int u = stack.back();
        stack.pop_back();
        const int deg = rp[u + 1] - rp[u];
        const double step = deg > 0 ? 360.0 / (double)deg : 0.0;
        double angle = 0.0;
        for (int e = rp[u]; e < rp[u + 1]; e++) {
            const int w = ci[e];
            if (placed[w]) continue;
            px[w] = px[u] + std::cos(kPi * angle / 180.0);
            py[w] = py[u] + std::sin(kPi * angle / 180.0);
            placed[w] = 1;
            stack.push_back(w);
            angle += step;
        }
    }
    for (int i = 0; i < n; i++)
        if (placed[i]) {
            xy[2 * i] = (float)px[i];
            xy[2 * i + 1] = (float)py[i];
        }
}

bl_status bl_layout_init_greedy(const bl_graph* g, int64_t v0, uint64_t seed, const bl_force_params* params,
                                bl_layout** out) {
    if (!out) return set_error(BL_EINVAL, "bl_layout_init_greedy: out is NULL");
    *out = nullptr;
    if (!g) return set_error(BL_EINVAL, "bl_layout_init_greedy: NULL graph");
    if (g->n == 0) return layout_create(g, nullptr, seed, 0, params, true, current_stream(), out);
    if (v0 >= g->n) return set_error(BL_EINVAL, "bl_layout_init_greedy: v0 out of range");
    if (v0 < 0) v0 = (int64_t)(splitmix64_at(seed, 0) % (uint64_t)g->n);
    std::vector<float> xy((size_t)2 * g->n);
    seeded_positions(g->n, seed, xy.data());
    greedy_positions(g, (int)v0, xy.data());
    return layout_create(g, xy.data(), seed, 0, params, true, current_stream(), out);
}

bl_status bl_layout_set_positions(bl_layout* L, const float* xy, int64_t start_iter) {
    if (!L || !xy) return set_error(BL_EINVAL, "bl_layout_set_positions: NULL argument");
    if (start_iter < 0) return set_error(BL_EINVAL, "bl_layout_set_positions: start_iter < 0");
    BL_CUDA_TRY(cudaMemcpyAsync(L->pos.p, xy, (size_t)L->g->n * sizeof(float2),
                                cudaMemcpyHostToDevice, current_stream()));
    L->carry_key = 0;
    L->t = start_iter;
    return BL_OK;
}

bl_status bl_layout_run(bl_layout* L, int32_t iters, int32_t batch, bl_mode mode, float theta) {
    if (!L) return set_error(BL_EINVAL, "bl_layout_run: NULL layout");
    if (iters < 0) return set_error(BL_EINVAL, "bl_layout_run: iters < 0");
    if (batch < 1 || batch > kMaxBatch) return set_error(BL_EINVAL, "bl_layout_run: batch must be in [1, 8192]");
    if (mode != BL_EXACT && mode != BL_BH) return set_error(BL_EINVAL, "bl_layout_run: mode must be BL_EXACT or BL_BH");
    if (mode == BL_BH && !(theta >= 0.0f)) return set_error(BL_EINVAL, "bl_layout_run: theta must be >= 0");
    if (mode == BL_EXACT && (int64_t)iters * div_up(L->g->n, batch) > 0x7fffffffLL)
        return set_error(BL_EINVAL, "bl_layout_run: more than 2^31 - 1 minibatch steps in one call; split the run");
    if (iters == 0) return BL_OK;
    cudaStream_t st = current_stream();
    EventPair ev;
    BL_CUDA_TRY(ev.create());
    BL_CUDA_TRY(cudaEventRecord(ev.e0, st));
    bl_status s = mode == BL_EXACT ? exact_run(L, iters, batch, false, nullptr, st)
                                   : bh_run(L, iters, batch, theta, st);
    if (s == BL_OK) {
        BL_CUDA_TRY(cudaEventRecord(ev.e1, st));
        BL_CUDA_TRY(cudaEventSynchronize(ev.e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.e0, ev.e1);
        L->last_ms = ms;
        s = check_stream_status(L);
    }
    if (s != BL_OK) return s;
    const double n = (double)L->g->n;
    L->last_iters = iters;
    L->t += iters;
    L->vupd += n * iters;
    if (mode == BL_EXACT) L->pairs += n * (n - 1.0) * iters;
    return BL_OK;
}

// Runs until the energy settles (Section 4.5 runs layouts to convergence, with
// successive iterations' energies differing by less than 1e-6; read relatively,
// |E_t - E_{t-1}| <= tol * max(E_{t-1}, 1), as energies are sums over all
// vertices). Iterations run in chunks; when the rule holds inside a chunk, the
// chunk's start positions are restored and only the iterations up to that point
// are run again, so the result is exactly that of stopping there (both engines
// give the same positions however iterations are split across launches).
bl_status bl_layout_run_until(bl_layout* L, int32_t max_iters, int32_t batch, bl_mode mode, float theta,
                              double tol, int32_t* iters_done, int32_t* converged) {
    if (!L) return set_error(BL_EINVAL, "bl_layout_run_until: NULL layout");
    if (max_iters < 0 || !(tol >= 0.0)) return set_error(BL_EINVAL, "bl_layout_run_until: bad max_iters or tol");
    if (iters_done) *iters_done = 0;
    if (converged) *converged = 0;
    const int n = L->g->n;
    cudaStream_t st = current_stream();
    BL_TRY(L->scratch.ensure(L->alloc, (size_t)std::max(n, 1) * sizeof(float2)));
    // the energy of the iteration before this call, when there is one
    double prev = 0.0;
    bool have_prev = false;
    if (L->last_iters > 0 && L->energy.p) {
        BL_CUDA_TRY(cudaMemcpyAsync(&prev, L->energy.as<double>() + (L->last_iters - 1), sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        BL_CUDA_TRY(cudaStreamSynchronize(st));
        have_prev = true;
    }
    const int chunk = mode == BL_EXACT ? 32 : 8;
    std::vector<double> hist;
    int done = 0;
    bool conv = false;
    while (done < max_iters && !conv) {
        const int c = std::min(chunk, max_iters - done);
        BL_CUDA_TRY(cudaMemcpyAsync(L->scratch.p, L->pos.p, (size_t)n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        const int64_t t0 = L->t;
        const double vupd0 = L->vupd, pairs0 = L->pairs;
        BL_TRY(bl_layout_run(L, c, batch, mode, theta));
        std::vector<double> e(c);
        int64_t cnt = 0;
        BL_TRY(bl_energy_history(L, e.data(), c, &cnt));
        int stop = c;
        for (int k = 0; k < c; k++) {
            if (have_prev && std::fabs(e[k] - prev) <= tol * std::max(prev, 1.0)) {
                stop = k + 1;
                conv = true;
                break;
            }
            prev = e[k];
            have_prev = true;
        }
        if (conv && stop < c) {   // back to the chunk's start, then exactly `stop` iterations
            BL_CUDA_TRY(cudaMemcpyAsync(L->pos.p, L->scratch.p, (size_t)n * sizeof(float2),
                                        cudaMemcpyDeviceToDevice, st));
            L->carry_key = 0;
            L->t = t0;
            L->vupd = vupd0;
            L->pairs = pairs0;
            BL_TRY(bl_layout_run(L, stop, batch, mode, theta));
        }
        hist.insert(hist.end(), e.begin(), e.begin() + stop);
        done += stop;
    }
    if (done > 0) {   // the call's whole energy history
        BL_TRY(L->energy.ensure(L->alloc, (size_t)done * sizeof(double)));
        BL_CUDA_TRY(cudaMemcpyAsync(L->energy.p, hist.data(), (size_t)done * sizeof(double),
                                    cudaMemcpyHostToDevice, st));
        BL_CUDA_TRY(cudaStreamSynchronize(st));
        L->last_iters = done;
    }
    if (iters_done) *iters_done = done;
    if (converged) *converged = conv ? 1 : 0;
    return BL_OK;
}

bl_status bl_positions(const bl_layout* L, float* xy, int64_t cap_floats) {
    if (!L || !xy) return set_error(BL_EINVAL, "bl_positions: NULL argument");
    if (cap_floats < 2 * (int64_t)L->g->n) return set_error(BL_EINVAL, "bl_positions: output too small");
    cudaStream_t st = current_stream();
    BL_CUDA_TRY(cudaMemcpyAsync(xy, L->pos.p, (size_t)L->g->n * sizeof(float2), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    return BL_OK;
}

bl_status bl_positions_device(const bl_layout* L, void** dptr) {
    if (!L || !dptr) return set_error(BL_EINVAL, "bl_positions_device: NULL argument");
    *dptr = L->pos.p;
    L->carry_key = 0;   // the caller may write the positions before the next run
    return BL_OK;
}

bl_status bl_energy_history(const bl_layout* L, double* out, int64_t cap, int64_t* count) {
    if (!L) return set_error(BL_EINVAL, "bl_energy_history: NULL layout");
    if (count) *count = L->last_iters;
    if (L->last_iters == 0 || out == nullptr) return BL_OK;   // NULL out: query the count
    if (cap < L->last_iters) return set_error(BL_EINVAL, "bl_energy_history: output too small");
    cudaStream_t st = current_stream();
    BL_CUDA_TRY(cudaMemcpyAsync(out, L->energy.p, (size_t)L->last_iters * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    return BL_OK;
}

bl_status bl_stats(const bl_layout* L, bl_stats_t* out) {
    if (!L || !out) return set_error(BL_EINVAL, "bl_stats: NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->iterations = L->t;
    double s = 1.0;
    for (int64_t k = 0; k < L->t; k++) s *= 0.999;
    out->step = s;
    if (L->last_iters > 0 && L->energy.p) {
        double e = 0.0;
        cudaStream_t st = current_stream();
        BL_CUDA_TRY(cudaMemcpyAsync(&e, L->energy.as<double>() + (L->last_iters - 1), sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        BL_CUDA_TRY(cudaStreamSynchronize(st));
        out->energy = e;
    }
    out->pair_interactions = L->pairs;
    out->vertex_updates = L->vupd;
    out->bh_far_nodes = L->far_nodes;
    out->bh_near_pairs = L->near_pairs;
    out->last_run_ms = L->last_ms;
    return BL_OK;
}

void bl_layout_free(bl_layout* L) {
    if (!L) return;
    cudaStreamSynchronize(current_stream());   // nothing of this layout may still be running
    layout_destroy(L);
}

bl_status bl_quality(const bl_layout* L, int32_t nsources, int32_t nqueries, uint64_t seed,
                     double* out, int64_t cap) {
    if (!L || !out) return set_error(BL_EINVAL, "bl_quality: NULL argument");
    if (cap < 6) return set_error(BL_EINVAL, "bl_quality: output needs 6 doubles");
    return quality_run(const_cast<bl_layout*>(L), nsources, nqueries, seed, out, cap, current_stream());
}

bl_status bl_debug_forces(bl_layout* L, bl_mode mode, float theta, int32_t lo, int32_t hi,
                          float* f_out) {
    if (!L || !f_out) return set_error(BL_EINVAL, "bl_debug_forces: NULL argument");
    const int n = L->g->n;
    if (lo < 0 || hi > n || lo > hi) return set_error(BL_EINVAL, "bl_debug_forces: bad range");
    if (mode != BL_EXACT && mode != BL_BH) return set_error(BL_EINVAL, "bl_debug_forces: bad mode");
    cudaStream_t st = current_stream();
    BL_TRY(L->scratch.ensure(L->alloc, (size_t)n * sizeof(float2)));
    float2* f = L->scratch.as<float2>();
    if (mode == BL_EXACT) {
        // one batch per CTA-sized slice; the batch size does not change snapshot forces
        BL_TRY(exact_run(L, 0, std::min(n, 1024), true, f, st));
    } else {
        BL_TRY(bh_debug_forces(L, theta, f, st));
    }
    BL_CUDA_TRY(cudaMemcpyAsync(f_out, f + lo, (size_t)(hi - lo) * sizeof(float2), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    return check_stream_status(L);
}

bl_status bl_debug_bh_counts(bl_layout* L, float theta, int32_t* far, int32_t* near, int64_t cap) {
    if (!L || !far || !near) return set_error(BL_EINVAL, "bl_debug_bh_counts: NULL argument");
    const int n = L->g->n;
    if (cap < n) return set_error(BL_EINVAL, "bl_debug_bh_counts: output too small");
    if (!(theta >= 0.0f)) return set_error(BL_EINVAL, "bl_debug_bh_counts: theta must be >= 0");
    cudaStream_t st = current_stream();
    BL_TRY(L->scratch.ensure(L->alloc, (size_t)n * sizeof(int2)));
    int2* q = L->scratch.as<int2>();
    BL_TRY(bh_debug_counts(L, theta, q, st));
    std::vector<int2> h((size_t)n);
    BL_CUDA_TRY(cudaMemcpyAsync(h.data(), q, (size_t)n * sizeof(int2), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n; i++) {
        far[i] = h[i].x;
        near[i] = h[i].y;
    }
    return BL_OK;
}

bl_status bl_set_phase_timing(bl_layout* L, int32_t on) {
    if (!L) return set_error(BL_EINVAL, "bl_set_phase_timing: NULL layout");
    L->phase_timing = on != 0;
    return BL_OK;
}

bl_status bl_measure_pair_rate(int32_t threads, int32_t skip_sp0, double* out, int64_t cap) {
    if (!out || cap < 4) return set_error(BL_EINVAL, "bl_measure_pair_rate: output needs 4 doubles");
    double ppc = 0.0, rpc = 0.0, ms = 0.0;
    BL_TRY(exact_pair_rate(threads, skip_sp0, &ppc, &rpc, &ms));
    const int warps = threads / 32;
    const double active = skip_sp0 ? warps - (warps + 3) / 4 : warps;
    const double pairs = (double)device_sm_count() * active * 32 * 256.0 * 400;
    out[0] = ppc;
    out[1] = rpc;
    out[2] = ms;
    out[3] = ms > 0 && ppc > 0 ? pairs / (ms * 1e-3) / (ppc * device_sm_count()) / 1e6 : 0.0;
    return BL_OK;
}

bl_status bl_get_phase_times(const bl_layout* L, double* out, int64_t cap) {
    if (!L || !out) return set_error(BL_EINVAL, "bl_get_phase_times: NULL argument");
    if (cap < kPhaseSlots + 3) return set_error(BL_EINVAL, "bl_get_phase_times: output needs 12 doubles");
    for (int q = 0; q < kPhaseSlots; q++) out[q] = L->phase_ms[q];
    out[kPhaseSlots] = L->phase_nodes;
    out[kPhaseSlots + 1] = L->phase_visits;
    out[kPhaseSlots + 2] = (double)L->phase_iters;
    return BL_OK;
}

bl_status bl_set_trace(bl_layout* L, int32_t max_steps) {
    if (!L || max_steps < 0) return set_error(BL_EINVAL, "bl_set_trace: bad argument");
    L->trace_steps = max_steps;
    return BL_OK;
}

bl_status bl_get_trace(const bl_layout* L, uint64_t* out, int64_t cap, int64_t* count) {
    if (!L || !count) return set_error(BL_EINVAL, "bl_get_trace: NULL argument");
    *count = L->trace_count;
    if (!out || L->trace_count == 0) return BL_OK;
    if (cap < L->trace_count) return set_error(BL_EINVAL, "bl_get_trace: output too small");
    cudaStream_t st = current_stream();
    BL_CUDA_TRY(cudaMemcpyAsync(out, L->trace.p, (size_t)L->trace_count * sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    return BL_OK;
}

bl_status bl_debug_bh_tree(bl_layout* L, uint32_t* codes, int32_t* perm, int32_t* first,
                           int32_t* count, int32_t* level, int32_t* skip, float* sumx, float* sumy,
                           int64_t cap, int64_t* nnodes, float* box) {
    if (!L || !nnodes) return set_error(BL_EINVAL, "bl_debug_bh_tree: NULL argument");
    return bh_debug_tree(L, codes, perm, first, count, level, skip, sumx, sumy, cap, nnodes, box,
                         current_stream());
}

}  // extern "C"
