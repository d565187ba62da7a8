// Many small graphs in one persistent launch (exact mode, Algorithm 2 per graph).
//
// Each CTA lays out one graph at a time with the graph's positions and row
// offsets resident in shared memory; CTAs take graphs from a work list ordered
// largest first. A minibatch step is three phases separated by CTA barriers:
//   A  all-pairs repulsion of the minibatch's rows (64 at a time) against every
//      column, packed FP32x2 over column pairs, one SFU reciprocal per pair;
//   B  four threads per row: the row's stripe sums, attraction and neighbour
//      correction over its CSR row, the update and its energy;
//   C  the new positions of the minibatch are written back (Jacobi inside the
//      minibatch, Gauss-Seidel across minibatches).
// The summation order of every row is fixed by the data alone (8 column stripes,
// folded every 16 column pairs, fixed reduction trees), so every launch shape the
// autotuner may pick gives bit-identical positions, and a graph's result does not
// depend on which other graphs share the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "bl_internal.cuh"

namespace bl {
namespace {

constexpr int kStripes = 8;      // column stripes per row
constexpr int kFold = 16;        // column pairs of a stripe between folds
constexpr int kRows = 64;        // rows per pass
constexpr int kMaxPasses = kBatchMaxBS / kRows;
constexpr float kPad = 1e30f;    // padding column: its terms are exactly zero

struct BatchItem {
    const int* rowptr;
    const int* colids;
    float2* pos;          // in/out
    double* energy;       // [iters] energy of each iteration of this launch
    double step0;         // Step at the first iteration of this launch
    int n, BS, iters, rn;
    float invK, negRK2;
    int am;               // attraction exponent a of the (a,-1) model
    int kahan;            // 1: the folds of each stripe sum compensated
};

struct BatchArgs {
    const BatchItem* items;
    int nitems;
    unsigned* next;       // work-list cursor, zero at launch
    int ncap;             // largest n the shared-memory carve-out holds
};

__host__ __device__ inline size_t batch_smem_bytes(int ncap) {
    const size_t np = (size_t)(ncap + 1) / 2;
    const size_t rp = ((size_t)(ncap + 1) * 4 + 15) / 16 * 16;
    return np * 16 + rp + 2 * kStripes * kRows * sizeof(float2) + kBatchMaxBS * sizeof(float2) +
           kRows * sizeof(double);
}

__device__ __forceinline__ float2 spos(const float* sp, int i) {
    const int b = 4 * (i >> 1) + (i & 1);
    return make_float2(sp[b], sp[b + 2]);
}

// Phase A: stripe sums of rows [p0, pend) into part[stripe][row - p0].
template <int T, int RPT>
__device__ __forceinline__ void phase_a(const float4* __restrict__ s_pos4, int np, int p0, int pend,
                                        bool kahan, float2* __restrict__ part) {
    constexpr int W = T / 32;
    constexpr int NG = 2 / RPT;   // row groups of 32*RPT rows per pass
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* sp = reinterpret_cast<const float*>(s_pos4);
    const f32x2 E = pk2(BL_EPS2, BL_EPS2);
    for (int item = warp; item < kStripes * NG; item += W) {
        const int s = item % kStripes;
        const int gr = item / kStripes;
        f32x2 XI[RPT], YI[RPT], AX[RPT], AY[RPT];
        float SX[RPT], SY[RPT], CX[RPT], CY[RPT];
#pragma unroll
        for (int m = 0; m < RPT; m++) {
            const int i = p0 + gr * 32 * RPT + m * 32 + lane;
            const float2 me = spos(sp, i < pend ? i : p0);
            XI[m] = pk2(me.x, me.x);
            YI[m] = pk2(me.y, me.y);
            AX[m] = AY[m] = pk2(0.f, 0.f);
            SX[m] = SY[m] = CX[m] = CY[m] = 0.f;
        }
        for (int qc = s; qc < np; qc += kStripes * kFold) {
            const int kend = min(kFold, (np - qc + kStripes - 1) / kStripes);
#pragma unroll 16   // a whole fold: 16 column pairs of loads and reciprocals in flight
            for (int k = 0; k < kend; k++) {
                const float4 p = s_pos4[qc + k * kStripes];
                const f32x2 X = pk2(p.x, p.y), Y = pk2(p.z, p.w);
#pragma unroll
                for (int m = 0; m < RPT; m++) {
                    f32x2 dx, dy, d2;
                    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(X), "l"(XI[m]));
                    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(Y), "l"(YI[m]));
                    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d2) : "l"(dy), "l"(E));
                    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d2) : "l"(dx), "l"(d2));
                    float da, db;
                    upk2(d2, da, db);
                    const f32x2 inv = pk2(rcp_sfu(da), rcp_sfu(db));
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(AX[m]) : "l"(dx), "l"(inv));
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(AY[m]) : "l"(dy), "l"(inv));
                }
            }
#pragma unroll
            for (int m = 0; m < RPT; m++) {
                float a0, a1, b0, b1;
                upk2(AX[m], a0, a1);
                upk2(AY[m], b0, b1);
                if (kahan) {   // compensated over the stripe's folds (uniform branch)
                    kahan_add(SX[m], CX[m], a0 + a1);
                    kahan_add(SY[m], CY[m], b0 + b1);
                } else {
                    SX[m] += a0 + a1;
                    SY[m] += b0 + b1;
                }
                AX[m] = AY[m] = pk2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int m = 0; m < RPT; m++) {
            const int r = gr * 32 * RPT + m * 32 + lane;
            part[s * kRows + r] = make_float2(SX[m] - CX[m], SY[m] - CY[m]);
        }
    }
}

template <int T, int RPT>
__global__ void __launch_bounds__(T, (768 / T > 0 ? 768 / T : 1)) batch_kernel(BatchArgs a) {
    constexpr int VPT = T >= 256 ? 1 : 256 / T;   // virtual phase-B threads per thread
    extern __shared__ __align__(16) unsigned char smem[];
    const int npcap = (a.ncap + 1) / 2;
    float4* s_pos4 = reinterpret_cast<float4*>(smem);
    int* s_rp = reinterpret_cast<int*>(smem + (size_t)npcap * 16);
    float2* s_part = reinterpret_cast<float2*>(smem + (size_t)npcap * 16 +
                                               ((size_t)(a.ncap + 1) * 4 + 15) / 16 * 16);
    float2* s_new = s_part + 2 * kStripes * kRows;   // [BS] new positions of the minibatch
    double* s_e = reinterpret_cast<double*>(s_new + kBatchMaxBS);
    float* sp = reinterpret_cast<float*>(s_pos4);
    __shared__ int s_item;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(a.next, 1u);
        __syncthreads();
        const int idx = s_item;
        if (idx >= a.nitems) break;
        const BatchItem g = a.items[idx];
        const int n = g.n, np = (n + 1) / 2;
        for (int q = tid; q < np; q += T) {
            const float2 u = g.pos[2 * q];
            const float2 v = 2 * q + 1 < n ? g.pos[2 * q + 1] : make_float2(kPad, kPad);
            s_pos4[q] = make_float4(u.x, v.x, u.y, v.y);
        }
        for (int i = tid; i <= n; i += T) s_rp[i] = g.rowptr[i];
        double e_slot[VPT];
#pragma unroll
        for (int vv = 0; vv < VPT; vv++) e_slot[vv] = 0.0;
        __syncthreads();
        double step = g.step0;
        for (int t = 0; t < g.iters; t++) {
            const float stepf = (float)step;
            for (int r0 = 0; r0 < n; r0 += g.BS) {
                const int r1 = min(r0 + g.BS, n);
#pragma unroll
                for (int pass = 0; pass < kMaxPasses; pass++) {
                    const int p0 = r0 + pass * kRows;
                    if (p0 >= r1) break;
                    const int pend = min(p0 + kRows, r1);
                    float2* part = s_part + (pass & 1) * kStripes * kRows;
                    phase_a<T, RPT>(s_pos4, np, p0, pend, g.kahan != 0, part);
                    __syncthreads();
                    // Phase B: virtual thread v -> row v/4, sub-thread v%4
#pragma unroll
                    for (int vv = 0; vv < VPT; vv++) {
                        const int v = tid + vv * T;
                        if (v >= 4 * kRows) break;   // whole warps
                        const int r = v >> 2, k = v & 3;
                        const int i = p0 + r;
                        const bool valid = i < pend;
                        const float2 sa = part[(2 * k) * kRows + r];
                        const float2 sb = part[(2 * k + 1) * kRows + r];
                        float px = sa.x + sb.x, py = sa.y + sb.y;
                        px += __shfl_xor_sync(0xffffffffu, px, 1);
                        py += __shfl_xor_sync(0xffffffffu, py, 1);
                        px += __shfl_xor_sync(0xffffffffu, px, 2);
                        py += __shfl_xor_sync(0xffffffffu, py, 2);
                        float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
                        const float2 me = spos(sp, valid ? i : p0);
                        if (valid) {
                            const int e1 = s_rp[i + 1];
                            for (int e = s_rp[i] + k; e < e1; e += 4)
                                edge_terms(me.x, me.y, spos(sp, __ldg(&g.colids[e])), g.invK, g.am, g.rn != 0,
                                           ax, ay, qx, qy);
                        }
#pragma unroll
                        for (int o = 1; o <= 2; o <<= 1) {
                            ax += __shfl_xor_sync(0xffffffffu, ax, o);
                            ay += __shfl_xor_sync(0xffffffffu, ay, o);
                            qx += __shfl_xor_sync(0xffffffffu, qx, o);
                            qy += __shfl_xor_sync(0xffffffffu, qy, o);
                        }
                        float2 np2 = me;
                        if (valid && k == 0) {
                            const float fx = fmaf(g.negRK2, px - qx, ax);
                            const float fy = fmaf(g.negRK2, py - qy, ay);
                            float gx = fx, gy = fy;
                            float n2 = fmaf(gx, gx, gy * gy);
                            if (n2 > 0.f) {
                                if (!(n2 < INFINITY)) {
                                    gx *= 0x1p-64f;
                                    gy *= 0x1p-64f;
                                    n2 = fmaf(gx, gx, gy * gy);
                                }
                                const float sc = stepf * rsqrt_sfu(n2);
                                np2 = make_float2(fmaf(sc, gx, me.x), fmaf(sc, gy, me.y));
                            }
                            e_slot[vv] += (double)fmaf(fx, fx, fy * fy);
                        }
                        if (k == 0 && valid) s_new[i - r0] = np2;
                    }
                }
                __syncthreads();
                // Phase C: the minibatch moves
                for (int i = r0 + tid; i < r1; i += T) {
                    const float2 q = s_new[i - r0];
                    const int b = 4 * (i >> 1) + (i & 1);
                    sp[b] = q.x;
                    sp[b + 2] = q.y;
                }
                __syncthreads();
            }
            // energy of iteration t: row slots in order
#pragma unroll
            for (int vv = 0; vv < VPT; vv++) {
                const int v = tid + vv * T;
                if (v < 4 * kRows && (v & 3) == 0) s_e[v >> 2] = e_slot[vv];
                e_slot[vv] = 0.0;
            }
            __syncthreads();
            if (tid == 0) {
                double e = 0.0;
                for (int r = 0; r < kRows; r++) e += s_e[r];
                g.energy[t] = e;
            }
            step *= 0.999;   // Algorithm 2: Step = Step * 0.999
        }
        for (int i = tid; i < n; i += T) g.pos[i] = spos(sp, i);
        __syncthreads();
    }
}

// ---- launch shapes the autotuner chooses from ------------------------------------
struct Shape {
    int T, RPT;
    const void* fn;
};
const Shape kShapes[] = {
    {256, 2, (const void*)batch_kernel<256, 2>},
    {256, 1, (const void*)batch_kernel<256, 1>},
    {512, 1, (const void*)batch_kernel<512, 1>},
    {128, 2, (const void*)batch_kernel<128, 2>},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

std::mutex g_tune_mu;
std::map<long long, int> g_tuned;   // (device, carve-out class) -> shape

int size_class(int ncap) {
    int c = 256;
    while (c < ncap) c *= 2;
    return c;
}

bl_status shape_grid(int shape, int ncap, int nitems, int* grid) {
    const Shape& sh = kShapes[shape];
    const size_t smem = batch_smem_bytes(ncap);
    BL_CUDA_TRY(cudaFuncSetAttribute(sh.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    BL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sh.fn, sh.T, smem));
    if (occ < 1) return set_error(BL_EINVAL, "batched layout: a graph does not fit one CTA's shared memory");
    *grid = std::max(1, std::min(occ * device_sm_count(), nitems));
    return BL_OK;
}

bl_status launch_shape(int shape, int ncap, const BatchItem* items, int nitems, unsigned* next,
                       cudaStream_t st) {
    int grid = 0;
    BL_TRY(shape_grid(shape, ncap, nitems, &grid));
    BL_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(unsigned), st));
    BatchArgs args{items, nitems, next, ncap};
    void* kargs[] = {&args};
    BL_CUDA_TRY(cudaLaunchKernel(kShapes[shape].fn, dim3(grid), dim3(kShapes[shape].T), kargs,
                                 batch_smem_bytes(ncap), st));
    return BL_OK;
}

// Times every shape on a copy of the work (10 iterations) and keeps the fastest
// for this carve-out class. Positions of the real layouts are not touched.
bl_status autotune(int ncap, const std::vector<BatchItem>& work, const Allocator& al, cudaStream_t st,
                   int* shape_out) {
    int dev = 0;
    BL_CUDA_TRY(cudaGetDevice(&dev));
    const long long key = ((long long)dev << 32) | (long long)size_class(ncap);
    if (const char* f = std::getenv("BL_BATCH_SHAPE")) {
        const int v = std::atoi(f);
        if (v >= 0 && v < kNumShapes) {
            *shape_out = v;
            return BL_OK;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *shape_out = it->second;
            return BL_OK;
        }
    }
    // too few graphs to tell the shapes apart (they differ in how CTAs share an
    // SM): the shape measured best on a large mix, not remembered
    if ((int)work.size() < 4 * device_sm_count()) {
        *shape_out = 0;
        return BL_OK;
    }
    // the whole work list up to 8,192 graphs (every k-th beyond): the shapes
    // differ in how many CTAs share an SM, which only shows when the launch has
    // enough graphs to fill every CTA slot several times
    const int want = 8192;
    const int stride = std::max<int>(1, (int)((work.size() + want - 1) / want));
    std::vector<BatchItem> smp;
    size_t pos_floats = 0;
    for (size_t k = 0; k < work.size(); k += stride) {
        smp.push_back(work[k]);
        pos_floats += 2 * (size_t)work[k].n;
    }
    // scratch copies of the sample, freed (after the stream drains) on every return
    struct Scratch {
        cudaStream_t st;
        DevBuf pos, en, items, cur;
        EventPair ev;
        ~Scratch() {
            cudaStreamSynchronize(st);
            for (DevBuf* b : {&pos, &en, &items, &cur}) b->release();
        }
    } sc{st, {}, {}, {}, {}, {}};
    DevBuf &pos = sc.pos, &en = sc.en, &items = sc.items, &cur = sc.cur;
    BL_TRY(pos.ensure(al, pos_floats * sizeof(float)));
    BL_TRY(en.ensure(al, smp.size() * 10 * sizeof(double)));
    BL_TRY(items.ensure(al, smp.size() * sizeof(BatchItem)));
    BL_TRY(cur.ensure(al, 16));
    size_t off = 0;
    for (size_t k = 0; k < smp.size(); k++) {
        float2* dst = pos.as<float2>() + off / 2;
        BL_CUDA_TRY(cudaMemcpyAsync(dst, smp[k].pos, (size_t)smp[k].n * sizeof(float2),
                                    cudaMemcpyDeviceToDevice, st));
        smp[k].pos = dst;
        smp[k].energy = en.as<double>() + 10 * k;
        smp[k].iters = std::min(smp[k].iters, 10);
        off += 2 * (size_t)smp[k].n;
    }
    BL_CUDA_TRY(cudaMemcpyAsync(items.p, smp.data(), smp.size() * sizeof(BatchItem),
                                cudaMemcpyHostToDevice, st));
    BL_CUDA_TRY(sc.ev.create());
    const cudaEvent_t e0 = sc.ev.e0, e1 = sc.ev.e1;
    int best = 0;
    float best_ms = 0.f;
    bl_status s = BL_OK;
    for (int sh = 0; sh < kNumShapes && s == BL_OK; sh++) {
        for (int rep = 0; rep < 2 && s == BL_OK; rep++) {   // first pass warms up
            cudaEventRecord(e0, st);
            s = launch_shape(sh, ncap, items.as<BatchItem>(), (int)smp.size(), cur.as<unsigned>(), st);
            cudaEventRecord(e1, st);
        }
        if (s != BL_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        // shape 0 (the best on a large mix) unless another is clearly faster:
        // near-equal timings would otherwise flip the choice from run to run
        if (sh == 0 || ms < 0.97f * best_ms) {
            best = sh;
            best_ms = ms;
        }
    }
    if (s != BL_OK) return s;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    *shape_out = best;
    return BL_OK;
}

}  // namespace

// Jobs in persistent launches of at most `chunk` iterations; the launches are
// captured once into a CUDA graph and replayed. Each launch's work list holds the
// jobs with iterations left in that chunk, largest graph first.
bl_status batch_launch(const BatchJob* jobs, int count, int chunk, cudaStream_t st) {
    int max_it = 0, ncap = 1;
    for (int k = 0; k < count; k++) {
        if (jobs[k].L->g->n > kBatchMaxN || jobs[k].BS < 1 || jobs[k].BS > kBatchMaxBS)
            return set_error(BL_EINVAL, "batched layout: graph or minibatch above the batched kernel's limits");
        max_it = std::max(max_it, jobs[k].iters);
        ncap = std::max(ncap, jobs[k].L->g->n);
    }
    if (count == 0 || max_it == 0) return BL_OK;
    ncap = std::min((ncap + 63) / 64 * 64, kBatchMaxN);
    if (chunk <= 0 || chunk > max_it) chunk = max_it;
    const int nchunks = (max_it + chunk - 1) / chunk;
    std::vector<int> order(count);
    for (int k = 0; k < count; k++) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const int na = jobs[a].L->g->n, nb = jobs[b].L->g->n;
        return na != nb ? na > nb : a < b;
    });
    const Allocator al = current_allocator();
    std::vector<BatchItem> items;
    std::vector<int> first(nchunks + 1, 0);
    for (int j = 0; j < count; j++) {
        bl_layout* L = jobs[j].L;
        BL_TRY(L->energy.ensure(L->alloc, (size_t)std::max(jobs[j].iters, 1) * sizeof(double)));
    }
    for (int c = 0; c < nchunks; c++) {
        first[c] = (int)items.size();
        for (int j : order) {
            const BatchJob& jb = jobs[j];
            const int it0 = c * chunk;
            if (it0 >= jb.iters) continue;
            bl_layout* L = jb.L;
            L->carry_key = 0;   // the exact engine's carried sums do not follow these moves
            double step = 1.0;
            for (int64_t q = 0; q < L->t + it0; q++) step *= 0.999;
            BatchItem it{};
            it.rowptr = L->g->rowptr.as<int>();
            it.colids = L->g->colids.as<int>();
            it.pos = L->pos.as<float2>();
            it.energy = L->energy.as<double>() + it0;
            it.step0 = step;
            it.n = L->g->n;
            it.BS = jb.BS;
            it.iters = std::min(chunk, jb.iters - it0);
            it.rn = L->prm.repulse_neighbors;
            it.invK = 1.0f / L->prm.K;
            it.negRK2 = -L->prm.R * L->prm.K * L->prm.K;
            it.am = model_exponent(L->prm.energy_model);
            it.kahan = kahan_on(L->prm.kahan, L->g->n) ? 1 : 0;
            items.push_back(it);
        }
    }
    first[nchunks] = (int)items.size();
    int shape = 0;
    {
        std::vector<BatchItem> sample(items.begin(), items.begin() + first[1]);
        BL_TRY(autotune(ncap, sample, al, st, &shape));
    }
    DevBuf ditems, dnext;
    bl_status s = ditems.ensure(al, items.size() * sizeof(BatchItem));
    if (s == BL_OK) s = dnext.ensure(al, (size_t)nchunks * 16);
    if (s == BL_OK) {
        const cudaError_t e = cudaMemcpyAsync(ditems.p, items.data(), items.size() * sizeof(BatchItem),
                                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_error(e, "batched layout: work list upload");
    }
    int grid = 0;
    if (s == BL_OK) s = shape_grid(shape, ncap, first[1], &grid);
    if (s == BL_OK) {
        cudaStream_t cs = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int c = 0; c < nchunks && e == cudaSuccess; c++) {
            unsigned* next = reinterpret_cast<unsigned*>(static_cast<char*>(dnext.p) + 16 * c);
            e = cudaMemsetAsync(next, 0, sizeof(unsigned), cs);
            BatchArgs args{ditems.as<BatchItem>() + first[c], first[c + 1] - first[c], next, ncap};
            void* kargs[] = {&args};
            if (e == cudaSuccess)
                e = cudaLaunchKernel(kShapes[shape].fn, dim3(grid), dim3(kShapes[shape].T), kargs,
                                     batch_smem_bytes(ncap), cs);
        }
        if (cs) {
            const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "batched layout: graph launch");
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
    }
    ditems.release();
    dnext.release();
    if (s != BL_OK) return s;
    for (int j = 0; j < count; j++) {
        bl_layout* L = jobs[j].L;
        const double n = (double)L->g->n;
        const int it = jobs[j].iters;
        L->last_iters = it;
        L->t += it;
        L->vupd += n * it;
        L->pairs += n * (n - 1.0) * it;
    }
    return BL_OK;
}

// Runs `iters` iterations of every layout in Ls (exact mode, minibatch BS).
// Graphs that fit the batched kernel share its launches; a graph whose work is
// above one SM's fair share (and any graph above the kernel's limits) runs on the
// whole-GPU engine afterwards, one at a time.
bl_status batch_run(bl_layout* const* Ls, int count, int iters, int BS, int chunk, cudaStream_t st,
                    double* elapsed_ms) {
    if (count == 0 || iters == 0) return BL_OK;
    const int sms = device_sm_count();
    double total = 0.0;
    for (int k = 0; k < count; k++) {
        const double n = Ls[k]->g->n;
        total += n * n;
    }
    std::vector<BatchJob> small;
    std::vector<bl_layout*> big;
    for (int k = 0; k < count; k++) {
        const int n = Ls[k]->g->n;
        const double w = (double)n * n;
        const bool fits = n <= kBatchMaxN && BS <= kBatchMaxBS && (w <= total / sms || n <= 2048);
        if (fits) small.push_back(BatchJob{Ls[k], iters, BS});
        else big.push_back(Ls[k]);
    }
    EventPair ev;
    BL_CUDA_TRY(ev.create());
    const cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    BL_CUDA_TRY(cudaEventRecord(e0, st));
    bl_status s = batch_launch(small.data(), (int)small.size(), chunk, st);
    for (size_t q = 0; q < big.size() && s == BL_OK; q++) {
        bl_layout* L = big[q];
        s = exact_run(L, iters, BS, false, nullptr, st);
        if (s == BL_OK) {
            const double n = (double)L->g->n;
            L->last_iters = iters;
            L->t += iters;
            L->vupd += n * iters;
            L->pairs += n * (n - 1.0) * iters;
        }
    }
    if (s == BL_OK) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (elapsed_ms) *elapsed_ms = ms;
        for (int k = 0; k < count; k++) Ls[k]->last_ms = ms;
    }
    return s;
}

}  // namespace bl

using namespace bl;

static int env_chunk() {
    const char* c = std::getenv("BL_BATCH_CHUNK");
    return c ? std::atoi(c) : 0;
}

extern "C" bl_status bl_layout_run_batch(bl_layout* const* Ls, int32_t count, int32_t iters, int32_t batch) {
    if (count < 0 || iters < 0) return set_error(BL_EINVAL, "bl_layout_run_batch: negative count");
    if (count > 0 && !Ls) return set_error(BL_EINVAL, "bl_layout_run_batch: NULL layout array");
    if (batch < 1 || batch > kMaxBatch)
        return set_error(BL_EINVAL, "bl_layout_run_batch: batch must be in [1, 8192]");
    for (int k = 0; k < count; k++)
        if (!Ls[k]) return set_error(BL_EINVAL, "bl_layout_run_batch: NULL layout");
    return batch_run(Ls, count, iters, batch, env_chunk(), current_stream(), nullptr);
}

extern "C" bl_status bl_layout_batch(const bl_graph* const* gs, int32_t count, const uint64_t* seeds,
                                     int32_t iters, int32_t batch, bl_mode mode, float theta,
                                     bl_layout** outs) {
    if (count < 0 || iters < 0) return set_error(BL_EINVAL, "bl_layout_batch: negative count");
    if (count > 0 && (!gs || !seeds || !outs)) return set_error(BL_EINVAL, "bl_layout_batch: NULL argument");
    if (batch < 1 || batch > kMaxBatch) return set_error(BL_EINVAL, "bl_layout_batch: batch must be in [1, 8192]");
    if (mode != BL_EXACT && mode != BL_BH)
        return set_error(BL_EINVAL, "bl_layout_batch: mode must be BL_EXACT or BL_BH");
    if (mode == BL_BH && !(theta >= 0.0f)) return set_error(BL_EINVAL, "bl_layout_batch: theta must be >= 0");
    for (int k = 0; k < count; k++) {
        outs[k] = nullptr;
        if (!gs[k]) return set_error(BL_EINVAL, "bl_layout_batch: NULL graph");
    }
    // seeded positions of every graph, uploaded without a wait per layout
    size_t total = 0;
    for (int k = 0; k < count; k++) total += 2 * (size_t)gs[k]->n;
    std::vector<float> xy(total);
    bl_status s = BL_OK;
    size_t off = 0;
    for (int k = 0; k < count && s == BL_OK; k++) {
        seeded_positions(gs[k]->n, seeds[k], xy.data() + off);
        s = layout_create(gs[k], xy.data() + off, seeds[k], 0, nullptr, false, current_stream(), &outs[k]);
        off += 2 * (size_t)gs[k]->n;
    }
    if (s == BL_OK) {
        const cudaError_t e = cudaStreamSynchronize(current_stream());
        if (e != cudaSuccess) s = cuda_error(e, "bl_layout_batch: upload");
    }
    if (s == BL_OK && iters > 0) {
        if (mode == BL_EXACT) {
            s = batch_run(outs, count, iters, batch, env_chunk(), current_stream(), nullptr);
        } else {
            for (int k = 0; k < count && s == BL_OK; k++) s = bl_layout_run(outs[k], iters, batch, BL_BH, theta);
        }
    }
    if (s != BL_OK) {
        const std::string msg = bl_last_error();
        for (int k = 0; k < count; k++) {
            bl_layout_free(outs[k]);
            outs[k] = nullptr;
        }
        return set_error(s, msg);
    }
    return BL_OK;
}
