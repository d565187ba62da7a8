// Quality metrics of a layout (Section 3.7): stress minimised over a uniform
// scale, 1-hop neighbourhood preservation and edge uniformity, all accumulated in
// FP64 on the GPU.
//
// Stress needs the hop distance of every (source, vertex) pair. The BFS runs 64
// sources at a time as the bits of one uint64 per vertex: a level pulls the
// frontier words of a vertex's neighbours, keeps the bits not yet visited, and
// each new bit is one pair at hop distance = level. A cooperative kernel walks
// the levels with a grid barrier between them.
//
// Neighbourhood preservation needs, per query i, the deg(i) layout-nearest
// vertices (squared FP64 distance, ties by id). One CTA per query radix-selects
// the deg(i)-th smallest 64-bit key (the bits of the non-negative double d^2):
// a histogram of the top 12 bits over all n candidates, a compaction of the
// selected bin into per-CTA scratch, then 12-bit digits over that list.
// Squared distances use the plain operation order dx*dx + dy*dy with each product
// and the sum rounded once, so the keys and therefore the counts are exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bl_internal.cuh"

namespace bl {
namespace {

constexpr int kQThreads = 256;
constexpr int kSrcBatch = 64;

// SplitMix64 output k of the stream whose state starts at `seed`.
inline uint64_t q_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// m distinct vertices: the first m entries of a partial Fisher-Yates shuffle of
// 0..n-1 whose step k swaps entry k with entry k + (z_k mod (n-k)).
std::vector<int> seeded_sample(int n, int m, uint64_t seed) {
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) idx[i] = i;
    for (int k = 0; k < m; k++) {
        const uint64_t r = q_splitmix64(seed, (uint64_t)k);
        const int j = k + (int)(r % (uint64_t)(n - k));
        std::swap(idx[k], idx[j]);
    }
    idx.resize(m);
    return idx;
}

__device__ __forceinline__ double pair_d2(float2 a, double xi, double yi) {
    const double dx = __dsub_rn((double)a.x, xi);
    const double dy = __dsub_rn((double)a.y, yi);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

template <class T>
__device__ T block_sum(T v, T* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) r += sh[k];
    return r;   // valid in thread 0
}

// ---------------------------------------------------------------------------
// stress: one cooperative launch per batch of up to 64 sources
// ---------------------------------------------------------------------------

struct StressArgs {
    const int* rowptr;
    const int* colids;
    const float2* pos;
    int n;
    const int* src;          // sources of this batch
    int nb;                  // sources in this batch (<= 64)
    int full;                // all-pairs mode: count only vertices above the source id
    unsigned long long* vis;
    unsigned long long* fa;
    unsigned long long* fb;
    unsigned* cnt;           // 3 rotating "something new" counters
    double* part_a;          // [G] sum x/d
    double* part_b;          // [G] sum (x/d)^2
    unsigned long long* part_p;   // [G] pairs
    unsigned* bar;
    int* status;
};

__global__ void __launch_bounds__(kQThreads) stress_bfs_kernel(StressArgs a) {
    __shared__ float2 s_pos[kSrcBatch];
    __shared__ int s_src[kSrcBatch];
    __shared__ double s_red[kQThreads / 32];
    __shared__ unsigned long long s_redp[kQThreads / 32];
    GridBarrier gb{a.bar, a.status, gridDim.x, 0};
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned long long allm = a.nb == 64 ? ~0ull : ((1ull << a.nb) - 1ull);
    if (threadIdx.x < a.nb) {
        s_src[threadIdx.x] = a.src[threadIdx.x];
        s_pos[threadIdx.x] = a.pos[a.src[threadIdx.x]];
    }
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        a.vis[v] = 0ull;
        a.fa[v] = 0ull;
    }
    if (!gb.sync()) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k < a.nb; k++) {
            a.vis[s_src[k]] = 1ull << k;
            a.fa[s_src[k]] = 1ull << k;
        }
        a.cnt[0] = a.cnt[1] = a.cnt[2] = 0u;
    }
    if (!gb.sync()) return;
    double acc_a = 0.0, acc_b = 0.0;
    unsigned long long acc_p = 0ull;
    unsigned long long* fcur = a.fa;
    unsigned long long* fnext = a.fb;
    for (int level = 1;; level++) {
        const double inv = 1.0 / (double)level;
        int fresh = 0;
        for (int v = gwarp; v < a.n; v += nwarps) {
            const unsigned long long mv = a.vis[v];
            unsigned long long nw = 0ull;
            if (mv != allm) {
                unsigned long long acc = 0ull;
                const int e1 = a.rowptr[v + 1];
                for (int e = a.rowptr[v] + lane; e < e1; e += 32) acc |= fcur[a.colids[e]];
                const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)acc);
                const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(acc >> 32));
                nw = (((unsigned long long)hi << 32) | lo) & ~mv & allm;
            }
            if (lane == 0) {
                fnext[v] = nw;
                if (nw) a.vis[v] = mv | nw;
            }
            if (nw) {
                fresh = 1;
                const float2 pv = a.pos[v];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int k = lane + 32 * h;
                    if (((nw >> k) & 1ull) && (!a.full || v > s_src[k])) {
                        const double dx = (double)pv.x - (double)s_pos[k].x;
                        const double dy = (double)pv.y - (double)s_pos[k].y;
                        const double q = sqrt(dx * dx + dy * dy) * inv;
                        acc_a += q;
                        acc_b += q * q;
                        acc_p += 1ull;
                    }
                }
            }
        }
        const int any = __syncthreads_or(fresh);
        if (threadIdx.x == 0) {
            if (any) atomicAdd(&a.cnt[level % 3], 1u);
            if (blockIdx.x == 0) a.cnt[(level + 1) % 3] = 0u;
        }
        if (!gb.sync()) return;
        if (*(volatile unsigned*)&a.cnt[level % 3] == 0u) break;
        unsigned long long* t = fcur;
        fcur = fnext;
        fnext = t;
    }
    const double sa = block_sum(acc_a, s_red);
    if (threadIdx.x == 0) a.part_a[blockIdx.x] = sa;
    const double sb = block_sum(acc_b, s_red);
    if (threadIdx.x == 0) a.part_b[blockIdx.x] = sb;
    const unsigned long long sp = block_sum(acc_p, s_redp);
    if (threadIdx.x == 0) a.part_p[blockIdx.x] = sp;
}

// ---------------------------------------------------------------------------
// neighbourhood preservation: one CTA per query (grid-stride over queries)
// ---------------------------------------------------------------------------

constexpr int kTopBins = 4096;   // top 12 bits of the key
constexpr int kDigitBits = 12;

struct NPArgs {
    const int* rowptr;
    const int* colids;
    const float2* pos;
    int n;
    const int* queries;      // [nq] or null = vertex q
    int nq;
    unsigned long long* lkey;   // [G][n] compacted keys
    int* lid;                   // [G][n] their ids
    double* jac;                // [nq] Jaccard of query q (0 when deg = 0)
    int* inter;                 // [nq] intersection size (-1 when deg = 0)
};

// Finds the bin holding the element of 1-based rank `need` in hist[0..nb) and
// leaves it in s_sel[0] with the rank inside the bin in s_sel[1] and the bin's
// count in s_sel[2]. Whole block; hist must be complete.
__device__ void select_bin(const unsigned* hist, int nb, int need, int* s_sel, unsigned* s_scan) {
    // per-thread chunk sums, then a serial scan by thread 0 (nb / blockDim small)
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    unsigned s = 0;
    for (int b = b0; b < min(nb, b0 + per); b++) s += hist[b];
    s_scan[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned c = 0;
        int t = 0;
        for (; t < (int)blockDim.x; t++) {
            if (c + s_scan[t] >= (unsigned)need) break;
            c += s_scan[t];
        }
        int b = min(t * per, nb - 1);
        for (; b < nb - 1; b++) {   // the counts always reach `need` by the last bin
            if (c + hist[b] >= (unsigned)need) break;
            c += hist[b];
        }
        s_sel[0] = b;
        s_sel[1] = need - (int)c;
        s_sel[2] = (int)hist[b];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kQThreads) np_kernel(NPArgs a) {
    __shared__ unsigned s_hist[kTopBins];
    __shared__ unsigned s_scan[kQThreads];
    __shared__ int s_sel[3];
    __shared__ int s_len;
    __shared__ int s_red[kQThreads / 32];
    unsigned long long* lkey = a.lkey + (size_t)blockIdx.x * a.n;
    int* lid = a.lid + (size_t)blockIdx.x * a.n;
    for (int q = blockIdx.x; q < a.nq; q += gridDim.x) {
        const int i = a.queries ? a.queries[q] : q;
        const int r0 = a.rowptr[i], r1 = a.rowptr[i + 1];
        const int k = r1 - r0;
        if (k == 0) {
            if (threadIdx.x == 0) {
                a.jac[q] = 0.0;
                a.inter[q] = -1;
            }
            continue;
        }
        const float2 pi = a.pos[i];
        const double xi = (double)pi.x, yi = (double)pi.y;
        // top 12 bits over all candidates j != i
        for (int b = threadIdx.x; b < kTopBins; b += blockDim.x) s_hist[b] = 0u;
        if (threadIdx.x == 0) s_len = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < a.n; j += blockDim.x) {
            if (j == i) continue;
            const unsigned long long key = (unsigned long long)__double_as_longlong(pair_d2(a.pos[j], xi, yi));
            atomicAdd(&s_hist[key >> 52], 1u);
        }
        __syncthreads();
        select_bin(s_hist, kTopBins, k, s_sel, s_scan);
        unsigned long long prefix = (unsigned long long)s_sel[0] << 52;
        int need = s_sel[1];
        unsigned long long pmask = 0xFFFull << 52;
        // compact the selected bin
        for (int j = threadIdx.x; j < a.n; j += blockDim.x) {
            if (j == i) continue;
            const unsigned long long key = (unsigned long long)__double_as_longlong(pair_d2(a.pos[j], xi, yi));
            if ((key & pmask) == prefix) {
                const int at = atomicAdd(&s_len, 1);
                lkey[at] = key;
                lid[at] = j;
            }
        }
        __syncthreads();
        const int len = s_len;
        // remaining 52 bits: digits at 40, 28, 16, 4 (12 bits) and 0 (4 bits)
        for (int shift = 52 - kDigitBits;; shift -= kDigitBits) {
            const int sh = shift < 0 ? 0 : shift;
            const int width = shift < 0 ? kDigitBits + shift : kDigitBits;
            const int nb = 1 << width;
            for (int b = threadIdx.x; b < nb; b += blockDim.x) s_hist[b] = 0u;
            __syncthreads();
            for (int t = threadIdx.x; t < len; t += blockDim.x) {
                const unsigned long long key = lkey[t];
                if ((key & pmask) == prefix) atomicAdd(&s_hist[(key >> sh) & (unsigned long long)(nb - 1)], 1u);
            }
            __syncthreads();
            select_bin(s_hist, nb, need, s_sel, s_scan);
            prefix |= (unsigned long long)s_sel[0] << sh;
            pmask |= (unsigned long long)(nb - 1) << sh;
            need = s_sel[1];
            if (sh == 0) break;
        }
        const unsigned long long T = prefix;   // key of the k-th nearest
        const int ties = s_sel[2];             // candidates with key == T
        // need = how many of the tied candidates (smallest ids first) are in L_i
        int mine = 0;
        for (int e = r0 + threadIdx.x; e < r1; e += blockDim.x) {
            const int j = a.colids[e];
            const unsigned long long key = (unsigned long long)__double_as_longlong(pair_d2(a.pos[j], xi, yi));
            int in = key < T;
            if (key == T) {
                if (ties == 1) {
                    in = 1;
                } else {
                    int below = 0;
                    for (int t = 0; t < len; t++) below += (lkey[t] == T && lid[t] < j);
                    in = below < need;
                }
            }
            mine += in;
        }
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += s_red[w];
            const int m = a.n - 1;
            const int uni = k + (k < m ? k : m) - tot;
            a.jac[q] = (double)tot / (double)uni;
            a.inter[q] = tot;
        }
        __syncthreads();
    }
}

// sums in query order, as a single thread: NP, queries used, intersections
__global__ void np_final_kernel(const double* jac, const int* inter, int nq, double* out3) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc = 0.0, it = 0.0;
    long long used = 0;
    for (int q = 0; q < nq; q++) {
        if (inter[q] < 0) continue;
        acc += jac[q];
        it += (double)inter[q];
        used++;
    }
    out3[0] = used ? acc / (double)used : 0.0;
    out3[1] = (double)used;
    out3[2] = it;
}

// ---------------------------------------------------------------------------
// edge uniformity: mean edge length, then the spread about it
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kQThreads) eu_kernel(const int* rowptr, const int* colids,
                                                       const float2* pos, int n, const double* mu,
                                                       double* part_s, unsigned long long* part_m) {
    __shared__ double s_red[kQThreads / 32];
    __shared__ unsigned long long s_redm[kQThreads / 32];
    double s = 0.0;
    unsigned long long m = 0;
    const double c = mu ? *mu : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 pi = pos[i];
        for (int e = rowptr[i]; e < rowptr[i + 1]; e++) {
            const int j = colids[e];
            if (j <= i) continue;
            const float2 pj = pos[j];
            const double dx = (double)pj.x - (double)pi.x;
            const double dy = (double)pj.y - (double)pi.y;
            const double l = sqrt(dx * dx + dy * dy);
            if (mu) s += (l - c) * (l - c);
            else s += l;
            m++;
        }
    }
    const double bs = block_sum(s, s_red);
    const unsigned long long bm = block_sum(m, s_redm);
    if (threadIdx.x == 0) {
        part_s[blockIdx.x] = bs;
        part_m[blockIdx.x] = bm;
    }
}

__global__ void eu_mean_kernel(const double* part_s, const unsigned long long* part_m, int G, double* mu,
                               double* eu) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    unsigned long long m = 0;
    for (int g = 0; g < G; g++) {
        s += part_s[g];
        m += part_m[g];
    }
    if (eu == nullptr) {
        *mu = m ? s / (double)m : 0.0;
    } else {
        const double c = *mu;
        *eu = m == 0 ? 0.0 : sqrt(s / ((double)m * c * c));
    }
}

// Scratch of one bl_quality call, released when it goes out of scope, on every
// return path, once the stream has drained (a caller's allocator may hand the
// memory out again at once).
struct QScratch {
    cudaStream_t st;
    DevBuf vis, fa, fb, cnt, bar, pa, pb, pp, src, lkey, lid, jac, inter, queries, eu;
    explicit QScratch(cudaStream_t s) : st(s) {}
    ~QScratch() {
        cudaStreamSynchronize(st);
        for (DevBuf* b : {&vis, &fa, &fb, &cnt, &bar, &pa, &pb, &pp, &src, &lkey, &lid, &jac, &inter,
                          &queries, &eu})
            b->release();
    }
};

}  // namespace

bl_status quality_run(bl_layout* L, int32_t nsources, int32_t nqueries, uint64_t seed, double* out,
                      int64_t cap, cudaStream_t st) {
    const int n = L->g->n;
    for (int k = 0; k < std::min<int64_t>(cap, 7); k++) out[k] = 0.0;
    if (n == 0) return BL_OK;
    const int* rowptr = L->g->rowptr.as<int>();
    const int* colids = L->g->colids.as<int>();
    const float2* pos = L->pos.as<float2>();
    const Allocator& al = L->alloc;
    QScratch s(st);
    const int sms = device_sm_count();

    // ---- stress ----
    const bool full = nsources <= 0 || nsources >= n;
    std::vector<int> srcs;
    if (full) {
        srcs.resize(n);
        for (int i = 0; i < n; i++) srcs[i] = i;
    } else {
        srcs = seeded_sample(n, nsources, seed);
    }
    const int ns = (int)srcs.size();
    int occ = 0;
    BL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stress_bfs_kernel, kQThreads, 0));
    const int G = std::max(1, std::min(occ, 4)) * sms;
    const int nbatches = div_up(ns, kSrcBatch);
    BL_TRY(s.vis.ensure(al, (size_t)n * 8));
    BL_TRY(s.fa.ensure(al, (size_t)n * 8));
    BL_TRY(s.fb.ensure(al, (size_t)n * 8));
    BL_TRY(s.cnt.ensure(al, 3 * sizeof(unsigned)));
    BL_TRY(s.bar.ensure(al, 256));
    BL_TRY(s.pa.ensure(al, (size_t)nbatches * G * sizeof(double)));
    BL_TRY(s.pb.ensure(al, (size_t)nbatches * G * sizeof(double)));
    BL_TRY(s.pp.ensure(al, (size_t)nbatches * G * sizeof(unsigned long long)));
    BL_TRY(s.src.ensure(al, (size_t)ns * sizeof(int)));
    BL_CUDA_TRY(cudaMemcpyAsync(s.src.p, srcs.data(), (size_t)ns * sizeof(int), cudaMemcpyHostToDevice, st));
    int* status = static_cast<int*>(L->status.p);
    for (int bt = 0; bt < nbatches; bt++) {
        StressArgs a{};
        a.rowptr = rowptr;
        a.colids = colids;
        a.pos = pos;
        a.n = n;
        a.src = s.src.as<int>() + (size_t)bt * kSrcBatch;
        a.nb = std::min(kSrcBatch, ns - bt * kSrcBatch);
        a.full = full ? 1 : 0;
        a.vis = s.vis.as<unsigned long long>();
        a.fa = s.fa.as<unsigned long long>();
        a.fb = s.fb.as<unsigned long long>();
        a.cnt = s.cnt.as<unsigned>();
        a.part_a = s.pa.as<double>() + (size_t)bt * G;
        a.part_b = s.pb.as<double>() + (size_t)bt * G;
        a.part_p = s.pp.as<unsigned long long>() + (size_t)bt * G;
        a.bar = s.bar.as<unsigned>();
        a.status = status;
        BL_CUDA_TRY(cudaMemsetAsync(s.bar.p, 0, 256, st));
        void* args[] = {&a};
        BL_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)stress_bfs_kernel, dim3(G), dim3(kQThreads),
                                                args, 0, st));
    }

    // ---- neighbourhood preservation ----
    const bool allq = nqueries <= 0 || nqueries >= n;
    const int nq = allq ? n : nqueries;
    if (!allq) {
        std::vector<int> qs = seeded_sample(n, nqueries, seed ^ 0x5bd1e995ull);
        BL_TRY(s.queries.ensure(al, (size_t)nq * sizeof(int)));
        BL_CUDA_TRY(cudaMemcpyAsync(s.queries.p, qs.data(), (size_t)nq * sizeof(int), cudaMemcpyHostToDevice,
                                    st));
    }
    const int Gq = std::max(1, std::min(nq, sms));
    BL_TRY(s.lkey.ensure(al, (size_t)Gq * n * sizeof(unsigned long long)));
    BL_TRY(s.lid.ensure(al, (size_t)Gq * n * sizeof(int)));
    BL_TRY(s.jac.ensure(al, (size_t)nq * sizeof(double)));
    BL_TRY(s.inter.ensure(al, (size_t)nq * sizeof(int)));
    BL_TRY(s.eu.ensure(al, 8 * sizeof(double)));
    NPArgs na{rowptr, colids, pos, n, allq ? nullptr : s.queries.as<int>(), nq,
              s.lkey.as<unsigned long long>(), s.lid.as<int>(), s.jac.as<double>(), s.inter.as<int>()};
    np_kernel<<<Gq, kQThreads, 0, st>>>(na);
    double* dres = s.eu.as<double>();   // [0] mu, [1] eu, [2..4] NP, used, intersections
    np_final_kernel<<<1, 32, 0, st>>>(s.jac.as<double>(), s.inter.as<int>(), nq, dres + 2);
    BL_CUDA_TRY(cudaGetLastError());

    // ---- edge uniformity ----
    const int Ge = std::max(1, std::min(div_up(n, kQThreads), 4 * sms));
    double* ps = s.pa.as<double>();                     // reuse: stress partials are read below,
    unsigned long long* pm = s.pp.as<unsigned long long>();   // so copy them out first
    std::vector<double> ha((size_t)nbatches * G), hb((size_t)nbatches * G);
    std::vector<unsigned long long> hp((size_t)nbatches * G);
    BL_CUDA_TRY(cudaMemcpyAsync(ha.data(), s.pa.p, ha.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaMemcpyAsync(hb.data(), s.pb.p, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaMemcpyAsync(hp.data(), s.pp.p, hp.size() * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    if (Ge > nbatches * G) {
        BL_TRY(s.pa.ensure(al, (size_t)Ge * sizeof(double)));
        BL_TRY(s.pp.ensure(al, (size_t)Ge * sizeof(unsigned long long)));
        ps = s.pa.as<double>();
        pm = s.pp.as<unsigned long long>();
    }
    eu_kernel<<<Ge, kQThreads, 0, st>>>(rowptr, colids, pos, n, nullptr, ps, pm);
    eu_mean_kernel<<<1, 32, 0, st>>>(ps, pm, Ge, dres + 0, nullptr);
    eu_kernel<<<Ge, kQThreads, 0, st>>>(rowptr, colids, pos, n, dres + 0, ps, pm);
    eu_mean_kernel<<<1, 32, 0, st>>>(ps, pm, Ge, dres + 0, dres + 1);
    BL_CUDA_TRY(cudaGetLastError());
    double hres[5];
    BL_CUDA_TRY(cudaMemcpyAsync(hres, dres, sizeof(hres), cudaMemcpyDeviceToHost, st));
    int dstat = 0;
    BL_CUDA_TRY(cudaMemcpyAsync(&dstat, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    if (dstat != 0) {
        cudaMemset(status, 0, sizeof(int));
        return set_error((bl_status)dstat, "bl_quality: a bounded device-side wait timed out");
    }
    // stress = pairs - a^2/b at the optimal scale s* = a/b
    double A = 0.0, B = 0.0, P = 0.0;
    for (size_t k = 0; k < ha.size(); k++) {
        A += ha[k];
        B += hb[k];
        P += (double)hp[k];
    }
    double stress = P - (B > 0.0 ? A * A / B : 0.0);
    if (!full) stress *= (double)n / (double)ns / 2.0;
    out[0] = stress;
    out[1] = B > 0.0 ? A / B : 0.0;
    out[2] = P;
    out[3] = hres[2];
    out[4] = hres[3];
    out[5] = hres[1];
    if (cap >= 7) out[6] = hres[4];
    return BL_OK;
}

}  // namespace bl
