// Barnes-Hut BatchLayout (Section 3.5; Algorithms S3, S4, S5).
//
// One iteration, on the snapshot S of the positions at iteration start
// (Algorithm S5 builds the tree before its minibatch loop):
//   1. bounding box -> root square (side D = max extent, anchored at the minimum);
//   2. Morton codes: each coordinate quantised to 16 bits in FP32 with a fixed op
//      order, bits interleaved (x in even bits, y in odd bits);
//   3. stable LSD radix sort of (code, vertex id), 4 passes of 8 bits;
//   4. quadtree in pre-order, built bottom-up from the sorted codes: a node is a
//      non-empty cell whose parent holds >= 2 vertices; it is a leaf when it holds
//      one vertex or sits at level 16. Sorted position k starts the cells of the
//      levels between the first level where its code differs from code[k-1] and
//      the first level where it differs from code[k+1]; an exclusive scan of those
//      counts gives every node its pre-order index, and a binary search gives each
//      cell's end and the index just past its subtree (skip);
//   5. node coordinate sums in FP32, level by level from the leaves: a leaf adds
//      its vertices in sorted order, an inner node adds its children in order;
//      centroid = sum / count;
//   6. theta-walk per vertex (S4): stackless pre-order traversal with skip links; a
//      node is accepted when (D/2^level)^2 < theta^2 * |g - c_i|^2 (FP32) and then
//      acts with its vertex count at its centroid; leaves add their vertices
//      directly (vertex i itself skipped by index). The 32 lanes of a warp walk 32
//      Morton-adjacent vertices and advance together to the smallest node any of
//      them still has to visit, so each node record is read once per warp;
//   7. neighbour correction: unless repulse_neighbors, the exact repulsion of each
//      vertex's CSR neighbours (at S) is taken back out;
//   8. minibatch sweep: batches in vertex-id order; the rows of batch b add the CSR
//      attraction at the live positions (earlier batches already moved this
//      iteration) to their repulsion and move by Step * ct/|ct|. Batch b depends
//      only on the earlier batches its rows have edges into: a persistent kernel
//      processes batches as their predecessors' flags appear.
// Positions are double-buffered: the sweep reads S (not yet moved vertices) from
// the old buffer and writes the new buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <vector>

#include "bl_internal.cuh"

namespace bl {

constexpr int kLevels = 16;
constexpr int kScanItems = 1024;     // elements per block of the scan
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;       // elements per thread of a sort tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSweepThreads = 256;

struct BHState {
    int n = 0;
    int64_t cap_nodes = 0;
    DevBuf keys0, keys1, vals0, vals1;   // sort ping-pong
    DevBuf hist, scan_part;             // radix digit counts, scan block sums
    DevBuf bpart, box;                  // bbox partials; box = {xmin, ymin, D, s, Dl2[17]}
    DevBuf cnt;                         // int[n+1]: nodes per sorted position -> first node
    DevBuf spos;                        // float2[n]: positions in sorted order
    DevBuf nd_first, nd_count, nd_level, nd_skip;
    DevBuf nd_sum;                      // float2 sums
    DevBuf nd_rec;                      // float4 {gx, gy, Dl^2, count}
    DevBuf nd_aux;                      // int2 {skip, leaf ? first : -1}
    DevBuf lvl;                         // int[64]: per-level counts, offsets, fill
    DevBuf lvl_info;                    // nodes bucketed by level: int4 {node, first, count, skip}
    DevBuf rep;                         // float2[n]: repulsion sums (unscaled)
    DevBuf walkcnt;                     // unsigned long long[3]: far nodes, near pairs, node visits
    // sweep
    int plan_bs = -1, plan_seg = 0, nlevels = 0, nbig = 0, nmid = 0, lvl0_rows = 0;
    int64_t ntasks = 0;
    int nsegsum = 0;                    // segment slots of the rows of several segments
    DevBuf split, bigrows, midrows, old;   // row split points, long and medium rows, old attraction
    DevBuf corr;                        // float2[n]: exact repulsion of the CSR neighbours at S
    DevBuf lvl_ptr, tasks, seg_off, seg_sum;   // level-set schedule; segment partial sums
    DevBuf scol;                        // earlier-minibatch columns of the rows of several segments
    DevBuf e_row, epart;                // per-row |ct|^2, reduction partials
    // the edge pass runs on a side stream while the tree is built and walked
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the iteration's critical path runs on a highest-priority stream forked from and
    // joined back to the caller's, so the edge pass (default priority) does not
    // hold SMs the tree build and sweep are waiting for
    cudaStream_t hi = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

void bh_state_free(BHState* s) {
    if (!s) return;
    DevBuf* bufs[] = {&s->keys0, &s->keys1, &s->vals0, &s->vals1, &s->hist, &s->scan_part,
                      &s->bpart, &s->box, &s->cnt, &s->spos, &s->nd_first, &s->nd_count,
                      &s->nd_level, &s->nd_skip, &s->nd_sum, &s->nd_rec, &s->nd_aux, &s->lvl,
                      &s->lvl_info, &s->rep, &s->walkcnt, &s->split, &s->bigrows, &s->midrows, &s->old,
                      &s->corr,
                      &s->lvl_ptr, &s->tasks, &s->seg_off, &s->seg_sum, &s->scol, &s->e_row,
                      &s->epart};
    for (DevBuf* b : bufs) b->release();
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    if (s->hi) cudaStreamDestroy(s->hi);
    delete s;
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (device-wide, three kernels)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int block_exclusive_scan_256(int v, int* s_warp, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < 8 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < 8) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[7];
    const int before = warp > 0 ? s_warp[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void scan_sums_kernel(const int* __restrict__ in, int n, int* __restrict__ part) {
    __shared__ int s_warp[8];
    const int base = blockIdx.x * kScanItems;
    int v = 0;
    for (int q = 0; q < 4; q++) {
        const int idx = base + threadIdx.x * 4 + q;
        v += idx < n ? in[idx] : 0;
    }
    int total;
    block_exclusive_scan_256(v, s_warp, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void scan_top_kernel(int* __restrict__ part, int nb) {
    // single block of 256 threads: exclusive scan over nb block sums, in place
    __shared__ int s_warp[8];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 256) {
        const int idx = base + threadIdx.x;
        const int v = idx < nb ? part[idx] : 0;
        int total;
        const int ex = block_exclusive_scan_256(v, s_warp, total);
        if (idx < nb) part[idx] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
}

__global__ void scan_apply_kernel(const int* in, int n, const int* __restrict__ part, int* out) {
    __shared__ int s_warp[8];
    const int base = blockIdx.x * kScanItems;
    int v[4];
    int sum = 0;
    for (int q = 0; q < 4; q++) {
        const int idx = base + threadIdx.x * 4 + q;
        v[q] = idx < n ? in[idx] : 0;
        sum += v[q];
    }
    int total;
    int run = block_exclusive_scan_256(sum, s_warp, total) + part[blockIdx.x];
    for (int q = 0; q < 4; q++) {
        const int idx = base + threadIdx.x * 4 + q;
        if (idx < n) out[idx] = run;
        run += v[q];
    }
}

// exclusive scan in -> out (may alias); part holds ceil(n/1024) ints
static bl_status exclusive_scan(const int* in, int* out, int n, int* part, cudaStream_t st) {
    const int nb = div_up(n, kScanItems);
    scan_sums_kernel<<<nb, 256, 0, st>>>(in, n, part);
    scan_top_kernel<<<1, 256, 0, st>>>(part, nb);
    scan_apply_kernel<<<nb, 256, 0, st>>>(in, n, part, out);
    BL_CUDA_TRY(cudaGetLastError());
    return BL_OK;
}

// ---------------------------------------------------------------------------
// bounding box and Morton codes (reading R8, R9)
// ---------------------------------------------------------------------------

__global__ void bbox_partial_kernel(const float2* __restrict__ pos, int n, float4* __restrict__ part) {
    float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 p = pos[i];
        xmin = fminf(xmin, p.x);
        xmax = fmaxf(xmax, p.x);
        ymin = fminf(ymin, p.y);
        ymax = fmaxf(ymax, p.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
        xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
        ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    }
    __shared__ float4 s_w[32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = make_float4(xmin, xmax, ymin, ymax);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 r = s_w[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            r.x = fminf(r.x, s_w[w].x);
            r.y = fmaxf(r.y, s_w[w].y);
            r.z = fminf(r.z, s_w[w].z);
            r.w = fmaxf(r.w, s_w[w].w);
        }
        part[blockIdx.x] = r;
    }
}

// box[0] = xmin, box[1] = ymin, box[2] = D, box[3] = 65536/D (0 when the box is
// degenerate: every code is then 0), box[4 + l] = (D * 2^-l)^2 for l = 0..16
__global__ void bbox_final_kernel(const float4* __restrict__ part, int nb, float* __restrict__ box) {
    // one warp: min and max are exact, so the order of the reduction is free
    const int lane = threadIdx.x;
    float4 r = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    for (int b = lane; b < nb; b += 32) {
        const float4 p = part[b];
        r.x = fminf(r.x, p.x);
        r.y = fmaxf(r.y, p.y);
        r.z = fminf(r.z, p.z);
        r.w = fmaxf(r.w, p.w);
    }
    for (int o = 16; o > 0; o >>= 1) {
        r.x = fminf(r.x, __shfl_xor_sync(0xffffffffu, r.x, o));
        r.y = fmaxf(r.y, __shfl_xor_sync(0xffffffffu, r.y, o));
        r.z = fminf(r.z, __shfl_xor_sync(0xffffffffu, r.z, o));
        r.w = fmaxf(r.w, __shfl_xor_sync(0xffffffffu, r.w, o));
    }
    if (lane != 0) return;
    const float dxr = __fsub_rn(r.y, r.x), dyr = __fsub_rn(r.w, r.z);
    const float D = dxr > dyr ? dxr : dyr;
    box[0] = r.x;
    box[1] = r.z;
    box[2] = D;
    box[3] = (D > 0.f && isfinite(D)) ? __fdiv_rn(65536.0f, D) : 0.f;
    for (int l = 0; l <= kLevels; l++) {
        const float Dl = ldexpf(D, -l);
        box[4 + l] = __fmul_rn(Dl, Dl);
    }
}

// spread the 16 bits of v to the even bit positions
__device__ __forceinline__ unsigned spread_bits(unsigned v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void morton_kernel(const float2* __restrict__ pos, int n, const float* __restrict__ box,
                              unsigned* __restrict__ keys, int* __restrict__ vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = box[3];
    unsigned code = 0u;
    if (s > 0.f) {
        const float2 p = pos[i];
        const float tx = __fmul_rn(__fsub_rn(p.x, box[0]), s);
        const float ty = __fmul_rn(__fsub_rn(p.y, box[1]), s);
        unsigned qx = (unsigned)floorf(tx), qy = (unsigned)floorf(ty);
        qx = min(qx, 65535u);
        qy = min(qy, 65535u);
        code = spread_bits(qx) | (spread_bits(qy) << 1);
    }
    keys[i] = code;
    vals[i] = i;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (u32 key, i32 value): 4 passes of 8 bits, one kernel
// per pass. One histogram kernel counts every digit of every pass (the counts do
// not depend on the order); a pass kernel takes tiles in ticket order, ranks each
// tile's keys by digit in index order (stable), and gets, for every digit, the
// count of that digit in all earlier tiles by decoupled look-back: each tile
// publishes its digit counts (flag "aggregate"), then walks back over the earlier
// tiles' published words, adding aggregates until it meets an inclusive prefix,
// and publishes its own inclusive prefix (Merrill and Garland's single-pass
// prefix scan, as used for radix sorting by Adinets and Merrill's Onesweep).
// ---------------------------------------------------------------------------

constexpr unsigned kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kCountMask = (1u << 30) - 1;

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// counts of every digit of every pass into hist[p * 256 + d] (zeroed before)
__global__ void radix_hist4_kernel(const unsigned* __restrict__ keys, int n, unsigned* __restrict__ hist) {
    __shared__ unsigned s_h[4 * 256];
    for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x) s_h[q] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned k = keys[i];
#pragma unroll
        for (int p = 0; p < 4; p++) atomicAdd(&s_h[p * 256 + ((k >> (8 * p)) & 255u)], 1u);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x)
        if (s_h[q]) atomicAdd(&hist[q], s_h[q]);
}

// digit counts -> exclusive digit bases, per pass (one block of 256 threads)
__global__ void radix_bases_kernel(unsigned* hist) {
    __shared__ int s_warp[8];
    for (int p = 0; p < 4; p++) {
        int total;
        const int ex = block_exclusive_scan_256((int)hist[p * 256 + threadIdx.x], s_warp, total);
        hist[p * 256 + threadIdx.x] = (unsigned)ex;
        __syncthreads();
    }
}

// One pass on digit (key >> shift) & 255. base: the pass's exclusive digit bases;
// status: [tiles][256] words of this pass and tile_ctr, all zero at launch. pass 0
// takes its values as the keys' indices (ident). A look-back wait that gives up
// sets *err to BL_ETIMEOUT (the tile's output is then garbage; the host reports it).
__global__ void __launch_bounds__(kSortThreads) radix_pass_kernel(
    const unsigned* __restrict__ kin, const int* __restrict__ vin, int n, int shift,
    const unsigned* __restrict__ base, unsigned* __restrict__ status, unsigned* __restrict__ tile_ctr,
    int ident, int* __restrict__ err, unsigned* __restrict__ kout, int* __restrict__ vout) {
    constexpr int W = kSortThreads / 32;
    __shared__ unsigned s_whist[W][256];   // digit counts per warp, then their exclusive prefix
    __shared__ unsigned s_dst[256];        // where this tile's keys of each digit start
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);   // tickets in order: the look-back
#pragma unroll                                                       // only waits on tiles already taken
    for (int w = 0; w < W; w++) s_whist[w][threadIdx.x] = 0u;
    __syncthreads();
    const int tile = s_tile;
    // the warp's keys: rows of 32 consecutive keys, rows in order
    const int wbase = tile * kSortTile + warp * 32 * kSortItems;
    const unsigned lt = (1u << lane) - 1u;
    unsigned key[kSortItems], rk[kSortItems];
    int val[kSortItems], dg[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int idx = wbase + r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? kin[idx] : 0u;
        val[r] = valid ? (ident ? idx : vin[idx]) : 0;
        dg[r] = valid ? (int)((key[r] >> shift) & 255u) : 256;   // 256: no key
    }
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {   // rank within the warp, in index order
        const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
        const unsigned before = dg[r] < 256 ? s_whist[warp][dg[r]] : 0u;
        __syncwarp();
        if (dg[r] < 256 && (peers & lt) == 0u) s_whist[warp][dg[r]] = before + __popc(peers);
        __syncwarp();
        rk[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {   // thread d: digit d's prefix over the warps, the tile's count, and its look-back
        const int d = threadIdx.x;
        unsigned tot = 0u;
#pragma unroll
        for (int w = 0; w < W; w++) {
            const unsigned c = s_whist[w][d];
            s_whist[w][d] = tot;
            tot += c;
        }
        unsigned* my = status + (size_t)tile * 256 + d;
        unsigned excl = 0u;
        if (tile == 0) {
            st_relaxed_u32(my, kFlagInc | tot);
        } else {
            st_relaxed_u32(my, kFlagAgg | tot);
            // look back four predecessors at a time (their loads in flight together),
            // adding their counts in order until an inclusive one
            unsigned long long t0 = 0;
            for (int pred = tile - 1; pred >= 0;) {
                unsigned v[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    v[u] = pred - u >= 0 ? ld_relaxed_u32(status + (size_t)(pred - u) * 256 + d) : kFlagInc;
                bool done = false, waiting = false;
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (done || waiting) continue;
                    if (pred - u < 0) {
                        done = true;
                        continue;
                    }
                    if ((v[u] & ~kCountMask) == 0u) {   // not published yet: wait for it
                        waiting = true;
                        pred -= u;
                        continue;
                    }
                    excl += v[u] & kCountMask;
                    if (v[u] & kFlagInc) done = true;
                }
                if (done) break;
                if (!waiting) {
                    pred -= 4;
                    continue;
                }
                __nanosleep(32);   // bounded wait for tile `pred`
                if (t0 == 0) t0 = global_ns();
                else if (global_ns() - t0 > kWaitLimitNs) {
                    atomicCAS(err, 0, (int)BL_ETIMEOUT);
                    break;
                }
            }
            st_relaxed_u32(my, kFlagInc | (excl + tot));
        }
        s_dst[d] = base[d] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; r++)
        if (dg[r] < 256) {
            const unsigned dst = s_dst[dg[r]] + s_whist[warp][dg[r]] + rk[r];
            kout[dst] = key[r];
            vout[dst] = val[r];
        }
}

// ---------------------------------------------------------------------------
// quadtree (reading R10) and node sums (R11)
// ---------------------------------------------------------------------------

// levels 0..L share their prefix when the codes agree on the top 2L bits
__device__ __forceinline__ int common_levels(unsigned a, unsigned b) {
    const unsigned x = a ^ b;
    return x == 0u ? kLevels : (__clz(x) >> 1);
}

__device__ __forceinline__ void node_levels(const unsigned* codes, int n, int k, int& lmin,
                                            int& lmax) {
    const unsigned c = codes[k];
    if (k > 0 && codes[k - 1] == c) {   // no cell starts here
        lmin = 1;
        lmax = 0;
        return;
    }
    lmin = k == 0 ? 0 : common_levels(codes[k - 1], c) + 1;
    if (k == n - 1) {
        lmax = lmin;
    } else {
        lmax = min(kLevels, max(lmin, common_levels(c, codes[k + 1]) + 1));
    }
}

__global__ void node_count_kernel(const unsigned* __restrict__ codes, int n, int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n) return;
    if (k == n) {
        cnt[n] = 0;
        return;
    }
    int lmin, lmax;
    node_levels(codes, n, k, lmin, lmax);
    cnt[k] = lmax - lmin + 1;
}

// first index >= lo whose top 2l bits differ from `prefix` (codes sorted)
__device__ __forceinline__ int cell_end(const unsigned* codes, int n, int lo, unsigned c, int l) {
    if (l == 0) return n;
    const unsigned mask = l >= kLevels ? 0xFFFFFFFFu : ~(0xFFFFFFFFu >> (2 * l));
    const unsigned top = c & mask;
    int a = lo, b = n;   // codes[a] has the prefix; find the first > top|~mask
    const unsigned last = top | ~mask;
    while (a < b) {
        const int m = (a + b) >> 1;
        if (codes[m] <= last)
            a = m + 1;
        else
            b = m;
    }
    return a;
}

__global__ void node_emit_kernel(const unsigned* __restrict__ codes, int n,
                                 const int* __restrict__ first_node, int* __restrict__ nd_first,
                                 int* __restrict__ nd_count, int* __restrict__ nd_level,
                                 int* __restrict__ nd_skip, int* __restrict__ lvl_cnt) {
    __shared__ int s_cnt[kLevels + 1];   // this block's nodes per level
    if (threadIdx.x <= kLevels) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        int lmin, lmax;
        node_levels(codes, n, k, lmin, lmax);
        const int M = first_node[n];
        const unsigned c = codes[k];
        int v = first_node[k];
        for (int l = lmin; l <= lmax; l++, v++) {
            const int e = cell_end(codes, n, k + 1, c, l);
            nd_first[v] = k;
            nd_count[v] = e - k;
            nd_level[v] = l;
            nd_skip[v] = e >= n ? M : first_node[e];
            atomicAdd(&s_cnt[l], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x <= kLevels && s_cnt[threadIdx.x] > 0) atomicAdd(&lvl_cnt[threadIdx.x], s_cnt[threadIdx.x]);
}

// lvl[0..16] counts -> lvl[20..37] offsets, lvl[40..56] fill cursors
__global__ void level_offsets_kernel(int* __restrict__ lvl) {
    if (threadIdx.x != 0) return;
    int acc = 0;
    for (int l = 0; l <= kLevels; l++) {
        lvl[20 + l] = acc;
        lvl[40 + l] = acc;
        acc += lvl[l];
    }
    lvl[20 + kLevels + 1] = acc;
}

__global__ void level_bucket_kernel(const int* __restrict__ nd_level, const int* __restrict__ nd_first,
                                    const int* __restrict__ nd_count, const int* __restrict__ nd_skip,
                                    const int* __restrict__ first_node, int n, int* __restrict__ lvl,
                                    int4* __restrict__ lvl_info) {
    // each block buckets a contiguous range: count per level in shared memory,
    // reserve each level's room with one global atomic, then scatter each node's
    // build fields (read here in pre-order, so coalesced) into its level's slots
    __shared__ int s_cnt[kLevels + 1], s_base[kLevels + 1];
    const int M = first_node[n];
    const int per = (M + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per, hi = min(M, lo + per);
    if (threadIdx.x <= kLevels) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) atomicAdd(&s_cnt[nd_level[v]], 1);
    __syncthreads();
    if (threadIdx.x <= kLevels) {
        const int c = s_cnt[threadIdx.x];
        s_base[threadIdx.x] = c > 0 ? atomicAdd(&lvl[40 + threadIdx.x], c) : 0;
        s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const int l = nd_level[v];
        lvl_info[s_base[l] + atomicAdd(&s_cnt[l], 1)] = make_int4(v, nd_first[v], nd_count[v], nd_skip[v]);
    }
}

__global__ void level_sums_kernel(int l, const int* __restrict__ lvl, const int4* __restrict__ lvl_info,
                                  const float2* __restrict__ spos, const int* __restrict__ nd_skip,
                                  const float* __restrict__ box, float2* __restrict__ nd_sum,
                                  float4* __restrict__ nd_rec, int2* __restrict__ nd_aux) {
    // Programmatic dependent launch: the next level's grid may be scheduled now, and
    // this grid reads nothing before the previous level's grid has completed and its
    // writes are visible.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lo = lvl[20 + l], hi = lvl[20 + l + 1];
    const float Dl2 = box[4 + l];
    for (int q = lo + blockIdx.x * blockDim.x + threadIdx.x; q < hi; q += gridDim.x * blockDim.x) {
        const int4 info = lvl_info[q];   // {node, first, count, skip}
        const int v = info.x, f = info.y, cnt = info.z, skip = info.w;
        const bool leaf = cnt == 1 || l == kLevels;
        float sx, sy;
        if (leaf) {
            sx = 0.f;
            sy = 0.f;
            for (int m = 0; m < cnt; m++) {   // vertices in sorted order
                const float2 p = spos[f + m];
                sx = __fadd_rn(sx, p.x);
                sy = __fadd_rn(sy, p.y);
            }
        } else {
            int c = v + 1;   // children in order, via skip links
            sx = nd_sum[c].x;
            sy = nd_sum[c].y;
            c = nd_skip[c];
            while (c < skip) {
                sx = __fadd_rn(sx, nd_sum[c].x);
                sy = __fadd_rn(sy, nd_sum[c].y);
                c = nd_skip[c];
            }
        }
        nd_sum[v] = make_float2(sx, sy);
        const float fc = (float)cnt;
        nd_rec[v] = make_float4(__fdiv_rn(sx, fc), __fdiv_rn(sy, fc), Dl2, fc);
        nd_aux[v] = make_int2(skip, leaf ? f : -1);
    }
}

__global__ void gather_sorted_kernel(const int* __restrict__ perm, const float2* __restrict__ pos,
                                     int n, float2* __restrict__ spos) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) spos[k] = pos[perm[k]];
}

// ---------------------------------------------------------------------------
// theta-walk (Algorithm S4), one query per lane; KAHAN: every term compensated
// ---------------------------------------------------------------------------

// s += v, compensated (Kahan) when KAHAN
template <bool KAHAN>
__device__ __forceinline__ void acc_add(float& s, float& c, float v) {
    if (KAHAN)
        kahan_add(s, c, v);
    else
        s += v;
}

template <bool KAHAN>
__global__ void __launch_bounds__(256) walk_kernel(
    const int* __restrict__ perm, const float2* __restrict__ spos, const int* __restrict__ first_node,
    int n, const float4* __restrict__ nd_rec, const int2* __restrict__ nd_aux, float theta2,
    float2* __restrict__ rep, unsigned long long* __restrict__ counts, int2* __restrict__ qcounts) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;   // sorted position = query
    const int M = first_node[n];
    const bool active = q < n;
    const int i = active ? perm[q] : -1;
    const float2 me = active ? spos[q] : make_float2(0.f, 0.f);
    float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
    unsigned next = active ? 0u : (unsigned)M;
    unsigned far = 0, near = 0, visits = 0;   // visits: node records this lane read
    auto visit = [&](unsigned v) {
        const float4 rec = nd_rec[v];
        const int2 aux = nd_aux[v];
        if (aux.y >= 0) {   // leaf: its vertices directly, self skipped by index
            const int cnt = (int)rec.w;
            near += (unsigned)cnt;   // leaf vertices visited, the query's own included
            for (int m = 0; m < cnt; m++) {
                const int k = aux.y + m;
                if (k == q) continue;   // the query itself: sorted position q is vertex i
                const float2 p = cnt == 1 ? make_float2(rec.x, rec.y) : spos[k];
                float ax = 0.f, ay = 0.f;
                rep_pair(me.x, me.y, p.x, p.y, ax, ay);
                acc_add<KAHAN>(sx, cx, ax);
                acc_add<KAHAN>(sy, cy, ay);
            }
            next = v + 1u;
        } else {
            const float dx = __fsub_rn(rec.x, me.x);
            const float dy = __fsub_rn(rec.y, me.y);
            const float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
            if (rec.z < __fmul_rn(theta2, d2)) {   // acceptance test (Section 3.5)
                const float w = __fmul_rn(rec.w, rcp_sfu(d2));
                acc_add<KAHAN>(sx, cx, dx * w);
                acc_add<KAHAN>(sy, cy, dy * w);
                far++;
                next = (unsigned)aux.x;
            } else {
                next = v + 1u;
            }
        }
    };
    // Every lane walks its own query's pre-order sequence at its own pace (the
    // lanes of a warp are neighbouring queries, so they mostly read the same hot
    // nodes, from L1); a lane's terms and their order are those of its own walk.
    while (__any_sync(0xffffffffu, next < (unsigned)M)) {
        if (next < (unsigned)M) {
            visits++;
            visit(next);
        }
    }
    if (active) rep[i] = make_float2(sx - cx, sy - cy);
    if (active && qcounts != nullptr) qcounts[i] = make_int2((int)far, (int)near);   // parity hook
    // interaction counts for reporting
    unsigned long long f = far, nr = near, vs = visits;
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o);
        nr += __shfl_xor_sync(0xffffffffu, nr, o);
        vs += __shfl_xor_sync(0xffffffffu, vs, o);
    }
    if ((threadIdx.x & 31) == 0 && counts != nullptr) {
        atomicAdd(&counts[0], f);
        atomicAdd(&counts[1], nr);
        atomicAdd(&counts[2], vs);
    }
}

// rep[i] -= exact repulsion of i's CSR neighbours at S (warp per row)
__global__ void nbr_correct_kernel(const int* __restrict__ rowptr, const int* __restrict__ colids,
                                   const float2* __restrict__ S, int n, float2* __restrict__ rep) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int i = warp;
    const float2 me = S[i];
    float ax = 0.f, ay = 0.f;
    for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
        const float2 p = S[colids[e]];
        rep_pair(me.x, me.y, p.x, p.y, ax, ay);
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    if (lane == 0) {
        const float2 r = rep[i];
        rep[i] = make_float2(r.x - ax, r.y - ay);
    }
}

// snapshot forces: ct_i = attraction at S + (-R K^2) rep_i (warp per row)
__global__ void bh_snapshot_force_kernel(const int* __restrict__ rowptr, const int* __restrict__ colids,
                                         const float2* __restrict__ S, int n, const float2* __restrict__ rep,
                                         float invK, int am, float negRK2, float2* __restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int i = warp;
    const float2 me = S[i];
    float ax = 0.f, ay = 0.f;
    for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
        const float2 p = S[colids[e]];
        const float dx = p.x - me.x, dy = p.y - me.y;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, BL_EPS2));
        const float a = attr_scale(d2, am) * invK;
        ax = fmaf(dx, a, ax);
        ay = fmaf(dy, a, ay);
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    if (lane == 0) {
        const float2 r = rep[i];
        out[i] = make_float2(fmaf(negRK2, r.x, ax), fmaf(negRK2, r.y, ay));
    }
}

// ---------------------------------------------------------------------------
// minibatch sweep (Algorithm S5's batch loop)
// ---------------------------------------------------------------------------

// Attraction of row i from its neighbours in its own or later minibatches: they
// have not moved yet when i's minibatch runs, so this part uses the snapshot S
// and is computed for all rows before the sweep (edge_pass_kernel, warp per row;
// rows with more than kBigRow edges get a whole block from edge_pass_big_kernel).
constexpr int kBigRow = 8192;

__device__ __forceinline__ void attr_term(float2 me, float2 p, float invK, int am, float& ax, float& ay) {
    const float dx = p.x - me.x, dy = p.y - me.y;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, BL_EPS2));
    const float sc = attr_scale(d2, am) * invK;
    ax = fmaf(dx, sc, ax);
    ay = fmaf(dy, sc, ay);
}

// One pass over every row's edges at the snapshot S: the attraction of the
// neighbours in the row's own or later minibatches (edges from split[i] on; they
// have not moved when the row's minibatch does) and, unless repulse_neighbors, the
// repulsion the tree gave the neighbours, taken back out of rep. A warp per row;
// rows with more than kBigRow edges are left to edge_pass_big_kernel.
__device__ __forceinline__ void edge_terms_strided(const int* __restrict__ colids,
                                                   const float2* __restrict__ S, float2 me, int e0,
                                                   int e1, int es, int start, int stride, float invK,
                                                   int am, bool rn, float& ax, float& ay, float& qx, float& qy) {
    for (int e = e0 + start; e < e1; e += 4 * stride) {
        int j[4];
        float2 p[4];
#pragma unroll
        for (int k = 0; k < 4; k++) j[k] = e + k * stride < e1 ? __ldg(&colids[e + k * stride]) : -1;
#pragma unroll
        for (int k = 0; k < 4; k++) p[k] = j[k] >= 0 ? S[j[k]] : me;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (j[k] < 0) continue;
            if (e + k * stride >= es) attr_term(me, p[k], invK, am, ax, ay);
            if (!rn) rep_pair(me.x, me.y, p[k].x, p[k].y, qx, qy);
        }
    }
}

constexpr int kShortRow = 256;   // rows up to this many edges: 8 lanes each

// old[i]: attraction from the neighbours that do not move before row i does;
// corr[i]: exact repulsion of all of i's neighbours (zero when the tree's
// repulsion keeps them), taken off the tree sum when the row is finished
__device__ __forceinline__ void edge_pass_finish(int i, float ax, float ay, float qx, float qy,
                                                 float2* __restrict__ old, float2* __restrict__ corr) {
    old[i] = make_float2(ax, ay);
    corr[i] = make_float2(qx, qy);
}

// Short rows (most of them): 8 lanes per row, 4 rows per warp.
__global__ void edge_pass_kernel(const int* __restrict__ rowptr, const int* __restrict__ colids,
                                 const int* __restrict__ split, const float2* __restrict__ S, int n,
                                 float invK, int am, int rn, float2* __restrict__ old,
                                 float2* __restrict__ corr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t >> 3, sub = t & 7;
    const unsigned mask = 0xFFu << (threadIdx.x & 24);   // this row's 8 lanes
    if (i >= n) return;   // whole 8-lane groups
    const int e0 = rowptr[i], e1 = rowptr[i + 1];
    if (e1 - e0 > kShortRow) return;   // edge_pass_mid_kernel / edge_pass_big_kernel
    const float2 me = S[i];
    float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
    edge_terms_strided(colids, S, me, e0, e1, split[i], sub, 8, invK, am, rn != 0, ax, ay, qx, qy);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(mask, ax, o);
        ay += __shfl_xor_sync(mask, ay, o);
        qx += __shfl_xor_sync(mask, qx, o);
        qy += __shfl_xor_sync(mask, qy, o);
    }
    if (sub == 0) edge_pass_finish(i, ax, ay, qx, qy, old, corr);
}

// Rows with more than kShortRow and at most kBigRow edges: a warp each.
__global__ void edge_pass_mid_kernel(const int* __restrict__ rowptr, const int* __restrict__ colids,
                                     const int* __restrict__ split, const float2* __restrict__ S,
                                     const int* __restrict__ mid_rows, int nmid, float invK, int am, int rn,
                                     float2* __restrict__ old, float2* __restrict__ corr) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nmid) return;
    const int i = mid_rows[w];
    const float2 me = S[i];
    float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
    edge_terms_strided(colids, S, me, rowptr[i], rowptr[i + 1], split[i], lane, 32, invK, am, rn != 0, ax, ay,
                       qx, qy);
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    qx = warp_sum(qx);
    qy = warp_sum(qy);
    if (lane == 0) edge_pass_finish(i, ax, ay, qx, qy, old, corr);
}

__global__ void __launch_bounds__(1024) edge_pass_big_kernel(
    const int* __restrict__ rowptr, const int* __restrict__ colids, const int* __restrict__ split,
    const float2* __restrict__ S, const int* __restrict__ big_rows, float invK, int am, int rn,
    float2* __restrict__ old, float2* __restrict__ corr) {
    __shared__ float4 s_w[32];
    const int i = big_rows[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float2 me = S[i];
    float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
    edge_terms_strided(colids, S, me, rowptr[i], rowptr[i + 1], split[i], threadIdx.x, blockDim.x, invK,
                       am, rn != 0, ax, ay, qx, qy);
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    qx = warp_sum(qx);
    qy = warp_sum(qy);
    if (lane == 0) s_w[warp] = make_float4(ax, ay, qx, qy);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            t.x += s_w[w].x;
            t.y += s_w[w].y;
            t.z += s_w[w].z;
            t.w += s_w[w].w;
        }
        edge_pass_finish(i, t.x, t.y, t.z, t.w, old, corr);
    }
}

// The sweep. Row i reads its neighbours in earlier minibatches at their new
// positions, so it can run once they have moved; its neighbours in its own or
// later minibatches are read at the snapshot, whatever the order. With
// level(i) = 1 + max level of i's earlier-minibatch neighbours (1 when there are
// none), all rows of one level are independent of each other and depend only on
// lower levels, and any order that runs a row after its earlier-minibatch
// neighbours computes exactly the sequential minibatch sweep. Tasks are stored
// level by level; a row with many earlier-minibatch edges is cut into segments
// (tasks) whose partial sums segment 0's warp combines in a fixed order. Such a
// row's earlier-minibatch columns are listed highest level first (`scol`), so
// segment 0 holds the neighbours that finish last, and the later segments, which
// need only lower levels, are scheduled at those levels: segment 0's warp waits
// for its neighbours and, in the same polling loop, for the other segments'
// partial sums, which are usually published long before.
struct SweepArgs {
    const int* rowptr;
    const int* colids;
    const int* scol;         // rows of several segments: their earlier-minibatch columns
    const float2* bold;      // positions at iteration start (S)
    float2* bnew;            // positions after this iteration's update
    const float2* rep;       // repulsion sums of the tree walk (unscaled)
    const float2* corr;      // their neighbour correction, rep - corr is the row's repulsion
    const float2* old;       // attraction from not-yet-moved neighbours
    const int* lvl_ptr;      // tasks of level l: [lvl_ptr[l], lvl_ptr[l+1])
    const int4* tasks;       // {row, first edge, end edge, segment | nseg << 16}
    const int* seg_off;      // per row: offset of its segment sums (rows with nseg > 1)
    float2* seg_sum;         // per row: partial sums of its segments 1.., all-ones until published
    double* e_row;           // |ct|^2 of every row
    int* status;
    int nlevels;
    int first_level;         // levels before it are done by level0_kernel
    int am;                  // attraction exponent a of the (a,-1) model
    float invK, negRK2, stepf;
    unsigned long long* trace;   // optional: start time of each level (CTA 0)
    unsigned long long* ttrace;  // optional: per task {start, neighbours gathered, done}
};

constexpr int kSegEdges = 128;   // earlier-minibatch edges per task (4 gathers per lane)
constexpr int kMaxSeg = 257;     // segments of one row (segment 0's warp reads the other 256)

// New positions are published with one 64-bit store (single-copy atomic), and
// before the sweep every slot holds kUnset (two NaNs no position can take): a
// row that needs a moved neighbour reads the slot until it is set. The position
// is its own ready flag.
constexpr unsigned long long kUnset = ~0ull;

__device__ __forceinline__ void publish_pos(float2* p, float x, float y) {
    const unsigned long long v =
        (unsigned long long)__float_as_uint(x) | ((unsigned long long)__float_as_uint(y) << 32);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long read_pos(const float2* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float2 unpack_pos(unsigned long long v) {
    return make_float2(__uint_as_float((unsigned)v), __uint_as_float((unsigned)(v >> 32)));
}

// The row's repulsion sum: the tree's, less its CSR neighbours' exact terms.
__device__ __forceinline__ float2 row_rep(const SweepArgs& a, int i) {
    const float2 r = a.rep[i], q = a.corr[i];
    return make_float2(__fsub_rn(r.x, q.x), __fsub_rn(r.y, q.y));
}

// The row's update: ct = attraction (this iteration's moved neighbours sx,sy +
// the not-yet-moved ones od) + repulsion rp scaled by -RK^2; me = start position.
__device__ __forceinline__ void finish_row(const SweepArgs& a, int i, float2 me, float2 rp, float2 od,
                                           float sx, float sy) {
    const float fx = fmaf(a.negRK2, rp.x, sx + od.x);
    const float fy = fmaf(a.negRK2, rp.y, sy + od.y);
    float nx = me.x, ny = me.y, gx = fx, gy = fy;
    float n2 = fmaf(gx, gx, gy * gy);
    if (n2 > 0.f) {
        if (!(n2 < INFINITY)) {
            gx *= 0x1p-64f;
            gy *= 0x1p-64f;
            n2 = fmaf(gx, gx, gy * gy);
        }
        const float sc = a.stepf * rsqrt_sfu(n2);
        nx = fmaf(sc, gx, me.x);
        ny = fmaf(sc, gy, me.y);
    }
    publish_pos(&a.bnew[i], nx, ny);   // first: the rows waiting for it
    a.e_row[i] = (double)fmaf(fx, fx, fy * fy);
}

// Everything a task needs that the sweep does not change: the task record, the
// row's start position, repulsion and not-yet-moved attraction, and the column
// ids of its first 128 edges (4 per lane). A warp loads its next task's while it
// runs the current one, so that a task then waits only for the moved neighbours'
// positions.
struct TaskPre {
    int4 tk;
    float2 me, rp, od;
    int off;   // the row's first segment slot (rows of several segments)
    int j[4];
};

// The static data of a task whose record `rec` is already in registers (the
// records are loaded one task earlier still, so no load here waits on another).
__device__ __forceinline__ void task_prefetch_rec(const SweepArgs& a, int4 rec, int lane, TaskPre& p) {
    p.tk = rec;
    const int i = p.tk.x;
    p.me = a.bold[i];
    p.rp = row_rep(a, i);
    p.od = a.old[i];
    const bool multi = (p.tk.w >> 16) > 1;
    p.off = multi ? a.seg_off[i] : 0;
    const int* cols = multi ? a.scol : a.colids;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int e = p.tk.y + lane + 32 * k;
        p.j[k] = e < p.tk.z ? __ldg(&cols[e]) : -1;
    }
}

// The first level: rows with no neighbour in an earlier minibatch. Nothing they
// read moves during the sweep, so they need no waiting: one thread per row.
__global__ void level0_kernel(SweepArgs a) {
    const int t1 = a.lvl_ptr[1];
    for (int t = a.lvl_ptr[0] + blockIdx.x * blockDim.x + threadIdx.x; t < t1; t += gridDim.x * blockDim.x) {
        const int i = a.tasks[t].x;
        finish_row(a, i, a.bold[i], row_rep(a, i), a.old[i], 0.f, 0.f);
    }
}

// Dataflow sweep: no level barriers. Warps take the tasks round robin in list
// order (task t goes to warp t mod warps); a task reads each moved neighbour's
// slot (and segment 0 its row's partial-sum slots) until it is published. Every
// task waits only for tasks earlier in the list, so the earliest unfinished task
// has all its inputs and its warp has finished everything before it, and all CTAs
// are resident (cooperative launch): the sweep cannot stall. Every wait is bounded
// (BL_ETIMEOUT).
struct Gather4 {
    int j[4];
    unsigned long long v[4];
};

// Reads the published positions of up to 4 ids per lane and, when `slot` is not
// null, the lane's segment partial-sum slot into `sv`, until all are set; false
// when the wait gave up.
__device__ __forceinline__ bool gather_wait(const SweepArgs& a, Gather4& g, int lane,
                                            const float2* slot, unsigned long long& sv) {
#pragma unroll
    for (int k = 0; k < 4; k++) g.v[k] = g.j[k] >= 0 ? read_pos(&a.bnew[g.j[k]]) : 0ull;
    if (slot != nullptr && sv == kUnset) sv = read_pos(slot);
    unsigned long long t0 = 0;
    for (unsigned spin = 0;; ++spin) {
        bool pending = slot != nullptr && sv == kUnset;
#pragma unroll
        for (int k = 0; k < 4; k++) pending |= g.j[k] >= 0 && g.v[k] == kUnset;
        if (!__any_sync(0xffffffffu, pending)) return true;
        __nanosleep(64);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (g.j[k] >= 0 && g.v[k] == kUnset) g.v[k] = read_pos(&a.bnew[g.j[k]]);
        if (slot != nullptr && sv == kUnset) sv = read_pos(slot);
        if ((spin & 127u) == 127u) {
            int bad = 0;
            if (lane == 0) {
                if (t0 == 0) t0 = global_ns();
                if (ld_volatile_i32(a.status) != 0) bad = 1;
                else if (global_ns() - t0 > kWaitLimitNs) {
                    atomicCAS(a.status, 0, (int)BL_ETIMEOUT);
                    bad = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) return false;
        }
    }
}

// A later segment's partial sum, published with one 64-bit store (a pair whose bits
// equal the all-ones unset pattern is stored as canonical NaNs).
__device__ __forceinline__ void publish_partial(float2* p, float x, float y) {
    unsigned long long v = (unsigned long long)__float_as_uint(x) | ((unsigned long long)__float_as_uint(y) << 32);
    if (v == kUnset) v = 0x7FFFFFFF7FFFFFFFull;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Segment 0's warp reads the partial sums of segments 1..nseg-1 of its row (lane l
// takes segments 1 + l + 32 m) until all are published, and sums all nseg of them
// (its own p0 in lane 0) in a fixed order: each lane its segments in order of m,
// then a fixed butterfly across the lanes. Bounded like gather_wait: false when the
// wait gave up.
__device__ __forceinline__ bool seg_wait(const SweepArgs& a, int off, int nseg, int lane, float p0x,
                                         float p0y, float& tx, float& ty) {
    constexpr int M = (kMaxSeg - 1 + 31) / 32;
    unsigned long long v[M];
#pragma unroll
    for (int m = 0; m < M; m++) {
        const int q = 1 + lane + 32 * m;
        v[m] = q < nseg ? read_pos(&a.seg_sum[off + q]) : 0ull;
    }
    unsigned long long t0 = 0;
    for (unsigned spin = 0;; ++spin) {
        bool pending = false;
#pragma unroll
        for (int m = 0; m < M; m++) pending |= 1 + lane + 32 * m < nseg && v[m] == kUnset;
        if (!__any_sync(0xffffffffu, pending)) break;
        __nanosleep(64);
#pragma unroll
        for (int m = 0; m < M; m++) {
            const int q = 1 + lane + 32 * m;
            if (q < nseg && v[m] == kUnset) v[m] = read_pos(&a.seg_sum[off + q]);
        }
        if ((spin & 127u) == 127u) {
            int bad = 0;
            if (lane == 0) {
                if (t0 == 0) t0 = global_ns();
                if (ld_volatile_i32(a.status) != 0) bad = 1;
                else if (global_ns() - t0 > kWaitLimitNs) {
                    atomicCAS(a.status, 0, (int)BL_ETIMEOUT);
                    bad = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) return false;
        }
    }
    float sx = lane == 0 ? p0x : 0.f, sy = lane == 0 ? p0y : 0.f;
#pragma unroll
    for (int m = 0; m < M; m++) {
        const int q = 1 + lane + 32 * m;
        if (q < nseg) {
            const float2 w = unpack_pos(v[m]);
            sx += w.x;
            sy += w.y;
        }
    }
    tx = warp_sum(sx);
    ty = warp_sum(sy);
    return true;
}

__device__ __forceinline__ bool task_run_df(const SweepArgs& a, const TaskPre& p, int lane, int t) {
    const int i = p.tk.x;
    if (a.ttrace && lane == 0) a.ttrace[3 * (size_t)t] = global_ns();
    const int seg = p.tk.w & 0xFFFF, nseg = p.tk.w >> 16;
    const float2 me = p.me;
    const int* cols = nseg > 1 ? a.scol : a.colids;
    // segment 0 of a row of at most 33 segments: lane l also waits for segment
    // 1 + l's partial sum
    const bool early = seg == 0 && nseg > 1 && nseg <= 33;
    const float2* slot = early && 1 + lane < nseg ? &a.seg_sum[p.off + 1 + lane] : nullptr;
    unsigned long long sv = kUnset;
    float sx = 0.f, sy = 0.f;
    Gather4 g;
#pragma unroll
    for (int k = 0; k < 4; k++) g.j[k] = p.j[k];
    for (int e = p.tk.y + lane;;) {
        if (!gather_wait(a, g, lane, slot, sv)) return false;
        if (a.ttrace && lane == 0 && e == p.tk.y) a.ttrace[3 * (size_t)t + 1] = global_ns();
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (g.j[k] >= 0) attr_term(me, unpack_pos(g.v[k]), a.invK, a.am, sx, sy);
        e += 128;
        if (!__any_sync(0xffffffffu, e < p.tk.z)) break;
#pragma unroll
        for (int k = 0; k < 4; k++) g.j[k] = e + 32 * k < p.tk.z ? __ldg(&cols[e + 32 * k]) : -1;
    }
    if (early) {
        // one butterfly over lane l's own terms plus segment 1 + l's partial sum
        if (slot != nullptr) {
            const float2 w = unpack_pos(sv);
            sx += w.x;
            sy += w.y;
        }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        if (lane == 0) finish_row(a, i, me, p.rp, p.od, sx, sy);
        if (a.ttrace && lane == 0) a.ttrace[3 * (size_t)t + 2] = global_ns();
        return true;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (nseg <= 1) {
        if (lane == 0) finish_row(a, i, me, p.rp, p.od, sx, sy);
    } else if (seg > 0) {
        // a later segment: its partial sum goes to its slot for segment 0's warp
        if (lane == 0) publish_partial(&a.seg_sum[p.off + seg], sx, sy);
    } else {
        // segment 0 combines the partials as the other segments publish them
        float tx, ty;
        if (!seg_wait(a, p.off, nseg, lane, sx, sy, tx, ty)) return false;
        if (lane == 0) finish_row(a, i, me, p.rp, p.od, tx, ty);
    }
    if (a.ttrace && lane == 0) a.ttrace[3 * (size_t)t + 2] = global_ns();
    return true;
}

// three CTAs per SM (the launch's shape): 80 registers a thread, no spills; more
// warps for the tasks than two CTAs give (R-MAT 20 sweep 0.563 -> 0.552 ms)
__global__ void __launch_bounds__(kSweepThreads, 3) dataflow_sweep_kernel(SweepArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int l0 = a.first_level;
    if (l0 >= a.nlevels) return;
    const int t1 = a.lvl_ptr[a.nlevels];
    int t = a.lvl_ptr[l0] + gw;
    int lnext = l0;   // trace: next level whose first task this warp may meet
    if (a.trace && gw == 0 && lane == 0)
        for (int q = 0; q < l0; q++) a.trace[q] = global_ns();
    // software pipeline over this warp's tasks t, t+nw, t+2nw, ...: while task t runs,
    // the static data of task t+nw is in flight and the record of task t+2nw too
    TaskPre cur;
    const int4 none = make_int4(0, 0, 0, 0);
    if (t < t1) task_prefetch_rec(a, a.tasks[t], lane, cur);
    int4 rec1 = t + nw < t1 ? a.tasks[t + nw] : none;
    for (; t < t1; t += nw) {
        if (a.trace && lane == 0) {
            while (lnext < a.nlevels && a.lvl_ptr[lnext] < t) lnext++;
            if (lnext < a.nlevels && a.lvl_ptr[lnext] == t) a.trace[lnext] = global_ns();
        }
        const int4 rec2 = t + 2 * nw < t1 ? a.tasks[t + 2 * nw] : none;   // two tasks ahead
        TaskPre nxt;
        const bool more = t + nw < t1;
        if (more) task_prefetch_rec(a, rec1, lane, nxt);   // static data of the next task
        if (!task_run_df(a, cur, lane, t)) return;
        if (more) cur = nxt;
        rec1 = rec2;
    }
    if (a.trace && lane == 0) atomicMax(&a.trace[a.nlevels], (unsigned long long)global_ns());
}

// energy of the iteration: fixed-order reduction of the rows' |ct|^2
__global__ void row_energy_kernel(const double* __restrict__ e_row, int n, double* __restrict__ part) {
    __shared__ double s_w[32];
    double e = 0.0;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per, hi = min(n, lo + per);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) e += e_row[i];
    e = warp_sum_d(e);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
        part[blockIdx.x] = t;
    }
}

__global__ void energy_parts_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
    double e = 0.0;
    for (int b = threadIdx.x; b < np; b += 32) e += part[b];
    e = warp_sum_d(e);
    if (threadIdx.x == 0) *out = e;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

static bl_status bh_ensure(bl_layout* L) {
    const int n = L->g->n;
    if ((int64_t)n > kBHMaxN)
        return set_error(BL_EINVAL, "Barnes-Hut mode: more vertices than the quadtree's 32-bit node indices allow");
    if (!L->bh) L->bh = new BHState();
    BHState* s = L->bh;
    if (!s->side) BL_CUDA_TRY(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
    if (!s->ev_fork) BL_CUDA_TRY(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
    if (!s->ev_join) BL_CUDA_TRY(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
    if (!s->hi) {
        int lo_prio = 0, hi_prio = 0;
        BL_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
        BL_CUDA_TRY(cudaStreamCreateWithPriority(&s->hi, cudaStreamNonBlocking, hi_prio));
    }
    if (!s->ev_in) BL_CUDA_TRY(cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming));
    if (!s->ev_out) BL_CUDA_TRY(cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming));
    if (s->n == n && s->cap_nodes > 0) return BL_OK;
    const Allocator& al = L->alloc;
    const size_t N = (size_t)n;
    const int nb_sort = div_up(n, kSortTile);
    const int64_t cap = 17 * (int64_t)n + 1;
    BL_TRY(s->keys0.ensure(al, N * 4));
    BL_TRY(s->keys1.ensure(al, N * 4));
    BL_TRY(s->vals0.ensure(al, N * 4));
    BL_TRY(s->vals1.ensure(al, N * 4));
    // radix sort: digit counts/bases [4][256], tile tickets [4] (at +1024), then
    // the look-back words [4][tiles][256]
    BL_TRY(s->hist.ensure(al, ((size_t)1024 + 64 + (size_t)4 * nb_sort * 256) * 4));
    BL_TRY(s->scan_part.ensure(al, (size_t)(div_up(std::max<int64_t>(cap, (int64_t)256 * nb_sort), kScanItems) + 1) * 4));
    BL_TRY(s->bpart.ensure(al, 1024 * sizeof(float4)));
    BL_TRY(s->box.ensure(al, 32 * sizeof(float)));
    BL_TRY(s->cnt.ensure(al, (N + 1) * 4));
    BL_TRY(s->spos.ensure(al, N * sizeof(float2)));
    BL_TRY(s->nd_first.ensure(al, (size_t)cap * 4));
    BL_TRY(s->nd_count.ensure(al, (size_t)cap * 4));
    BL_TRY(s->nd_level.ensure(al, (size_t)cap * 4));
    BL_TRY(s->nd_skip.ensure(al, (size_t)cap * 4));
    BL_TRY(s->nd_sum.ensure(al, (size_t)cap * sizeof(float2)));
    BL_TRY(s->nd_rec.ensure(al, (size_t)cap * sizeof(float4)));
    BL_TRY(s->nd_aux.ensure(al, (size_t)cap * sizeof(int2)));
    BL_TRY(s->lvl.ensure(al, 64 * 4));
    BL_TRY(s->lvl_info.ensure(al, (size_t)cap * sizeof(int4)));
    BL_TRY(s->rep.ensure(al, N * sizeof(float2)));
    BL_TRY(s->walkcnt.ensure(al, 4 * sizeof(unsigned long long)));
    s->n = n;
    s->cap_nodes = cap;
    return BL_OK;
}

// Builds the tree of positions S; leaves codes/perm (sorted) in keys0/vals0.
// marks (optional, phase timing): events recorded after the Morton codes and
// after the sort.
static bl_status bh_build(bl_layout* L, const float2* S, cudaStream_t st, cudaEvent_t* marks = nullptr) {
    BHState* s = L->bh;
    const int n = L->g->n;
    const int nbb = std::min(1024, div_up(n, 256));
    bbox_partial_kernel<<<nbb, 256, 0, st>>>(S, n, s->bpart.as<float4>());
    bbox_final_kernel<<<1, 32, 0, st>>>(s->bpart.as<float4>(), nbb, s->box.as<float>());
    morton_kernel<<<div_up(n, 256), 256, 0, st>>>(S, n, s->box.as<float>(), s->keys0.as<unsigned>(),
                                                  s->vals0.as<int>());
    if (marks) BL_CUDA_TRY(cudaEventRecord(marks[0], st));
    const int nbs = div_up(n, kSortTile);
    unsigned* kin = s->keys0.as<unsigned>();
    unsigned* kout = s->keys1.as<unsigned>();
    int* vin = s->vals0.as<int>();
    int* vout = s->vals1.as<int>();
    unsigned* hist = s->hist.as<unsigned>();
    unsigned* tickets = hist + 1024;
    unsigned* look = hist + 1024 + 64;
    BL_CUDA_TRY(cudaMemsetAsync(hist, 0, ((size_t)1024 + 64 + (size_t)4 * nbs * 256) * 4, st));
    radix_hist4_kernel<<<std::min(nbs * 4, device_sm_count() * 4), 256, 0, st>>>(kin, n, hist);
    radix_bases_kernel<<<1, 256, 0, st>>>(hist);
    for (int pass = 0; pass < 4; pass++) {
        radix_pass_kernel<<<nbs, kSortThreads, 0, st>>>(kin, vin, n, 8 * pass, hist + 256 * pass,
                                                        look + (size_t)pass * nbs * 256, tickets + pass,
                                                        pass == 0 ? 1 : 0, static_cast<int*>(L->status.p),
                                                        kout, vout);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    if (marks) BL_CUDA_TRY(cudaEventRecord(marks[1], st));
    // after 4 passes the sorted data is back in keys0/vals0
    gather_sorted_kernel<<<div_up(n, 256), 256, 0, st>>>(vin, S, n, s->spos.as<float2>());
    node_count_kernel<<<div_up(n + 1, 256), 256, 0, st>>>(kin, n, s->cnt.as<int>());
    BL_TRY(exclusive_scan(s->cnt.as<int>(), s->cnt.as<int>(), n + 1, s->scan_part.as<int>(), st));
    BL_CUDA_TRY(cudaMemsetAsync(s->lvl.p, 0, 64 * 4, st));
    node_emit_kernel<<<div_up(n, 256), 256, 0, st>>>(kin, n, s->cnt.as<int>(), s->nd_first.as<int>(),
                                                     s->nd_count.as<int>(), s->nd_level.as<int>(),
                                                     s->nd_skip.as<int>(), s->lvl.as<int>());
    level_offsets_kernel<<<1, 32, 0, st>>>(s->lvl.as<int>());
    const int sms = device_sm_count();
    level_bucket_kernel<<<sms * 4, 256, 0, st>>>(s->nd_level.as<int>(), s->nd_first.as<int>(),
                                                 s->nd_count.as<int>(), s->nd_skip.as<int>(), s->cnt.as<int>(),
                                                 n, s->lvl.as<int>(), s->lvl_info.as<int4>());
    // bottom-up, one launch per level; each launch may start while the previous one
    // drains (programmatic dependent launch), and waits inside for its completion
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(div_up(n, 256), sms * 8));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int l = kLevels; l >= 0; l--)
        BL_CUDA_TRY(cudaLaunchKernelEx(&cfg, level_sums_kernel, l, (const int*)s->lvl.as<int>(),
                                       (const int4*)s->lvl_info.as<int4>(), (const float2*)s->spos.as<float2>(),
                                       (const int*)s->nd_skip.as<int>(), (const float*)s->box.as<float>(),
                                       s->nd_sum.as<float2>(), s->nd_rec.as<float4>(), s->nd_aux.as<int2>()));
    BL_CUDA_TRY(cudaGetLastError());
    return BL_OK;
}

// repulsion sums of every vertex from the tree of S, neighbours taken out
static bl_status bh_repulsion(bl_layout* L, const float2* S, float theta, cudaStream_t st,
                              bool correct = true, int2* qcounts = nullptr) {
    BHState* s = L->bh;
    const int n = L->g->n;
    BL_CUDA_TRY(cudaMemsetAsync(s->walkcnt.p, 0, 4 * sizeof(unsigned long long), st));
    const float th = theta;
    const float theta2 = th * th;
    auto walk = kahan_on(L->prm.kahan, n) ? walk_kernel<true> : walk_kernel<false>;
    walk<<<div_up(n, 256), 256, 0, st>>>(s->vals0.as<int>(), s->spos.as<float2>(), s->cnt.as<int>(), n,
                                         s->nd_rec.as<float4>(), s->nd_aux.as<int2>(), theta2,
                                         s->rep.as<float2>(), s->walkcnt.as<unsigned long long>(), qcounts);
    if (correct && !L->prm.repulse_neighbors)
        nbr_correct_kernel<<<div_up((int64_t)n * 32, 256), 256, 0, st>>>(
            L->g->rowptr.as<int>(), L->g->colids.as<int>(), S, n, s->rep.as<float2>());
    BL_CUDA_TRY(cudaGetLastError());
    return BL_OK;
}

// Per (graph, minibatch size): the split point of every row (first edge into its
// own or a later minibatch), the rows with many such edges, the level of every
// row and the sweep's tasks grouped by level.
// Earlier-minibatch edges per sweep task (rows with more are cut into segments);
// BL_BH_SEG overrides it.
static int seg_edges() {
    const char* e = std::getenv("BL_BH_SEG");
    const int v = e ? std::atoi(e) : 0;
    return v >= 32 ? v : kSegEdges;
}

static bl_status bh_plan(bl_layout* L, int BS, cudaStream_t st) {
    BHState* s = L->bh;
    const int segE = seg_edges();
    if (s->plan_bs == BS && s->plan_seg == segE) return BL_OK;
    const bl_graph* g = L->g;
    const int n = g->n;
    const int* rp = g->h_rowptr.data();
    const int* ci = g->h_colids.data();
    std::vector<int> split(n), level(n), bigrows, midrows;
    int nlev = 0;
    for (int i = 0; i < n; i++) {
        const int lo = (i / BS) * BS;
        const int* sp = std::lower_bound(ci + rp[i], ci + rp[i + 1], lo);
        split[i] = (int)(sp - ci);
        if (rp[i + 1] - rp[i] > kBigRow) bigrows.push_back(i);   // edge_pass_big_kernel
        else if (rp[i + 1] - rp[i] > kShortRow) midrows.push_back(i);   // edge_pass_mid_kernel
        int d = 0;
        for (const int* c = ci + rp[i]; c < sp; c++) d = std::max(d, level[*c]);
        level[i] = d + 1;
        nlev = std::max(nlev, d + 1);
    }
    // Tasks. A row of at most segE earlier-minibatch edges is one task at the row's
    // level. A longer row is cut into segments over its columns listed highest
    // level first: segment 0 (the highest levels) stays at the row's level, and a
    // later segment q, whose partial sum needs only its own columns, goes to level
    // 1 + (the highest level among them), so it runs as soon as those columns are
    // final rather than beside segment 0. Inside a level the later segments come
    // first; every task then waits only for tasks before it in the list (the
    // sweep's progress argument), rows in id order inside each group.
    std::vector<int> nseg(n);
    for (int i = 0; i < n; i++) {
        const int nd = split[i] - rp[i];
        nseg[i] = std::min(kMaxSeg, std::max(1, div_up(nd, segE)));   // longer segments past kMaxSeg
    }
    std::vector<int4> recs;
    std::vector<int> key;    // 2 (level - 1) + (0: later segment, 1: row or segment 0)
    std::vector<int> seg_off(n, 0);
    std::vector<int> scol;   // rows of several segments: columns by level, highest first
    int nsegsum = 0;
    for (int i = 0; i < n; i++) {
        const int ns = nseg[i];
        if (ns >= 65536) return set_error(BL_EINVAL, "Barnes-Hut sweep: row too long");
        int e0 = rp[i], e1 = split[i];
        if (ns > 1) {
            seg_off[i] = nsegsum;
            nsegsum += ns;
            const size_t base = scol.size();
            scol.insert(scol.end(), ci + e0, ci + e1);
            std::sort(scol.begin() + base, scol.end(), [&](int u, int v) {
                return level[u] != level[v] ? level[u] > level[v] : u < v;
            });
            if (scol.size() > (size_t)0x7fffffff)
                return set_error(BL_EINVAL, "Barnes-Hut sweep: too many edges in long rows");
            e1 = (int)scol.size();
            e0 = (int)base;
        }
        for (int q = 0; q < ns; q++) {
            const int a0 = e0 + (int)((int64_t)(e1 - e0) * q / ns);
            const int a1 = e0 + (int)((int64_t)(e1 - e0) * (q + 1) / ns);
            recs.push_back(make_int4(i, a0, a1, q | (ns << 16)));
            key.push_back(q > 0 ? 2 * level[scol[a0]] : 2 * (level[i] - 1) + 1);
        }
    }
    std::vector<int> kstart(2 * nlev + 1, 0);
    for (int k : key) kstart[k + 1]++;
    for (int k = 0; k < 2 * nlev; k++) kstart[k + 1] += kstart[k];
    std::vector<int> lvl_ptr(nlev + 1, 0);   // levels 1..nlev -> slots 0..nlev-1
    for (int l = 0; l <= nlev; l++) lvl_ptr[l] = kstart[2 * l];
    std::vector<int4> tasks(recs.size());
    for (size_t t = 0; t < recs.size(); t++) tasks[kstart[key[t]]++] = recs[t];
    const Allocator& al = L->alloc;
    auto up = [&](DevBuf& d, const void* h, size_t bytes) -> bl_status {
        BL_TRY(d.ensure(al, std::max<size_t>(bytes, 16)));
        if (bytes) BL_CUDA_TRY(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, st));
        return BL_OK;
    };
    BL_TRY(up(s->split, split.data(), split.size() * 4));
    BL_TRY(up(s->bigrows, bigrows.data(), bigrows.size() * 4));
    BL_TRY(up(s->midrows, midrows.data(), midrows.size() * 4));
    BL_TRY(up(s->lvl_ptr, lvl_ptr.data(), lvl_ptr.size() * 4));
    BL_TRY(up(s->tasks, tasks.data(), tasks.size() * sizeof(int4)));
    BL_TRY(up(s->seg_off, seg_off.data(), seg_off.size() * 4));
    BL_TRY(up(s->scol, scol.data(), scol.size() * 4));
    BL_TRY(s->seg_sum.ensure(al, (size_t)std::max(nsegsum, 1) * sizeof(float2)));

    BL_TRY(s->e_row.ensure(al, (size_t)n * 8));
    BL_TRY(s->epart.ensure(al, 1024 * 8));
    BL_TRY(s->old.ensure(al, (size_t)n * sizeof(float2)));
    BL_TRY(s->corr.ensure(al, (size_t)n * sizeof(float2)));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    s->nbig = (int)bigrows.size();
    s->nmid = (int)midrows.size();
    s->nlevels = nlev;
    s->plan_bs = BS;
    s->plan_seg = segE;
    s->lvl0_rows = nlev > 0 ? lvl_ptr[1] : 0;
    s->ntasks = (int64_t)tasks.size();
    s->nsegsum = nsegsum;
    return BL_OK;
}

// Phase timing (bl_set_phase_timing): per iteration, events around each phase.
// Main stream: 0 start, 1 Morton codes done, 2 sort done, 3 tree done, 4 walk
// done, 5 edge pass joined (sweep starts), 6 sweep done, 7 energy done; side
// stream: 8 edge pass starts, 9 edge pass done.
constexpr int kPhaseEvents = 10;
struct PhaseEvents {
    std::vector<cudaEvent_t> ev;
    ~PhaseEvents() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    cudaError_t create(int iters) {
        ev.assign((size_t)iters * kPhaseEvents, nullptr);
        for (cudaEvent_t& e : ev) {
            const cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    }
    cudaEvent_t* at(int t) { return ev.empty() ? nullptr : ev.data() + (size_t)t * kPhaseEvents; }
};

bl_status bh_run(bl_layout* L, int iters, int BS, float theta, cudaStream_t caller, bool sync) {
    L->carry_key = 0;   // the exact engine's carried sums do not follow these moves
    BL_TRY(bh_ensure(L));
    BL_TRY(bh_plan(L, BS, caller));
    BHState* s = L->bh;
    const int n = L->g->n;
    BL_TRY(L->pos2.ensure(L->alloc, (size_t)n * sizeof(float2)));
    BL_TRY(L->energy.ensure(L->alloc, (size_t)std::max(iters, 1) * sizeof(double)));
    double step = 1.0;
    for (int64_t k = 0; k < L->t; k++) step *= 0.999;
    int per_sm = 3;   // sweep CTAs per SM (measured best on R-MAT 20); BL_BH_SWEEP_CTAS overrides it
    int occ = 0;
    BL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dataflow_sweep_kernel, kSweepThreads, 0));
    if (const char* e = std::getenv("BL_BH_SWEEP_CTAS")) per_sm = std::max(1, std::atoi(e));
    const int G = std::max(1, std::min(occ, per_sm)) * device_sm_count();
    const int nep = std::min(1024, div_up(n, 1024));
    // st: the stream of the iteration's critical path, forked from the caller's
    cudaStream_t st = s->hi;
    BL_CUDA_TRY(cudaEventRecord(s->ev_in, caller));
    BL_CUDA_TRY(cudaStreamWaitEvent(st, s->ev_in, 0));
    PhaseEvents pe;
    if (L->phase_timing && sync) BL_CUDA_TRY(pe.create(iters));
    auto mark = [&](int t, int q, cudaStream_t on) -> cudaError_t {
        cudaEvent_t* e = pe.at(t);
        return e ? cudaEventRecord(e[q], on) : cudaSuccess;
    };
    for (int t = 0; t < iters; t++) {
        const float2* S = L->pos.as<float2>();
        float2* bnew = L->pos2.as<float2>();
        BL_CUDA_TRY(mark(t, 0, st));
        // side stream: one pass over the edges (attraction from neighbours that
        // have not moved yet, all rows at once, and the neighbour correction of
        // the tree repulsion) and the sweep's resets; it needs only S and the
        // graph, so it runs while the tree of S is built and walked
        const int rn = L->prm.repulse_neighbors;
        const int am = model_exponent(L->prm.energy_model);
        BL_CUDA_TRY(cudaEventRecord(s->ev_fork, st));
        BL_CUDA_TRY(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
        BL_CUDA_TRY(mark(t, 8, s->side));
        edge_pass_kernel<<<div_up((int64_t)n * 8, 256), 256, 0, s->side>>>(
            L->g->rowptr.as<int>(), L->g->colids.as<int>(), s->split.as<int>(), S, n, 1.0f / L->prm.K, am,
            rn, s->old.as<float2>(), s->corr.as<float2>());
        if (s->nmid > 0)
            edge_pass_mid_kernel<<<div_up((int64_t)s->nmid * 32, 256), 256, 0, s->side>>>(
                L->g->rowptr.as<int>(), L->g->colids.as<int>(), s->split.as<int>(), S, s->midrows.as<int>(),
                s->nmid, 1.0f / L->prm.K, am, rn, s->old.as<float2>(), s->corr.as<float2>());
        if (s->nbig > 0)
            edge_pass_big_kernel<<<s->nbig, 1024, 0, s->side>>>(
                L->g->rowptr.as<int>(), L->g->colids.as<int>(), s->split.as<int>(), S, s->bigrows.as<int>(),
                1.0f / L->prm.K, am, rn, s->old.as<float2>(), s->corr.as<float2>());
        BL_CUDA_TRY(mark(t, 9, s->side));
        if (s->nsegsum > 0)   // every segment slot unset
            BL_CUDA_TRY(cudaMemsetAsync(s->seg_sum.p, 0xFF, (size_t)s->nsegsum * sizeof(float2), s->side));
        BL_CUDA_TRY(cudaMemsetAsync(bnew, 0xFF, (size_t)n * sizeof(float2), s->side));   // every slot kUnset
        BL_CUDA_TRY(cudaGetLastError());
        BL_CUDA_TRY(cudaEventRecord(s->ev_join, s->side));
        // main stream: the tree of S and its walk
        BL_TRY(bh_build(L, S, st, pe.at(t) ? pe.at(t) + 1 : nullptr));
        BL_CUDA_TRY(mark(t, 3, st));
        BL_TRY(bh_repulsion(L, S, theta, st, false));
        BL_CUDA_TRY(mark(t, 4, st));
        BL_TRY(layout_reset_sync_words(L, st));
        SweepArgs a{};
        a.rowptr = L->g->rowptr.as<int>();
        a.colids = L->g->colids.as<int>();
        a.scol = s->scol.as<int>();
        a.bold = S;
        a.bnew = bnew;
        a.rep = s->rep.as<float2>();
        a.corr = s->corr.as<float2>();
        a.old = s->old.as<float2>();
        a.lvl_ptr = s->lvl_ptr.as<int>();
        a.tasks = s->tasks.as<int4>();
        a.seg_off = s->seg_off.as<int>();
        a.seg_sum = s->seg_sum.as<float2>();
        a.e_row = s->e_row.as<double>();
        a.status = static_cast<int*>(L->status.p);
        a.nlevels = s->nlevels;
        a.invK = 1.0f / L->prm.K;
        a.am = am;
        a.negRK2 = -L->prm.R * L->prm.K * L->prm.K;
        a.stepf = (float)step;
        a.trace = nullptr;
        a.ttrace = nullptr;
        if (L->trace_steps > 0 && t == iters - 1) {   // trace the last iteration's sweep
            const int64_t ntasks = s->ntasks;
            const bool per_task = L->trace_steps >= 2;
            const size_t cnt = (size_t)(s->nlevels + 1) + (per_task ? 3 * (size_t)ntasks : 0);
            const size_t tb = cnt * sizeof(unsigned long long);
            BL_TRY(L->trace.ensure(L->alloc, tb));
            BL_CUDA_TRY(cudaMemsetAsync(L->trace.p, 0, tb, st));
            a.trace = L->trace.as<unsigned long long>();
            if (per_task) a.ttrace = a.trace + (s->nlevels + 1);
            L->trace_count = (int64_t)cnt;
        }
        a.first_level = s->nlevels > 0 ? 1 : 0;
        BL_CUDA_TRY(cudaStreamWaitEvent(st, s->ev_join, 0));
        BL_CUDA_TRY(mark(t, 5, st));
        if (a.first_level == 1) {
            const int n0 = s->lvl0_rows;
            level0_kernel<<<std::max(1, std::min(div_up(n0, 256), 8 * device_sm_count())), 256, 0, st>>>(a);
        }
        void* args[] = {&a};
        BL_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)dataflow_sweep_kernel, dim3(G),
                                                dim3(kSweepThreads), args, 0, st));
        BL_CUDA_TRY(mark(t, 6, st));
        row_energy_kernel<<<nep, 256, 0, st>>>(s->e_row.as<double>(), n, s->epart.as<double>());
        energy_parts_kernel<<<1, 32, 0, st>>>(s->epart.as<double>(), nep, L->energy.as<double>() + t);
        BL_CUDA_TRY(cudaGetLastError());
        BL_CUDA_TRY(mark(t, 7, st));
        std::swap(L->pos, L->pos2);
        step *= 0.999;
    }
    // the caller's stream continues after the iterations
    BL_CUDA_TRY(cudaEventRecord(s->ev_out, st));
    BL_CUDA_TRY(cudaStreamWaitEvent(caller, s->ev_out, 0));
    if (!sync) return BL_OK;
    // interaction counts of the last iteration
    unsigned long long c[3] = {0, 0, 0};
    int nodes = 0;
    BL_CUDA_TRY(cudaMemcpyAsync(c, s->walkcnt.p, sizeof(c), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaMemcpyAsync(&nodes, s->cnt.as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    L->far_nodes = (double)c[0];
    L->near_pairs = (double)c[1];
    if (pe.at(0)) {   // phase times of this run, summed over its iterations
        static const int kFrom[kPhaseSlots] = {0, 1, 2, 3, 4, 5, 6, 8, 0};
        static const int kTo[kPhaseSlots] = {1, 2, 3, 4, 5, 6, 7, 9, 7};
        double acc[kPhaseSlots] = {};
        for (int t = 0; t < iters; t++)
            for (int q = 0; q < kPhaseSlots; q++) {
                float ms = 0.f;
                BL_CUDA_TRY(cudaEventElapsedTime(&ms, pe.at(t)[kFrom[q]], pe.at(t)[kTo[q]]));
                acc[q] += ms;
            }
        for (int q = 0; q < kPhaseSlots; q++) L->phase_ms[q] = acc[q];
        L->phase_nodes = nodes;
        L->phase_visits = (double)c[2];
        L->phase_iters = iters;
    }
    return BL_OK;
}

bl_status bh_debug_forces(bl_layout* L, float theta, float2* f_out, cudaStream_t st) {
    BL_TRY(bh_ensure(L));
    const int n = L->g->n;
    const float2* S = L->pos.as<float2>();
    BL_TRY(bh_build(L, S, st));
    BL_TRY(bh_repulsion(L, S, theta, st));
    bh_snapshot_force_kernel<<<div_up((int64_t)n * 32, 256), 256, 0, st>>>(
        L->g->rowptr.as<int>(), L->g->colids.as<int>(), S, n, L->bh->rep.as<float2>(), 1.0f / L->prm.K,
        model_exponent(L->prm.energy_model), -L->prm.R * L->prm.K * L->prm.K, f_out);
    BL_CUDA_TRY(cudaGetLastError());
    unsigned long long c[2] = {0, 0};
    BL_CUDA_TRY(cudaMemcpyAsync(c, L->bh->walkcnt.p, sizeof(c), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    L->far_nodes = (double)c[0];
    L->near_pairs = (double)c[1];
    return BL_OK;
}

bl_status bh_debug_counts(bl_layout* L, float theta, int2* qcounts, cudaStream_t st) {
    BL_TRY(bh_ensure(L));
    const float2* S = L->pos.as<float2>();
    BL_TRY(bh_build(L, S, st));
    BL_TRY(bh_repulsion(L, S, theta, st, false, qcounts));
    return BL_OK;
}

bl_status bh_debug_tree(bl_layout* L, uint32_t* codes, int32_t* perm, int32_t* first, int32_t* count,
                        int32_t* level, int32_t* skip, float* sumx, float* sumy, int64_t cap,
                        int64_t* nnodes, float* box, cudaStream_t st) {
    BL_TRY(bh_ensure(L));
    BHState* s = L->bh;
    const int n = L->g->n;
    BL_TRY(bh_build(L, L->pos.as<float2>(), st));
    int M = 0;
    BL_CUDA_TRY(cudaMemcpyAsync(&M, s->cnt.as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    *nnodes = M;
    if (box) {
        float b[3];
        BL_CUDA_TRY(cudaMemcpy(b, s->box.p, sizeof(b), cudaMemcpyDeviceToHost));
        box[0] = b[0];
        box[1] = b[1];
        box[2] = b[2];
    }
    if (codes) BL_CUDA_TRY(cudaMemcpy(codes, s->keys0.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
    if (perm) BL_CUDA_TRY(cudaMemcpy(perm, s->vals0.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
    if (M > cap) return set_error(BL_EINVAL, "bl_debug_bh_tree: node arrays too small");
    if (first) BL_CUDA_TRY(cudaMemcpy(first, s->nd_first.p, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (count) BL_CUDA_TRY(cudaMemcpy(count, s->nd_count.p, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (level) BL_CUDA_TRY(cudaMemcpy(level, s->nd_level.p, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (skip) BL_CUDA_TRY(cudaMemcpy(skip, s->nd_skip.p, (size_t)M * 4, cudaMemcpyDeviceToHost));
    if (sumx || sumy) {
        std::vector<float2> sm((size_t)M);
        BL_CUDA_TRY(cudaMemcpy(sm.data(), s->nd_sum.p, (size_t)M * sizeof(float2), cudaMemcpyDeviceToHost));
        for (int v = 0; v < M; v++) {
            if (sumx) sumx[v] = sm[v].x;
            if (sumy) sumy[v] = sm[v].y;
        }
    }
    return BL_OK;
}

}  // namespace bl
