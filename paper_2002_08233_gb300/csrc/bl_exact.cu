// Exact-mode BatchLayout engine (Section 2.2, Section 3.3, Algorithm 2).
//
// Column formulation of the minibatch sweep. Iteration t visits batches
// k = 0..B-1 in order; batch k's force ct_i needs, for every other batch c, the
// positions of c as they are when k is processed: updated this iteration if
// c < k, from the previous iteration if c >= k. So the moment batch c is updated,
// its new positions are exactly what every row needs from c until c moves again:
// they form a column tile that every row adds once. A prologue adds, for each
// row, the columns c >= batch(row) at the starting positions; after that, every
// row receives every column exactly once per iteration, so a launch of T
// iterations evaluates exactly T*n^2 pairs.
//
// Launch shape: one persistent cooperative CTA per SM; row i belongs to CTA
// (i mod G), so each minibatch's rows are spread over all CTAs (about BS/G
// "critical" rows per CTA and batch). Inside a CTA the warps specialise:
//   - the bulk warps keep their rows' positions and repulsion sums (optionally
//     Kahan-compensated) in registers and only run the pair loop: at step
//     s = (t, k) they add the column tile of batch k-1 to every row that still
//     needs it; with one row per thread, each row's sum is kept in two halves
//     (the first and second half of every tile) so that the host can spread the
//     work evenly over the SM's four sub-partitions (see plan_pieces);
//   - one control warp runs the step chain: wait until all CTAs have published
//     batch k-1 (monotonic counter, bounded spin), copy that column tile into
//     shared memory, then for the CTA's rows of batch k add the tile, add the CSR
//     attraction and take back the neighbour repulsion, move each vertex by
//     Step * ct/|ct| (Algorithm 2's update), publish and arrive on the counter;
//   - the last bulk warp stages the next rows' neighbour positions with cp.async
//     (ids two steps ahead, positions one step ahead) and, once they have landed,
//     sums those rows' CSR terms over every neighbour but the ones in the batch
//     moving now; the control warp adds just those from the next tile.
// The roles meet at named barriers (tile ready / bulk done / CSR sums ready), so
// the latency of the step chain hides behind the bulk warps' pair work. The pair
// loop uses packed FP32x2 arithmetic (two columns per instruction) and one SFU
// reciprocal per pair.
//
// Positions are double-buffered by iteration parity: iteration t writes
// buf[(t+1)&1] and reads not-yet-moved vertices from buf[t&1]. A CTA can lag
// the others by at most one step, so nothing still to be read is overwritten.

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "bl_internal.cuh"

namespace bl {

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Column tiles are stored in pairs: float4 q = (x_2q, x_2q+1, y_2q, y_2q+1).
// The pair loop: rows m in [mlo, mhi) of the thread against the tile's first
// 2*np columns; (XI, YI) hold each row's coordinates twice, (AX, AY) two partial
// sums per row. mlo/mhi are warp-uniform, so skipped rows cost no SFU work.
template <int RPT>
__device__ __forceinline__ void tile_pairs2(const float4* __restrict__ tile, int np, int mlo,
                                            int mhi, const f32x2 (&XI)[RPT],
                                            const f32x2 (&YI)[RPT], f32x2 (&AX)[RPT],
                                            f32x2 (&AY)[RPT]) {
    const f32x2 E = pk2(BL_EPS2, BL_EPS2);
    auto pair2 = [&](const f32x2 X, const f32x2 Y, int m) {
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
    };
    if (mlo == 0 && mhi == RPT) {   // every row: no predicate in the loop
#pragma unroll 16
        for (int q = 0; q < np; q++) {
            const float4 p = tile[q];
            const f32x2 X = pk2(p.x, p.y), Y = pk2(p.z, p.w);
#pragma unroll
            for (int m = 0; m < RPT; m++) pair2(X, Y, m);
        }
        return;
    }
#pragma unroll 4
    for (int q = 0; q < np; q++) {
        const float4 p = tile[q];
        const f32x2 X = pk2(p.x, p.y), Y = pk2(p.z, p.w);
#pragma unroll
        for (int m = 0; m < RPT; m++)
            if (m >= mlo && m < mhi) pair2(X, Y, m);
    }
}

// warp-uniform range [mlo, mhi) covering every m flagged in need[] by any lane
template <int RPT>
__device__ __forceinline__ void need_range(const bool (&need)[RPT], int& mlo, int& mhi) {
    if (RPT == 1) {   // one vote
        const bool any = __any_sync(0xffffffffu, need[0]);
        mlo = any ? 0 : 1;
        mhi = any ? 1 : 0;
        return;
    }
    int lo = RPT, hi = 0;
#pragma unroll
    for (int m = 0; m < RPT; m++)
        if (need[m]) {
            lo = min(lo, m);
            hi = m + 1;
        }
    mlo = (int)__reduce_min_sync(0xffffffffu, (unsigned)lo);
    mhi = (int)__reduce_max_sync(0xffffffffu, (unsigned)hi);
}

// Shared-memory carve-up (bytes); the host sizes the launch with the same code.
struct EngineSmem {
    int tile, pos, rpl, rpe, crep, off, cid, nbr, pre, prel, ctl, total;
    __host__ __device__ EngineSmem(int BS, int nloc, int CR, int CAP, int NW) {
        const int TQ = (BS + 1) / 2;
        tile = 0;                                        // 2 x TQ float4: column tiles
        pos = tile + 2 * TQ * 16;                        // nloc float2: local positions
        rpl = pos + ((nloc * 8 + 15) / 16) * 16;         // nloc int: rowptr[i]
        rpe = rpl + ((nloc * 4 + 15) / 16) * 16;         // nloc int: rowptr[i+1]
        crep = rpe + ((nloc * 4 + 15) / 16) * 16;        // 2 steps x 2 halves x CR float2: bulk sums
        off = crep + ((4 * CR * 8 + 15) / 16) * 16;      // 3 x (CR+1) int: edge offsets
        cid = off + ((3 * (CR + 1) * 4 + 15) / 16) * 16; // 3 x CAP int: staged column ids
        nbr = cid + 3 * CAP * 4;                         // 2 x CAP float2: staged positions
        pre = nbr + 2 * CAP * 8;                         // 2 x CR float4: CSR sums without the last batch
        prel = pre + 2 * CR * 16;                        // 2 x CR int: edges into the last batch
        ctl = prel + ((2 * CR * 4 + 15) / 16) * 16;      // control words
        total = ctl + 64;
    }
};

// critical rows of batch k in CTA `rank`: local indices [lo, hi)
__device__ __forceinline__ void crit_range(int k, int BS, int n, int rank, int G, int& lo,
                                           int& hi) {
    const int a = k * BS - rank;
    const int b = min((k + 1) * BS, n) - rank;
    lo = a > 0 ? (a + G - 1) / G : 0;
    hi = b > 0 ? (b + G - 1) / G : 0;
    if (hi < lo) hi = lo;
}

// Named CTA barriers between the warp roles. The non-aligned forms count
// threads, and each call site first reconverges its warp.
__device__ __forceinline__ void bar_sync_n(int id, int count) {
    __syncwarp();
    asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int count) {
    __syncwarp();
    asm volatile("barrier.cta.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
constexpr int kBarTile = 1;   // control warp -> bulk warps: tile of step s ready
constexpr int kBarDone = 2;   // bulk warps -> control warp: step s finished
constexpr int kBarPre = 3;    // staging warp -> control warp: CSR sums of step s+1 ready
constexpr int kCritLanes = 4; // critical rows the control warp finishes together

// phase timestamp (global timer, ns) of step s, slot q, when tracing
__device__ __forceinline__ void trace_mark(const ExactTask& tk, int rank, int s, int q) {
    if (tk.trace != nullptr && s < tk.trace_steps)
        tk.trace[((size_t)rank * tk.trace_steps + s) * kTraceSlots + q] = global_ns();
}

// column q of a paired tile
__device__ __forceinline__ float2 tile_col(const float4* tile, int q) {
    const float4 p = tile[q >> 1];
    return (q & 1) ? make_float2(p.y, p.w) : make_float2(p.x, p.z);
}

template <int RPT, int TB>
__global__ void __launch_bounds__(TB + 32, 1) exact_grid_kernel(ExactTask tk, ExactParams prm) {
    constexpr int T = TB + 32;
    constexpr int NW = TB / 32;   // bulk warps
    extern __shared__ __align__(16) unsigned char smem[];
    const int G = gridDim.x, rank = blockIdx.x;
    const int n = tk.n, BS = tk.BS, B = tk.B;
    const int CR = tk.crit_cap, CAP = tk.nbr_cap;
    const int nloc = n > rank ? (n - rank + G - 1) / G : 0;
    const EngineSmem L(BS, (n + G - 1) / G, CR, CAP, NW);
    const int TQ = (BS + 1) / 2;
    float4* s_tile = reinterpret_cast<float4*>(smem + L.tile);
    float2* s_pos = reinterpret_cast<float2*>(smem + L.pos);
    int* s_rpl = reinterpret_cast<int*>(smem + L.rpl);
    int* s_rpe = reinterpret_cast<int*>(smem + L.rpe);
    float2* s_crep = reinterpret_cast<float2*>(smem + L.crep);
    int* s_off = reinterpret_cast<int*>(smem + L.off);
    int* s_cid = reinterpret_cast<int*>(smem + L.cid);
    float2* s_nbr = reinterpret_cast<float2*>(smem + L.nbr);
    float4* s_pre = reinterpret_cast<float4*>(smem + L.pre);
    int* s_prel = reinterpret_cast<int*>(smem + L.prel);
    volatile int* s_ctl = reinterpret_cast<volatile int*>(smem + L.ctl);

    const int tid = threadIdx.x, lane = tid & 31;
    const bool is_ctl = tid < 32;
    const int tb = tid - 32;                 // bulk thread index
    const int wb = tb >> 5;                  // bulk warp index
    const bool is_stager = wb == NW - 1;     // bulk warp that stages neighbours
    const bool snapshot = tk.iters == 0;
    const bool rn = prm.repulse_neighbors != 0;
    const float invK = prm.invK, negRK2 = prm.negRK2;
    const int am = prm.am;
    const bool kahan = prm.kahan != 0;
    float2* const buf0 = tk.pos;
    float2* const buf1 = tk.pos_alt;

    // ---- bulk state: blocks of 32 consecutive local rows per warp (so a warp's rows
    //      share few minibatches and whole warps skip columns they do not need).
    //      One row per thread: every row's repulsion is kept as two sums, over the
    //      first and the second half of every column tile, and a warp's piece (set by
    //      the host) is a whole block (both halves), one half of a block, or a block
    //      of at most 16 rows folded onto the warp (lanes 0-15 the first half, lanes
    //      16-31 the second), so that the pieces spread the work evenly over the four
    //      sub-partitions (hardware warp w runs on sub-partition w % 4), the control
    //      warp's getting less. Several rows per thread: a block per warp and turn,
    //      the control warp's sub-partition served last, one sum per row. -----------------
    const int wslot = (wb + 1) % 4 == 0 ? (NW - NW / 4) + (wb + 1) / 4 - 1
                                         : wb - (wb + 1) / 4;
    const int pcode = RPT == 1 && !is_ctl ? tk.piece[wb] : 0;
    const bool pfold = (pcode >> 18) & 1;
    // halves this thread sums for its row (bit 0: first, bit 1: second)
    const int hm = RPT > 1 ? 1 : (pfold ? (lane < 16 ? 1 : 2) : ((pcode >> 16) & 3));
    f32x2 XI[RPT], YI[RPT];
    float sx[2][RPT], sy[2][RPT], cx[2][RPT], cy[2][RPT];
    int bi[RPT], lrow[RPT], cslot[RPT];   // batch, local row, slot among its batch's critical rows
#pragma unroll
    for (int m = 0; m < RPT; m++) {
        const int li = RPT == 1 ? 32 * (pcode & 0xFFFF) + (pfold ? (lane & 15) : lane)
                                : lane + 32 * (wslot + NW * m);
        const bool v = !is_ctl && hm != 0 && li < nloc;
        const int i = rank + G * li;
        const float2 p = v ? __ldcg(&buf0[i]) : make_float2(0.f, 0.f);
        XI[m] = pk2(p.x, p.x);
        YI[m] = pk2(p.y, p.y);
#pragma unroll
        for (int h = 0; h < 2; h++) sx[h][m] = sy[h][m] = cx[h][m] = cy[h][m] = 0.f;
        bi[m] = v ? i / BS : -1;
        lrow[m] = li;
        int lo = 0, hi = 0;
        if (v) crit_range(bi[m], BS, n, rank, G, lo, hi);
        cslot[m] = li - lo;
    }
    for (int li = tid; li < nloc; li += T) {
        const int i = rank + G * li;
        s_pos[li] = __ldcg(&buf0[i]);
        s_rpl[li] = __ldg(&tk.rowptr[i]);
        s_rpe[li] = __ldg(&tk.rowptr[i + 1]);
    }
    if (tid == 0) s_ctl[0] = 0;

    // s += v into a row's sum (compensated across tiles when kahan)
    auto acc = [&](float& sum, float& comp, float v) {
        if (kahan)
            kahan_add(sum, comp, v);
        else
            sum += v;
    };
    // pair loop + tail + Kahan for the flagged rows against a paired tile of nc columns
    auto add_tile = [&](const float4* tile, int nc, const bool (&need)[RPT]) {
        if constexpr (RPT == 1) {
            // half 0: column pairs [0, hp); half 1: [hp, np) and an odd last column
            if (!__any_sync(0xffffffffu, need[0])) return;   // warp-uniform
            const int np = nc >> 1, hp = np >> 1;
            float xi, yi, dummy;
            upk2(XI[0], xi, dummy);
            upk2(YI[0], yi, dummy);
            // the sum of column pairs [q0, q0 + len) (+ the odd column for half 1)
            auto half_sum = [&](bool second, const float4* t0, int len, float& vx, float& vy) {
                f32x2 AX[1] = {pk2(0.f, 0.f)}, AY[1] = {pk2(0.f, 0.f)};
                tile_pairs2<1>(t0, len, 0, 1, XI, YI, AX, AY);
                float a0, a1, b0, b1;
                upk2(AX[0], a0, a1);
                upk2(AY[0], b0, b1);
                vx = a0 + a1;
                vy = b0 + b1;
                if (second && (nc & 1)) {
                    const float2 pc = tile_col(tile, nc - 1);
                    rep_pair(xi, yi, pc.x, pc.y, vx, vy);
                }
            };
            float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f;
            if (pfold) {   // half-warps on the two halves (the same length unless np is odd)
                const bool second = lane >= 16;
                f32x2 AX[1] = {pk2(0.f, 0.f)}, AY[1] = {pk2(0.f, 0.f)};
                tile_pairs2<1>(tile + (second ? hp : 0), hp, 0, 1, XI, YI, AX, AY);
                if (second && (np & 1)) tile_pairs2<1>(tile + 2 * hp, 1, 0, 1, XI, YI, AX, AY);
                float a0, a1, b0, b1;
                upk2(AX[0], a0, a1);
                upk2(AY[0], b0, b1);
                float vx = a0 + a1, vy = b0 + b1;
                if (second && (nc & 1)) {
                    const float2 pc = tile_col(tile, nc - 1);
                    rep_pair(xi, yi, pc.x, pc.y, vx, vy);
                }
                if (second) {
                    ax1 = vx;
                    ay1 = vy;
                } else {
                    ax0 = vx;
                    ay0 = vy;
                }
            } else {
                if (hm & 1) half_sum(false, tile, hp, ax0, ay0);
                if (hm & 2) half_sum(true, tile + hp, np - hp, ax1, ay1);
            }
            if (need[0]) {
                if (hm & 1) {
                    acc(sx[0][0], cx[0][0], ax0);
                    acc(sy[0][0], cy[0][0], ay0);
                }
                if (hm & 2) {
                    acc(sx[1][0], cx[1][0], ax1);
                    acc(sy[1][0], cy[1][0], ay1);
                }
            }
        } else {
            int mlo, mhi;
            need_range<RPT>(need, mlo, mhi);
            if (mlo >= mhi) return;
            f32x2 AX[RPT], AY[RPT];
#pragma unroll
            for (int m = 0; m < RPT; m++) AX[m] = AY[m] = pk2(0.f, 0.f);
            tile_pairs2<RPT>(tile, nc >> 1, mlo, mhi, XI, YI, AX, AY);
#pragma unroll
            for (int m = 0; m < RPT; m++) {
                float a0, a1, b0, b1, xi, yi, dummy;
                upk2(AX[m], a0, a1);
                upk2(AY[m], b0, b1);
                upk2(XI[m], xi, dummy);
                upk2(YI[m], yi, dummy);
                float ax = a0 + a1, ay = b0 + b1;
                if (nc & 1) {
                    const float2 pc = tile_col(tile, nc - 1);
                    rep_pair(xi, yi, pc.x, pc.y, ax, ay);
                }
                if (need[m]) {
                    acc(sx[0][m], cx[0][m], ax);
                    acc(sy[0][m], cy[0][m], ay);
                }
            }
        }
    };
    // tile of column c into buffer dst (paired layout), threads [t0, t0+nt) copying
    auto copy_tile = [&](float4* dst, const float2* src, int nc, int t, int nt) {
        for (int q = t; q < (nc + 1) / 2; q += nt) {
            const float2 a = __ldcg(&src[2 * q]);
            const float2 b = (2 * q + 1 < nc) ? __ldcg(&src[2 * q + 1]) : make_float2(0.f, 0.f);
            dst[q] = make_float4(a.x, b.x, a.y, b.y);
        }
    };

    // A row's (half-)sums in the carry buffer: slot (rank * ceil(n/G) + local row) * 2
    // + half, {sx, sy, cx, cy}. Each (row, half) is summed by exactly one thread.
    const size_t carry_base = (size_t)rank * (size_t)((n + G - 1) / G);
    auto carry_rows = [&](bool store) {
#pragma unroll
        for (int m = 0; m < RPT; m++) {
            if (bi[m] < 0) continue;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                if (!(hm & (1 << h))) continue;
                float4* c = tk.carry + (carry_base + (size_t)lrow[m]) * 2 + h;
                if (store) {
                    *c = make_float4(sx[h][m], sy[h][m], cx[h][m], cy[h][m]);
                } else {
                    const float4 v = *c;
                    sx[h][m] = v.x;
                    sy[h][m] = v.y;
                    cx[h][m] = v.z;
                    cy[h][m] = v.w;
                }
            }
        }
    };

    // ---- prologue: columns c >= batch(row), c < B-1, at the starting positions
    //      (every column in snapshot mode); the next tile is fetched into registers
    //      while the bulk warps add the current one. A launch that continues the
    //      previous one's run loads these sums from the carry buffer instead, where
    //      that launch left them (the same sums: the same tiles, at the same
    //      positions, added in the same order) ----------------------------------------
    if (!snapshot && tk.carry_in) {
        if (!is_ctl) carry_rows(false);
        __syncthreads();
    } else {
        const bool one_each = TQ <= T;
        float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
        auto fetch = [&](int c) {
            const int nc = min(BS, n - c * BS);
            const float2* src = buf0 + (size_t)c * BS;
            if (tid < (nc + 1) / 2) {
                const float2 a = __ldcg(&src[2 * tid]);
                const float2 b = (2 * tid + 1 < nc) ? __ldcg(&src[2 * tid + 1]) : make_float2(0.f, 0.f);
                nxt = make_float4(a.x, b.x, a.y, b.y);
            }
        };
        if (one_each) fetch(0);
        for (int c = 0; c < B; c++) {
            const int nc = min(BS, n - c * BS);
            float4* tile = s_tile + (size_t)(c & 1) * TQ;
            if (one_each) {
                if (tid < (nc + 1) / 2) tile[tid] = nxt;
                __syncthreads();
                if (c + 1 < B) fetch(c + 1);
            } else {
                copy_tile(tile, buf0 + (size_t)c * BS, nc, tid, T);
                __syncthreads();
            }
            if (!is_ctl) {
                bool need[RPT];
#pragma unroll
                // the last batch's tile is added at step 0 instead, as it is when a
                // launch continues across an iteration boundary, so that results do
                // not depend on how the iterations are split into launches
                for (int m = 0; m < RPT; m++)
                    need[m] = bi[m] >= 0 && (snapshot || (bi[m] <= c && c < B - 1));
                add_tile(tile, nc, need);
            }
            if (!one_each) __syncthreads();
        }
        __syncthreads();
    }

    // bulk: post the sums of the rows of batch kk into crep (half h at
    // crep[h * CR + slot]; one sum per row: the second half is zero) and restart
    // them (a row's slot among its batch's critical rows is fixed: cslot, set above)
    auto post_rows = [&](int kk, float2* crep) {
#pragma unroll
        for (int m = 0; m < RPT; m++) {
            if (bi[m] == kk) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    if (hm & (1 << h)) {
                        crep[h * CR + cslot[m]] = make_float2(sx[h][m] - cx[h][m], sy[h][m] - cy[h][m]);
                        sx[h][m] = sy[h][m] = cx[h][m] = cy[h][m] = 0.f;
                    }
                }
                if (RPT > 1) crep[CR + cslot[m]] = make_float2(0.f, 0.f);
            }
        }
    };

    // ---- neighbour staging (one warp) -----------------------------------------------
    // column ids of the edges of batch kk's rows into id slot `slot` (async)
    auto stage_ids = [&](int kk, int slot) {
        int lo, hi;
        crit_range(kk, BS, n, rank, G, lo, hi);
        int* off = s_off + slot * (CR + 1);
        int* cid = s_cid + (size_t)slot * CAP;
        if (lane == 0) {
            int acc = 0;
            for (int c = 0; c < hi - lo; c++) {
                off[c] = acc;
                acc += s_rpe[lo + c] - s_rpl[lo + c];
            }
            off[hi - lo] = acc;
        }
        __syncwarp();
        const int tot = min(off[hi - lo], CAP);
        int c = 0;
        for (int f = lane; f < tot; f += 32) {
            while (off[c + 1] <= f) c++;
            cp_async4(&cid[f], &tk.colids[s_rpl[lo + c] + (f - off[c])]);
        }
        cp_async_commit();
    };
    // positions of those neighbours (ids in `slot`, landed) into position slot
    // `pslot`, as the step of batch kk reads them (bnew/bold: that step's buffers):
    // batch(j) < kk moved in this iteration (bnew), batch(j) >= kk not yet (bold);
    // batch kprev comes from the column tile instead (kprev < 0: no tile)
    auto stage_pos = [&](int kk, int kprev, int slot, int pslot, const float2* bnew,
                         const float2* bold) {
        int lo, hi;
        crit_range(kk, BS, n, rank, G, lo, hi);
        const int* off = s_off + slot * (CR + 1);
        const int* cid = s_cid + (size_t)slot * CAP;
        float2* nbr = s_nbr + (size_t)pslot * CAP;
        const int tot = min(off[hi - lo], CAP);
        for (int f = lane; f < tot; f += 32) {
            const int j = cid[f];
            const int bj = j / BS;
            if (kprev >= 0 && bj == kprev) continue;
            cp_async8(&nbr[f], bj < kk ? bnew + j : bold + j);
        }
        cp_async_commit();
    };
    // The staging warp, once the positions of step s+1 have landed: the CSR sums of
    // batch kk's rows over every neighbour except those in batch kl (the batch the
    // control warp moves at step s, whose positions only the tile of step s+1 has),
    // one row at a time over the whole warp (lanes over the edges in order, then a
    // butterfly), into s_pre[pslot]; s_prel counts each row's edges into batch kl,
    // whose terms the control warp adds at step s+1.
    auto csr_pre = [&](int kk, int kl, int slot, int pslot, const float2* bnew, const float2* bold) {
        int lo, hi;
        crit_range(kk, BS, n, rank, G, lo, hi);
        const int* off = s_off + slot * (CR + 1);
        const int* cid = s_cid + (size_t)slot * CAP;
        const float2* nbr = s_nbr + (size_t)pslot * CAP;
        const int kllo = kl * BS, kln = min(BS, n - kllo);
        for (int c = 0; c < hi - lo; c++) {
            const int li = lo + c;
            const int e0 = s_rpl[li], e1 = s_rpe[li];
            const float2 me = s_pos[li];
            float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
            int late = 0;
            for (int ee = e0 + lane; ee < e1; ee += 32) {
                const int f = off[c] + (ee - e0);
                const int j = f < CAP ? cid[f] : __ldg(&tk.colids[ee]);
                if ((unsigned)(j - kllo) < (unsigned)kln) {
                    late++;
                    continue;
                }
                const float2 pj = f < CAP ? nbr[f] : __ldcg(j < kk * BS ? bnew + j : bold + j);
                edge_terms(me.x, me.y, pj, invK, am, rn, ax, ay, qx, qy);
            }
            ax = warp_sum(ax);
            ay = warp_sum(ay);
            qx = warp_sum(qx);
            qy = warp_sum(qy);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) late += __shfl_xor_sync(0xffffffffu, late, o);
            if (lane == 0) {
                s_pre[pslot * CR + c] = make_float4(ax, ay, qx, qy);
                s_prel[pslot * CR + c] = late;
            }
        }
        __syncwarp();
    };

    // ---- control warp: finish the rows of batch k --------------------------------------
    // Rows kCritLanes at a time. Column kprev: 8 lanes per row over the tile, then a
    // 3-level butterfly inside each 8-lane group. CSR: one lane per row (rows with
    // more than 32 edges: the whole warp). Lane r then moves row r (or records the
    // snapshot force). Returns this lane's energy contribution.
    int cur_s = 0;   // step being traced (control warp)
    auto ctl_critical = [&](int k, int kprev, int slot, int pslot, const float4* tile,
                            float stepf, const float2* bnew, const float2* bold,
                            const float2* crep, float2* out, bool pre_ok) -> double {
        int lo, hi;
        crit_range(k, BS, n, rank, G, lo, hi);
        const int* off = s_off + slot * (CR + 1);
        const int* cid = s_cid + (size_t)slot * CAP;
        const float2* nbr = s_nbr + (size_t)pslot * CAP;
        const int kplo = kprev >= 0 ? kprev * BS : 0;
        const int kpn = kprev >= 0 ? min(BS, n - kplo) : 0;
        auto nbr_pos = [&](int c, int ee, int e0) -> float2 {
            const int f = off[c] + (ee - e0);
            const int j = f < CAP ? cid[f] : __ldg(&tk.colids[ee]);
            const unsigned o = (unsigned)(j - kplo);
            if (o < (unsigned)kpn) return tile_col(tile, (int)o);
            if (f < CAP) return nbr[f];
            return __ldcg(j < k * BS ? bnew + j : bold + j);
        };
        double e = 0.0;
        // the staging warp's CSR sums of this step (once per step, rows or not)
        if (pre_ok && !snapshot && cur_s > 0) bar_sync_n(kBarPre, 64);
        for (int c0 = 0; c0 < hi - lo; c0 += kCritLanes) {
            const int nr = min(kCritLanes, hi - lo - c0);
            // column kprev: lane group g = lane / 8 takes row c0 + g
            // W lanes per row: the whole warp shares the column tile among the rows
            const int lw = nr == 1 ? 5 : (nr == 2 ? 4 : 3);
            const int W = 1 << lw;
            const int g = lane >> lw, gl = lane & (W - 1);
            float rx = 0.f, ry = 0.f;
            if (g < nr) {   // column pairs gl, gl + W, ... packed two columns an instruction
                const float2 me = s_pos[lo + c0 + g];
                const f32x2 X0 = pk2(me.x, me.x), Y0 = pk2(me.y, me.y), E = pk2(BL_EPS2, BL_EPS2);
                f32x2 AX = pk2(0.f, 0.f), AY = pk2(0.f, 0.f);
#pragma unroll 4
                for (int q = gl; q < (kpn >> 1); q += W) {
                    const float4 p = tile[q];
                    const f32x2 X = pk2(p.x, p.y), Y = pk2(p.z, p.w);
                    f32x2 dx, dy, d2;
                    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(X), "l"(X0));
                    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(Y), "l"(Y0));
                    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d2) : "l"(dy), "l"(E));
                    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d2) : "l"(dx), "l"(d2));
                    float da, db;
                    upk2(d2, da, db);
                    const f32x2 inv = pk2(rcp_sfu(da), rcp_sfu(db));
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(AX) : "l"(dx), "l"(inv));
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(AY) : "l"(dy), "l"(inv));
                }
                float a0, a1, b0, b1;
                upk2(AX, a0, a1);
                upk2(AY, b0, b1);
                rx = a0 + a1;
                ry = b0 + b1;
                if ((kpn & 1) && gl == 0) {   // an odd last column: the group's first lane
                    const float2 pc = tile_col(tile, kpn - 1);
                    rep_pair(me.x, me.y, pc.x, pc.y, rx, ry);
                }
            }
            for (int o = W >> 1; o > 0; o >>= 1) {
                rx += __shfl_xor_sync(0xffffffffu, rx, o);
                ry += __shfl_xor_sync(0xffffffffu, ry, o);
            }
            if (lane == 0 && c0 == 0 && !snapshot) trace_mark(tk, rank, cur_s, 9);
            // with the staging warp's sums (pre_ok): each row's sum without batch kprev,
            // plus, when it has edges into kprev, their terms from the tile (whole warp)
            float hax = 0.f, hay = 0.f, hqx = 0.f, hqy = 0.f;
            if (pre_ok) {
                for (int r = 0; r < nr; r++) {
                    const int c = c0 + r;
                    float4 v = s_pre[pslot * CR + c];
                    if (s_prel[pslot * CR + c] > 0) {   // warp-uniform
                        const int li = lo + c;
                        const int e0 = s_rpl[li], e1 = s_rpe[li];
                        const float2 me = s_pos[li];
                        float lx = 0.f, ly = 0.f, lqx = 0.f, lqy = 0.f;
                        for (int ee = e0 + lane; ee < e1; ee += 32) {
                            const int f = off[c] + (ee - e0);
                            const int j = f < CAP ? cid[f] : __ldg(&tk.colids[ee]);
                            const unsigned o = (unsigned)(j - kplo);
                            if (o < (unsigned)kpn)
                                edge_terms(me.x, me.y, tile_col(tile, (int)o), invK, am, rn, lx, ly, lqx, lqy);
                        }
                        v.x += warp_sum(lx);
                        v.y += warp_sum(ly);
                        v.z += warp_sum(lqx);
                        v.w += warp_sum(lqy);
                    }
                    if (lane == r) {
                        hax = v.x; hay = v.y; hqx = v.z; hqy = v.w;
                    }
                }
            }
            // hub rows: whole-warp CSR sums
            for (int r = 0; r < nr && !pre_ok; r++) {
                const int li = lo + c0 + r;
                const int e0 = s_rpl[li], e1 = s_rpe[li];
                if (e1 - e0 <= 32) continue;   // warp-uniform
                const float2 me = s_pos[li];
                float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
                for (int ee = e0 + lane; ee < e1; ee += 32)
                    edge_terms(me.x, me.y, nbr_pos(c0 + r, ee, e0), invK, am, rn, ax, ay, qx, qy);
                ax = warp_sum(ax);
                ay = warp_sum(ay);
                qx = warp_sum(qx);
                qy = warp_sum(qy);
                if (lane == r) {
                    hax = ax; hay = ay; hqx = qx; hqy = qy;
                }
            }
            // rows with at most 32 edges: the row's W lanes split its edges
            float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
            if (g < nr && !pre_ok) {
                const int li = lo + c0 + g;
                const int e0 = s_rpl[li], e1 = s_rpe[li];
                if (e1 - e0 <= 32) {
                    const float2 me = s_pos[li];
                    for (int ee = e0 + gl; ee < e1; ee += W)
                        edge_terms(me.x, me.y, nbr_pos(c0 + g, ee, e0), invK, am, rn, ax, ay, qx, qy);
                }
            }
            for (int o = W >> 1; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
                qx += __shfl_xor_sync(0xffffffffu, qx, o);
                qy += __shfl_xor_sync(0xffffffffu, qy, o);
            }
            if (lane == 0 && c0 == 0 && !snapshot) trace_mark(tk, rank, cur_s, 11);
            // the first lane of group g finishes row c0 + g (hub sums sit in lane g)
            const float hax_g = __shfl_sync(0xffffffffu, hax, g & 31);
            const float hay_g = __shfl_sync(0xffffffffu, hay, g & 31);
            const float hqx_g = __shfl_sync(0xffffffffu, hqx, g & 31);
            const float hqy_g = __shfl_sync(0xffffffffu, hqy, g & 31);
            const float rxs = rx, rys = ry;
            if (gl == 0 && g < nr) {
                const int c = c0 + g;
                const int li = lo + c;
                const int i = rank + G * li;
                const float2 me = s_pos[li];
                const int e0 = s_rpl[li], e1 = s_rpe[li];
                if (pre_ok || e1 - e0 > 32) {   // sums held by lane g
                    ax = hax_g; ay = hay_g; qx = hqx_g; qy = hqy_g;
                }
                // the bulk sums' two column halves, first + second
                float sxr = crep[c].x + crep[CR + c].x, cxr = 0.f;
                float syr = crep[c].y + crep[CR + c].y, cyr = 0.f;
                if (kprev >= 0) {
                    if (kahan) {
                        kahan_add(sxr, cxr, rxs);
                        kahan_add(syr, cyr, rys);
                    } else {
                        sxr += rxs;
                        syr += rys;
                    }
                }
                const float fx = fmaf(negRK2, (sxr - cxr) - qx, ax);
                const float fy = fmaf(negRK2, (syr - cyr) - qy, ay);
                if (snapshot) {
                    out[i] = make_float2(fx, fy);
                } else {
                    float nx = me.x, ny = me.y;
                    float gx = fx, gy = fy;
                    float n2 = fmaf(gx, gx, gy * gy);
                    if (n2 > 0.f) {
                        if (!(n2 < INFINITY)) {
                            gx *= 0x1p-64f;
                            gy *= 0x1p-64f;
                            n2 = fmaf(gx, gx, gy * gy);
                        }
                        const float sc = stepf * rsqrt_sfu(n2);
                        nx = fmaf(sc, gx, me.x);
                        ny = fmaf(sc, gy, me.y);
                    }
                    out[i] = make_float2(nx, ny);
                    s_pos[li] = make_float2(nx, ny);
                    e += (double)fmaf(fx, fx, fy * fy);   // |ct|^2 in FP32, summed in FP64
                }
            }
            __syncwarp();
        }
        return e;
    };

    if (snapshot) {
        for (int k = 0; k < B; k++) {
            if (!is_ctl) post_rows(k, s_crep);
            if (is_stager) {
                stage_ids(k, 0);
                cp_async_wait_all();
                __syncwarp();
                stage_pos(k, -1, 0, 0, buf0, buf0);
                cp_async_wait_all();
                __syncwarp();
            }
            __syncthreads();
            if (is_ctl) ctl_critical(k, -1, 0, 0, s_tile, 0.f, buf0, buf0, s_crep, tk.f_out, false);
            __syncthreads();
        }
        return;
    }

    // ---- main loop ---------------------------------------------------------------------
    const int S = tk.iters * B;
    const unsigned Gu = (unsigned)G;
    if (!is_ctl) post_rows(0, s_crep);   // batch 0's sums for step 0
    if (is_stager) {                     // ids of steps 0 and 1, positions of step 0
        stage_ids(0, 0);
        if (S > 1) stage_ids(1 % B, 1);
        cp_async_wait_all();
        __syncwarp();
        stage_pos(0, -1, 0, 0, buf1, buf0);
        cp_async_wait_all();
        __syncwarp();
        // step 0 takes batch B-1 from its tile (the start positions), like every step
        // its previous batch, so that a launch's first step sums as a continuing one
        csr_pre(0, B - 1, 0, 0, buf1, buf0);
    }
    __syncthreads();

    if (is_ctl) {
        double step = tk.step0;
        double e_iter = 0.0;
        for (int s = 0; s < S; s++) {
            const int it = s / B;
            const int k = s - it * B;
            if (k == 0 && s > 0) step *= 0.999;   // Algorithm 2: Step = Step * 0.999
            const float2* bold = (it & 1) ? buf1 : buf0;
            float2* bnew = (it & 1) ? buf0 : buf1;
            const int kprev = (k + B - 1) % B;   // step 0: the last batch at the start positions
            float4* tile = s_tile + (size_t)(s & 1) * TQ;
            cur_s = s;
            if (lane == 0) trace_mark(tk, rank, s, 0);
            if (s > 0) {
                // wait until every CTA has published batch kprev (bounded)
                int ok = 1;
                if (lane == 0) {
                    const unsigned target = (unsigned)s * Gu;
                    const unsigned long long t0 = global_ns();
                    for (unsigned spin = 0;; ++spin) {
                        if ((int)(ld_acquire_u32(prm.bar) - target) >= 0) break;
                        __nanosleep(32);   // 152 CTAs poll the same word
                        if ((spin & 255u) == 255u) {
                            if (ld_volatile_i32(prm.status) != 0) { ok = 0; break; }
                            if (global_ns() - t0 > kWaitLimitNs) {
                                atomicCAS(prm.status, 0, (int)BL_ETIMEOUT);
                                ok = 0;
                                break;
                            }
                        }
                    }
                    trace_mark(tk, rank, s, 1);
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __syncwarp();   // lane 0's acquire orders the other lanes' loads
                if (!ok) {
                    s_ctl[0] = 1;                 // tell the bulk warps to leave
                    bar_sync_n(kBarDone, T);      // their step s-1 is over
                    bar_arrive_n(kBarTile, T);
                    return;
                }
            }
            {
                // the buffer batch kprev was written to at step s-1 (step 0: the
                // launch's start positions)
                const float2* bprev = s == 0 ? buf0 : ((k == 0) ? bold : bnew);
                {   // the control warp copies the tile; each lane issues 4 column pairs'
                    // loads before storing any, so the copy costs about one round trip
                    const float2* src = bprev + (size_t)kprev * BS;
                    const int nc = min(BS, n - kprev * BS);
                    const int nq = (nc + 1) / 2;
                    for (int q0 = 0; q0 < nq; q0 += 128) {
                        float2 va[4], vb[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int q = q0 + lane + 32 * u;
                            va[u] = q < nq ? __ldcg(&src[2 * q]) : make_float2(0.f, 0.f);
                            vb[u] = (q < nq && 2 * q + 1 < nc) ? __ldcg(&src[2 * q + 1]) : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int q = q0 + lane + 32 * u;
                            if (q < nq) tile[q] = make_float4(va[u].x, vb[u].x, va[u].y, vb[u].y);
                        }
                    }
                }
                __syncwarp();
            }
            if (lane == 0) trace_mark(tk, rank, s, 2);
            if (s > 0) bar_sync_n(kBarDone, T);   // bulk finished step s-1
            if (lane == 0) trace_mark(tk, rank, s, 3);
            bar_arrive_n(kBarTile, T);            // bulk may start step s
            const double e = ctl_critical(k, kprev, s % 3, s & 1, tile, (float)step, bnew, bold,
                                          s_crep + (size_t)(s & 1) * 2 * CR, bnew, true);
            if (lane == 0) trace_mark(tk, rank, s, 4);
            e_iter += e;
            __syncwarp();
            if (lane == 0) {
                red_release_add_u32(prm.bar, 1u);   // this CTA's part of batch k is out
                trace_mark(tk, rank, s, 6);
            }
            if (k == B - 1) {
                const double et = warp_sum_d(e_iter);   // fixed butterfly over lanes
                if (lane == 0 && tk.e_iter != nullptr) tk.e_iter[(size_t)it * G + rank] = et;
                e_iter = 0.0;
            }
        }
        bar_sync_n(kBarDone, T);   // the bulk warps' last step
    } else {
        for (int s = 0; s < S; s++) {
            const int it = s / B;
            const int k = s - it * B;
            const int kprev = (k + B - 1) % B;   // step 0: the last batch at the start positions
            const int kpn = min(BS, n - kprev * BS);
            bar_sync_n(kBarTile, T);
            if (s_ctl[0]) return;
            if (tb == 0) trace_mark(tk, rank, s, 7);
            const float4* tile = s_tile + (size_t)(s & 1) * TQ;
            // rows moved at step s-1 by the control warp (every lane reads, so that
            // the warp does not diverge; a row's own slot, or slot 0 for a lane
            // without a row)
#pragma unroll
            for (int m = 0; m < RPT; m++) {
                const bool moved = s > 0 && bi[m] == kprev;
                const float2 p = s_pos[bi[m] >= 0 ? lrow[m] : 0];
                if (moved) {
                    XI[m] = pk2(p.x, p.x);
                    YI[m] = pk2(p.y, p.y);
                }
            }
            if (tb == 0) trace_mark(tk, rank, s, 5);
            if (is_stager && s + 1 < S) {   // neighbours of step s+1, ids of step s+2
                const int kn = (k + 1) % B;
                const int itn = kn == 0 ? it + 1 : it;
                const float2* nb = (itn & 1) ? buf0 : buf1;
                const float2* ob = (itn & 1) ? buf1 : buf0;
                stage_pos(kn, k, (s + 1) % 3, (s + 1) & 1, nb, ob);
                if (s + 2 < S) stage_ids((k + 2) % B, (s + 2) % 3);
            }
            // in the last iteration the rows already moved need more columns only
            // when their sums are carried to the next launch
            const bool last_iter = (it + 1 == tk.iters) && tk.carry == nullptr;
            bool need[RPT];
#pragma unroll
            for (int m = 0; m < RPT; m++)
                need[m] = bi[m] >= 0 && bi[m] != k && (!last_iter || bi[m] >= k);
            if (tb == 0) trace_mark(tk, rank, s, 10);
            add_tile(tile, kpn, need);
            // the launch's last step: every row's sums as the next step would find
            // them (before batch 0's are posted), for a launch that continues the run
            if (s + 1 == S && tk.carry != nullptr) carry_rows(true);
            post_rows((k + 1) % B, s_crep + (size_t)((s + 1) & 1) * 2 * CR);
            if (tb == 0) trace_mark(tk, rank, s, 8);
            bar_arrive_n(kBarDone, T);
            // the staging warp: once the positions of step s+1 have landed, that step's
            // CSR sums, announced to the control warp on their own barrier (the control
            // warp reads neither the staged positions nor these sums before then)
            if (is_stager && s + 1 < S) {
                const int kn = (k + 1) % B;
                const int itn = kn == 0 ? it + 1 : it;
                cp_async_wait_all();
                __syncwarp();
                csr_pre(kn, k, (s + 1) % 3, (s + 1) & 1, (itn & 1) ? buf0 : buf1, (itn & 1) ? buf1 : buf0);
                bar_arrive_n(kBarPre, 64);
            }
        }
    }
}

__global__ void energy_reduce_kernel(const double* __restrict__ e_iter, int iters, int G,
                                     double* __restrict__ energy) {
    // one warp per iteration; fixed order over the per-CTA sums
    const int it = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (it >= iters) return;
    const double* p = e_iter + (size_t)it * G;
    double e = 0.0;
    for (int q = lane; q < G; q += 32) e += p[q];
    e = warp_sum_d(e);
    if (lane == 0) energy[it] = e;
}

bl_status energy_reduce(const double* e_iter, int iters, int G, double* energy, cudaStream_t st) {
    if (iters <= 0) return BL_OK;
    const int wpb = 8;
    energy_reduce_kernel<<<div_up(iters, wpb), wpb * 32, 0, st>>>(e_iter, iters, G, energy);
    BL_CUDA_TRY(cudaGetLastError());
    return BL_OK;
}

// ---------------------------------------------------------------------------
// ceiling probes: the pair loop and the SFU reciprocal alone (profiling)
// ---------------------------------------------------------------------------

// Every thread: one row against a 256-column tile in shared memory, `reps` times,
// with the engine's pair loop (tile_pairs2). Warps on sub-partition 0 (w % 4 == 0)
// sit out when skip_sp0. Lane 0 of each warp records its clock64 span.
__global__ void __launch_bounds__(512, 1) pair_rate_kernel(const float4* __restrict__ src, int reps,
                                                           int skip_sp0, float* out,
                                                           long long* span) {
    constexpr int NP = 128;
    __shared__ float4 tile[NP];
    for (int q = threadIdx.x; q < NP; q += blockDim.x) tile[q] = src[q];
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const float x = 0.001f * threadIdx.x, y = 0.002f * threadIdx.x + 0.5f;
    f32x2 XI[1] = {pk2(x, x)}, YI[1] = {pk2(y, y)};
    f32x2 AX[1] = {pk2(0.f, 0.f)}, AY[1] = {pk2(0.f, 0.f)};
    const long long t0 = clock64();
    if (!(skip_sp0 && w % 4 == 0))
        for (int r = 0; r < reps; r++) tile_pairs2<1>(tile, NP, 0, 1, XI, YI, AX, AY);
    const long long t1 = clock64();
    float a, b, c, d;
    upk2(AX[0], a, b);
    upk2(AY[0], c, d);
    out[blockIdx.x * blockDim.x + threadIdx.x] = a + b + c + d;
    if ((threadIdx.x & 31) == 0) span[blockIdx.x * 16 + w] = t1 - t0;
}

// Every thread: 8 independent chains x <- rcp.approx(x/2 + 1), `reps` rounds (timed with
// CUDA events: the clock of the SM is read at issue, ahead of the chains' results).
__global__ void __launch_bounds__(512, 1) rcp_rate_kernel(int reps, float* out) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = 1.5f + 0.01f * k + 1e-4f * threadIdx.x;
    for (int r = 0; r < reps; r++) {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = rcp_sfu(fmaf(v[k], 0.5f, 1.0f));   // no rcp(rcp(x)) to fold
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) sum += v[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

bl_status exact_pair_rate(int threads, int skip_sp0, double* pairs_per_clk, double* rcp_per_clk,
                          double* pair_ms) {
    if (threads < 32 || threads > 512 || threads % 32 != 0)
        return set_error(BL_EINVAL, "pair-rate probe: threads a multiple of 32 in [32, 512]");
    const int sms = device_sm_count();
    cudaStream_t st = current_stream();
    const Allocator& al = current_allocator();
    DevBuf src, out, span;
    BL_TRY(src.ensure(al, 128 * sizeof(float4)));
    BL_TRY(out.ensure(al, (size_t)sms * 512 * sizeof(float)));
    BL_TRY(span.ensure(al, (size_t)sms * 16 * sizeof(long long)));
    float4 h[128];
    for (int q = 0; q < 128; q++)
        h[q] = make_float4(0.01f * q, 0.011f * q + 0.5f, 0.013f * q, 0.017f * q + 0.25f);
    std::vector<long long> hs((size_t)sms * 16);
    const int reps = 400;
    cudaEvent_t a = nullptr, b = nullptr;
    bl_status s = BL_OK;
    cudaError_t e = cudaMemcpyAsync(src.p, h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    auto max_span = [&](long long& m) {
        e = cudaMemcpyAsync(hs.data(), span.p, hs.size() * sizeof(long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        m = 0;
        for (long long v : hs) m = std::max(m, v);
    };
    const int warps = threads / 32;
    const int active = skip_sp0 ? warps - (warps + 3) / 4 : warps;
    long long m = 0;
    for (int pass = 0; pass < 2 && e == cudaSuccess; pass++) {   // warm-up, then measured
        if (e == cudaSuccess) e = cudaMemsetAsync(span.p, 0, hs.size() * sizeof(long long), st);
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        if (e == cudaSuccess) {
            pair_rate_kernel<<<sms, threads, 0, st>>>(src.as<float4>(), reps, skip_sp0, out.as<float>(),
                                                      span.as<long long>());
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) max_span(m);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && m > 0) {
        *pairs_per_clk = (double)active * 32 * 256.0 * reps / (double)m;
        *pair_ms = ms;
    }
    // SM clock of the pair kernel (its spans against its events), for the reciprocals
    const double mhz = (e == cudaSuccess && ms > 0 && m > 0) ? (double)m / (ms * 1e3) : 0.0;
    const int rreps = 20000;
    for (int pass = 0; pass < 2 && e == cudaSuccess; pass++) {
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) {
            rcp_rate_kernel<<<sms, 512, 0, st>>>(rreps, out.as<float>());
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
    }
    float rms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&rms, a, b);
    if (e == cudaSuccess && rms > 0 && mhz > 0)
        *rcp_per_clk = 512.0 * 8 * rreps / ((double)rms * 1e3 * mhz);
    if (e != cudaSuccess) s = cuda_error(e, "pair-rate probe");
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    src.release();
    out.release();
    span.release();
    return s;
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------

template <int RPT, int TB>
static bl_status launch_grid_t(const ExactPlan& pl, const ExactTask& tk, const ExactParams& prm,
                               cudaStream_t st) {
    constexpr int T = TB + 32;
    auto kern = exact_grid_kernel<RPT, TB>;
    const EngineSmem L(tk.BS, div_up(tk.n, pl.G), tk.crit_cap, tk.nbr_cap, TB / 32);
    const size_t smem = (size_t)L.total;
    BL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    BL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, smem));
    if (occ < 1) return set_error(BL_ECUDA, "exact engine: kernel does not fit on an SM");
    if (pl.G > occ * device_sm_count())
        return set_error(BL_EINVAL, "exact engine: grid exceeds co-resident CTAs");
    ExactTask t = tk;
    for (int w = 0; w < 16; w++) t.piece[w] = pl.piece[w];
    ExactParams p = prm;
    void* args[] = {&t, &p};
    BL_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(pl.G), dim3(T), args, smem, st));
    return BL_OK;
}
template <int TB>
static bl_status dispatch_rpt(const ExactPlan& pl, const ExactTask& tk, const ExactParams& prm,
                              cudaStream_t st) {
    switch (pl.rpt) {
        case 1: return launch_grid_t<1, TB>(pl, tk, prm, st);
        case 2: return launch_grid_t<2, TB>(pl, tk, prm, st);
        case 3: return launch_grid_t<3, TB>(pl, tk, prm, st);
        case 4: return launch_grid_t<4, TB>(pl, tk, prm, st);
        default: break;
    }
    if constexpr (TB == 256) {
        switch (pl.rpt) {
            case 6: return launch_grid_t<6, TB>(pl, tk, prm, st);
            case 8: return launch_grid_t<8, TB>(pl, tk, prm, st);
            default: break;
        }
    }
    return set_error(BL_EINVAL, "exact engine: unsupported rows per thread");
}

// Bulk pieces for one row per thread. The nloc rows of a CTA form blocks of 32;
// a block is two units (its halves), and a last block of at most 16 rows is one
// unit folded onto one warp. Each sub-partition gets an equal share of the units,
// the control warp's the remainder, as whole blocks per warp plus at most one
// single unit (a fold, or a half whose other half goes to another sub-partition). Bulk warp w runs on
// sub-partition (w + 1) % 4. piece[w] = block | halves << 16 | fold << 18 (0: idle).
// Returns false when the pieces do not fit the warps (the caller then gives each
// warp one whole block in turn).
static bool plan_pieces(int nloc, int NW, int* piece) {
    const int nfull = nloc / 32, rem = nloc % 32;
    const bool fold = rem > 0 && rem <= 16;
    const int nwhole = nfull + (rem > 16 ? 1 : 0);   // blocks of two half units
    const int U = 2 * nwhole + (fold ? 1 : 0);
    std::vector<int> warps[4];
    for (int w = 0; w < NW; w++) warps[(w + 1) % 4].push_back(w);
    int budget[4] = {0, 0, 0, 0};
    const int target = (U + 3) / 4;
    int left = U;
    for (int j = 1; j <= 3; j++) {
        budget[j] = std::min({target, 2 * (int)warps[j].size(), left});
        left -= budget[j];
    }
    budget[0] = std::min(left, 2 * (int)warps[0].size());
    left -= budget[0];
    for (int j = 1; j <= 3 && left > 0; j++) {   // what sub-partition 0 cannot hold
        const int add = std::min(left, 2 * (int)warps[j].size() - budget[j]);
        budget[j] += add;
        left -= add;
    }
    if (left > 0) return false;
    for (int w = 0; w < 16; w++) piece[w] = 0;
    int next_block = 0, pending = -1;   // pending: second half of a split block
    bool fold_left = fold;
    for (int j : {1, 2, 3, 0}) {
        int need = budget[j];
        size_t wi = 0;
        while (need >= 2 && next_block < nwhole && wi < warps[j].size()) {
            piece[warps[j][wi++]] = next_block++ | (3 << 16);
            need -= 2;
        }
        while (need > 0 && wi < warps[j].size()) {
            if (fold_left) {
                piece[warps[j][wi++]] = nfull | (1 << 18);
                fold_left = false;
            } else if (pending >= 0) {
                piece[warps[j][wi++]] = pending | (2 << 16);
                pending = -1;
            } else if (next_block < nwhole) {
                piece[warps[j][wi++]] = next_block | (1 << 16);
                pending = next_block++;
            } else {
                return false;
            }
            need--;
        }
        if (need > 0) return false;
    }
    return next_block == nwhole && pending < 0 && !fold_left;
}


// Launch shape: G = one CTA per SM (at least 64 rows each); bulk threads TB and
// rows per thread by the rows per CTA: up to 512 rows one row per thread, the
// bulk rounded up to whole warps (256, 320, 384, 448 or 512 threads) so that few
// lanes idle in the pair loop; up to 2048 rows 512 threads x 2..4 rows, beyond
// that 256 threads x 6..8 rows.
bl_status exact_plan(int n, int BS, int ctas_hint, int threads_hint, ExactPlan* out) {
    if (n <= 0 || BS <= 0) return set_error(BL_EINVAL, "exact engine: empty problem");
    const int sms = device_sm_count();
    if (threads_hint <= 0) {   // tuning override: bulk threads per CTA
        const char* e = std::getenv("BL_EXACT_THREADS");
        if (e) threads_hint = std::atoi(e);
    }
    const int G = ctas_hint > 0 ? ctas_hint : std::min(sms, std::max(1, div_up(n, 64)));
    const int nloc = div_up(n, G);
    const bool hint_ok = threads_hint == 256 || threads_hint == 320 || threads_hint == 384 ||
                         threads_hint == 448 || threads_hint == 512;
    // Default 256 or 512: a shape with fewer bulk warps leaves more rows on the
    // sub-partition the control warp shares, which slows the per-minibatch chain
    // (measured: 448 threads on n = 65,536 ran 6% slower than 512). The in-between
    // shapes stay available through BL_EXACT_THREADS.
    int T = hint_ok ? threads_hint : (nloc <= 256 ? 256 : 512);
    if (T != 256 && T != 512 && div_up(nloc, T) > 1) T = 512;   // the in-between shapes take one row each
    if (T == 288) T = 320;
    if (T == 352) T = 384;
    if (T == 416) T = 448;
    if (T == 480) T = 512;
    int rpt = div_up(nloc, T);
    if (T == 512 && rpt > 4) {
        T = 256;
        rpt = div_up(nloc, T);
    }
    static const int kChoices256[] = {1, 2, 3, 4, 6, 8};
    static const int kChoices512[] = {1, 2, 3, 4};
    int chosen = -1;
    if (T == 256) {
        for (int c : kChoices256)
            if (c >= rpt) { chosen = c; break; }
    } else {
        for (int c : kChoices512)
            if (c >= rpt) { chosen = c; break; }
    }
    if (chosen < 0)
        return set_error(BL_EINVAL, "exact engine: too many vertices for exact mode (use BL_BH)");
    out->G = G;
    out->T = T;
    out->rpt = chosen;
    for (int w = 0; w < 16; w++) out->piece[w] = 0;
    if (chosen == 1 && !plan_pieces(nloc, T / 32, out->piece)) {
        const int NW = T / 32;   // one whole block per warp, the control warp's sub-partition last
        for (int wb = 0; wb < NW; wb++) {
            const int ws = (wb + 1) % 4 == 0 ? (NW - NW / 4) + (wb + 1) / 4 - 1 : wb - (wb + 1) / 4;
            out->piece[wb] = 32 * ws < nloc ? (ws | (3 << 16)) : 0;
        }
    }
    out->crit_cap = div_up(std::min(BS, n), G) + 1;
    out->nbr_cap = 2048;
    while (EngineSmem(BS, nloc, out->crit_cap, out->nbr_cap, T / 32).total > 200 * 1024 &&
           out->nbr_cap > 256)
        out->nbr_cap /= 2;
    if (EngineSmem(BS, nloc, out->crit_cap, out->nbr_cap, T / 32).total > 220 * 1024)
        return set_error(BL_EINVAL, "exact engine: batch too large for shared memory");
    return BL_OK;
}

bl_status exact_launch(const ExactPlan& pl, const ExactTask& task, const ExactParams& prm,
                       cudaStream_t st) {
    if (task.n <= 0) return BL_OK;
    if (task.BS > kMaxBatch) return set_error(BL_EINVAL, "exact engine: batch too large");
    // the kernel counts minibatch steps (iterations x minibatches) in int32
    if ((int64_t)task.iters * task.B > 0x7fffffffLL)
        return set_error(BL_EINVAL, "exact engine: more than 2^31 - 1 minibatch steps in one launch");
    switch (pl.T) {
        case 512: return dispatch_rpt<512>(pl, task, prm, st);
        case 448: return launch_grid_t<1, 448>(pl, task, prm, st);
        case 384: return launch_grid_t<1, 384>(pl, task, prm, st);
        case 320: return launch_grid_t<1, 320>(pl, task, prm, st);
        default: return dispatch_rpt<256>(pl, task, prm, st);
    }
}

}  // namespace bl
