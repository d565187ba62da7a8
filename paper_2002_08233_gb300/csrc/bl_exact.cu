// Exact-mode BatchLayout engine (Section 2.2, Section 3.3, Algorithm 2).
//
// Column formulation of the minibatch sweep. Iteration t visits batches
// k = 0..B-1 in order; batch k's force ct_i needs, for every other batch c, the
// positions of c as they are when k is processed: updated this iteration if
// c < k, from the previous iteration if c >= k. Equivalently, the moment batch c
// is updated, its new positions are exactly what every row needs from c until
// c moves again. So one global step s = (t, k):
//   1. column phase: the positions batch k-1 received at step s-1 (a BS-vertex
//      column tile) are added to the repulsion accumulator of every row whose
//      next update still lies inside this launch;
//   2. update phase: the rows of batch k now hold the repulsion of all j (their
//      last missing column was just added); the CTAs owning them add the CSR
//      attraction (warp per row, shuffle reduction), remove the neighbour
//      repulsion the all-pairs sum included, and move each vertex by
//      Step * ct/|ct| (Algorithm 2's update);
//   3. grid barrier.
// A prologue adds, for each row, the columns c >= batch(row) at the starting
// positions. Over a launch every row receives every column exactly once per
// iteration, so a launch of T iterations evaluates exactly T*n^2 pairs.
//
// Rows are split evenly across CTAs (CTA ranges need not align with batches)
// and each thread keeps its rows' positions and Kahan-compensated repulsion
// sums in registers for the whole launch. New positions of batch k go to a
// staging buffer (two, alternating by step) so that nothing a CTA may still
// read as "old" is overwritten inside the step (Jacobi semantics within a batch);
// the owners copy them into the position array one step later.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>

#include "bl_internal.cuh"

namespace bl {

template <int RPT, int T, class Bar>
__device__ __forceinline__ void exact_engine(const ExactTask& tk, const ExactParams& prm, int rank,
                                             int nrank, Bar& bar, float2* __restrict__ stage) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = tk.n, BS = tk.BS, B = tk.B;
    float4* s_col = reinterpret_cast<float4*>(smem);            // ceil(BS/2) float4
    float4* s_row = s_col + ((BS + 1) >> 1);                     // BS float4
    double* s_e = reinterpret_cast<double*>(s_row + BS);         // T/32 doubles

    const int rows_per = (n + nrank - 1) / nrank;
    const int r0 = min(n, rank * rows_per);
    const int r1 = min(n, r0 + rows_per);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int W = T / 32;
    const bool snapshot = tk.iters == 0;
    const bool rn = prm.repulse_neighbors != 0;

    float xi[RPT], yi[RPT], sx[RPT], sy[RPT], cx[RPT], cy[RPT];
    int bi[RPT];
#pragma unroll
    for (int m = 0; m < RPT; m++) {
        const int i = r0 + tid + m * T;
        const bool v = i < r1;
        const float2 p = v ? __ldcg(&tk.pos[i]) : make_float2(0.f, 0.f);
        xi[m] = p.x;
        yi[m] = p.y;
        sx[m] = sy[m] = cx[m] = cy[m] = 0.f;
        bi[m] = v ? i / BS : -1;
    }
    if (r0 >= r1 && snapshot) return;   // nothing owned, nothing to wait for
    const int b_first = r0 < r1 ? r0 / BS : B;      // first batch with a row here
    const int b_last = r0 < r1 ? (r1 - 1) / BS : -1;

    // ---- column tile: load BS positions into shared memory --------------------
    auto load_col = [&](const float2* src, int nc) {
        for (int q = tid; q < (nc + 1) / 2; q += T) {
            const float2 a = __ldcg(&src[2 * q]);
            const float2 b = (2 * q + 1 < nc) ? __ldcg(&src[2 * q + 1]) : make_float2(0.f, 0.f);
            s_col[q] = make_float4(a.x, a.y, b.x, b.y);
        }
    };
    // ---- pair loop over the staged tile; adds to rows flagged in `need` --------
    auto accumulate = [&](int nc, const bool (&need)[RPT]) {
        float ax[RPT], ay[RPT];
#pragma unroll
        for (int m = 0; m < RPT; m++) ax[m] = ay[m] = 0.f;
        const int np = nc >> 1;
#pragma unroll 4
        for (int q = 0; q < np; q++) {
            const float4 p = s_col[q];
#pragma unroll
            for (int m = 0; m < RPT; m++) {
                rep_pair(xi[m], yi[m], p.x, p.y, ax[m], ay[m]);
                rep_pair(xi[m], yi[m], p.z, p.w, ax[m], ay[m]);
            }
        }
        if (nc & 1) {
            const float4 p = s_col[np];
#pragma unroll
            for (int m = 0; m < RPT; m++) rep_pair(xi[m], yi[m], p.x, p.y, ax[m], ay[m]);
        }
#pragma unroll
        for (int m = 0; m < RPT; m++)
            if (need[m]) {
                kahan_add(sx[m], cx[m], ax[m]);
                kahan_add(sy[m], cy[m], ay[m]);
            }
    };
    // ---- update phase for the rows of batch k in [r0, r1) ------------------------
    // prev_lo/prev_n: the batch updated one step earlier, whose new positions are
    // read from prev_stage instead of the position array. Returns false on error.
    auto update_batch = [&](int k, float stepf, const float2* prev_stage, int prev_lo, int prev_n,
                            float2* out_stage, double* e_slot) {
        const int blo = max(r0, k * BS), bhi = min(r1, (k + 1) * BS);
        if (blo >= bhi) return;   // CTA-uniform
#pragma unroll
        for (int m = 0; m < RPT; m++) {
            const int i = r0 + tid + m * T;
            if (i >= blo && i < bhi)
                s_row[i - blo] = make_float4(xi[m], yi[m], sx[m] - cx[m], sy[m] - cy[m]);
        }
        __syncthreads();
        double e_acc = 0.0;
        for (int r = blo + warp; r < bhi; r += W) {
            const float4 me = s_row[r - blo];
            float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
            const int e0 = __ldg(&tk.rowptr[r]), e1 = __ldg(&tk.rowptr[r + 1]);
            for (int e = e0 + lane; e < e1; e += 32) {
                const int j = __ldg(&tk.colids[e]);
                const unsigned pj_off = (unsigned)(j - prev_lo);
                const float2 pj = pj_off < (unsigned)prev_n ? __ldcg(&prev_stage[pj_off])
                                                            : __ldcg(&tk.pos[j]);
                const float dx = pj.x - me.x;
                const float dy = pj.y - me.y;
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, BL_EPS2));
                // attraction (d^2/K) * (c_j - c_i)/d = (d/K) (c_j - c_i)
                const float a = d2 * rsqrt_sfu(d2) * prm.invK;
                ax = fmaf(dx, a, ax);
                ay = fmaf(dy, a, ay);
                if (!rn) {   // the all-pairs sum repelled this neighbour: take it back
                    const float inv = rcp_sfu(d2);
                    qx = fmaf(dx, inv, qx);
                    qy = fmaf(dy, inv, qy);
                }
            }
            ax = warp_sum(ax);
            ay = warp_sum(ay);
            qx = warp_sum(qx);
            qy = warp_sum(qy);
            if (lane == 0) {
                const float fx = fmaf(prm.negRK2, me.z - qx, ax);
                const float fy = fmaf(prm.negRK2, me.w - qy, ay);
                if (snapshot) {
                    tk.f_out[r] = make_float2(fx, fy);
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
                    out_stage[r - k * BS] = make_float2(nx, ny);
                    s_row[r - blo].x = nx;
                    s_row[r - blo].y = ny;
                    e_acc += (double)fx * (double)fx + (double)fy * (double)fy;
                }
            }
        }
        if (lane == 0) s_e[warp] = e_acc;
        __syncthreads();
        if (tid == 0 && e_slot != nullptr) {
            double e = 0.0;
            for (int w = 0; w < W; w++) e += s_e[w];
            *e_slot = e;
        }
#pragma unroll
        for (int m = 0; m < RPT; m++) {
            const int i = r0 + tid + m * T;
            if (i >= blo && i < bhi) {
                if (!snapshot) {
                    const float4 v = s_row[i - blo];
                    xi[m] = v.x;
                    yi[m] = v.y;
                }
                sx[m] = sy[m] = cx[m] = cy[m] = 0.f;
            }
        }
        __syncthreads();
    };

    // ---- prologue: columns c >= batch(row) at the starting positions (every column
    //      in snapshot mode) ---------------------------------------------------------
    {
        bool need[RPT];
        for (int c = snapshot ? 0 : b_first; c < B; c++) {
            const int nc = min(BS, n - c * BS);
#pragma unroll
            for (int m = 0; m < RPT; m++) need[m] = bi[m] >= 0 && (snapshot || bi[m] <= c);
            load_col(tk.pos + (size_t)c * BS, nc);
            __syncthreads();
            accumulate(nc, need);
            __syncthreads();
        }
    }
    if (snapshot) {
        // every row now holds the repulsion of all j at the same positions
        for (int k = b_first; k <= b_last; k++)
            update_batch(k, 0.f, nullptr, 0, 0, nullptr, nullptr);
        return;
    }
    if (!bar.sync()) return;   // nobody moves before every prologue has read

    // ---- main loop over global steps ------------------------------------------------
    const int S = tk.iters * B;
    double step = tk.step0;
    int prev_k = -1;
    for (int s = 0; s < S; s++) {
        const int it = s / B;
        const int k = s - it * B;
        if (k == 0 && s > 0) step *= 0.999;   // Algorithm 2: Step = Step * 0.999
        const float2* prev_stage = stage + (size_t)((s + 1) & 1) * BS;   // written at s-1
        float2* cur_stage = stage + (size_t)(s & 1) * BS;
        int prev_lo = 0, prev_n = 0;
        if (s > 0) {
            prev_lo = prev_k * BS;
            prev_n = min(BS, n - prev_lo);
            // owners make the position array current for the batch moved at s-1
#pragma unroll
            for (int m = 0; m < RPT; m++)
                if (bi[m] == prev_k) tk.pos[r0 + tid + m * T] = make_float2(xi[m], yi[m]);
            // column phase: does any row here still need column prev_k in this launch?
            const bool last_iter = (it + 1 == tk.iters);
            const bool any = !last_iter || (b_last >= k);
            if (any && r0 < r1) {
                bool need[RPT];
#pragma unroll
                for (int m = 0; m < RPT; m++) need[m] = bi[m] >= 0 && (!last_iter || bi[m] >= k);
                load_col(prev_stage, prev_n);
                __syncthreads();
                accumulate(prev_n, need);
                __syncthreads();
            }
        }
        if (k >= b_first && k <= b_last) {
            const int slot = rank - (k * BS) / rows_per;
            double* e_slot = tk.epart ? tk.epart + ((size_t)s * tk.P + slot) : nullptr;
            update_batch(k, (float)step, prev_stage, prev_lo, prev_n, cur_stage, e_slot);
        }
        prev_k = k;
        if (!bar.sync()) return;
    }
    // the last batch's owners publish its positions
#pragma unroll
    for (int m = 0; m < RPT; m++)
        if (bi[m] == prev_k) tk.pos[r0 + tid + m * T] = make_float2(xi[m], yi[m]);
}

template <int RPT, int T>
__global__ void __launch_bounds__(T) exact_grid_kernel(ExactTask tk, ExactParams prm,
                                                       float2* stage) {
    GridBarrier bar{prm.bar, prm.status, gridDim.x, 0u};
    exact_engine<RPT, T>(tk, prm, (int)blockIdx.x, (int)gridDim.x, bar, stage);
}

__global__ void energy_reduce_kernel(const double* __restrict__ epart, int iters, int B, int P,
                                     double* __restrict__ energy) {
    // one warp per iteration, fixed order: lanes stride over (batch, slot), then a
    // butterfly of fixed shape
    const int it = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (it >= iters) return;
    const double* p = epart + (size_t)it * B * P;
    double e = 0.0;
    for (int q = lane; q < B * P; q += 32) e += p[q];
    e = warp_sum_d(e);
    if (lane == 0) energy[it] = e;
}

bl_status energy_reduce(const double* epart, int iters, int B, int P, double* energy,
                        cudaStream_t st) {
    if (iters <= 0) return BL_OK;
    const int wpb = 8;
    energy_reduce_kernel<<<div_up(iters, wpb), wpb * 32, 0, st>>>(epart, iters, B, P, energy);
    BL_CUDA_TRY(cudaGetLastError());
    return BL_OK;
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------

template <int RPT, int T>
static bl_status launch_grid_t(const ExactTask& tk, const ExactParams& prm, cudaStream_t st,
                               int G, float2* stage) {
    auto kern = exact_grid_kernel<RPT, T>;
    const size_t smem = (size_t)((tk.BS + 1) / 2) * sizeof(float4) +
                        (size_t)tk.BS * sizeof(float4) + (T / 32) * sizeof(double);
    BL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    BL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, smem));
    if (occ < 1) return set_error(BL_ECUDA, "exact engine: kernel does not fit on an SM");
    const int max_g = occ * device_sm_count();
    if (G > max_g) return set_error(BL_EINVAL, "exact engine: grid exceeds co-resident CTAs");
    ExactTask t = tk;
    ExactParams p = prm;
    float2* s = stage;
    void* args[] = {&t, &p, &s};
    BL_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(T), args, smem, st));
    return BL_OK;
}

// rows-per-thread choices compiled in
static const int kRptChoices[] = {1, 2, 3, 4, 6, 8};

template <int T>
static bl_status dispatch_rpt(const ExactPlan& pl, const ExactTask& tk, const ExactParams& prm,
                              cudaStream_t st, float2* stage) {
    switch (pl.rpt) {
        case 1: return launch_grid_t<1, T>(tk, prm, st, pl.G, stage);
        case 2: return launch_grid_t<2, T>(tk, prm, st, pl.G, stage);
        case 3: return launch_grid_t<3, T>(tk, prm, st, pl.G, stage);
        case 4: return launch_grid_t<4, T>(tk, prm, st, pl.G, stage);
        case 6: return launch_grid_t<6, T>(tk, prm, st, pl.G, stage);
        case 8: return launch_grid_t<8, T>(tk, prm, st, pl.G, stage);
        default: return set_error(BL_EINVAL, "exact engine: unsupported rows per thread");
    }
}

bl_status exact_plan(int n, int BS, int ctas_hint, int threads_hint, ExactPlan* out) {
    if (n <= 0 || BS <= 0) return set_error(BL_EINVAL, "exact engine: empty problem");
    const int sms = device_sm_count();
    int T = threads_hint == 512 ? 512 : 256;
    // default grid: one CTA per SM, but keep at least 64 rows per CTA
    int G = ctas_hint > 0 ? ctas_hint : std::min(sms, std::max(1, div_up(n, 64)));
    int rpt = div_up(div_up(n, G), T);
    if (rpt > 8 && T == 256) {
        T = 512;
        rpt = div_up(div_up(n, G), T);
    }
    int chosen = -1;
    for (int c : kRptChoices)
        if (c >= rpt) { chosen = c; break; }
    if (chosen < 0) return set_error(BL_EINVAL, "exact engine: graph too large for the grid engine");
    out->G = G;
    out->T = T;
    out->rpt = chosen;
    const int rows_per = div_up(n, G);
    out->P = div_up(BS, rows_per) + 1;
    return BL_OK;
}

bl_status exact_launch(const ExactPlan& pl, const ExactTask& task, const ExactParams& prm,
                       float2* stage, cudaStream_t st) {
    if (task.n <= 0) return BL_OK;
    if (task.BS > kMaxBatch) return set_error(BL_EINVAL, "exact engine: batch too large");
    switch (pl.T) {
        case 512: return dispatch_rpt<512>(pl, task, prm, st, stage);
        default: return dispatch_rpt<256>(pl, task, prm, st, stage);
    }
}

}  // namespace bl
