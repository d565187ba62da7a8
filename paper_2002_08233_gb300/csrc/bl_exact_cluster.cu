// Exact mode for small graphs on one thread-block cluster (Algorithm 2).
//
// For a small graph the whole-GPU engine spends a minibatch step on its
// cross-CTA chain (publish, poll, tile copy through L2), not on pair work. Here
// the layout runs on one cluster of up to 16 CTAs that each keep a full copy of
// the positions in shared memory. A minibatch's rows are dealt round robin over
// the CTAs; each CTA sums its rows' forces against every column of its local
// copy, moves them, and writes the new positions into every CTA's inbox through
// distributed shared memory. One cluster barrier per minibatch makes them
// visible; each CTA then copies the inbox into its positions. The inboxes are
// double-buffered by minibatch parity, so a CTA that runs ahead writes the other
// buffer: the next write into a buffer comes after the next barrier, which every
// CTA reaches only after it has copied that buffer out.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "bl_internal.cuh"

namespace cg = cooperative_groups;

namespace bl {
namespace {

constexpr int kClThreads = 512;
constexpr int kClWarps = kClThreads / 32;

struct ClusterTask {
    int n, BS, B, iters;
    int nnz;
    const int* rowptr;
    const int* colids;
    float2* pos;        // in: start positions; out: positions after `iters` iterations
    double* e_iter;     // [iters][C] per-CTA energies
    double step0;
    float invK, negRK2;
    int rn, am;
    int kahan;          // 1: each lane's strided repulsion sum compensated
    int csr_smem;       // CSR copied into shared memory
    int gs;             // threads per row group (multiple of 32)
};

struct ClusterSmem {
    size_t pos, inbox, rp, ci, red, e, total;
    __host__ __device__ ClusterSmem(int n, int BS, int nnz, bool csr, int groups) {
        pos = 0;
        inbox = pos + ((size_t)n * 8 + 15) / 16 * 16;
        rp = inbox + (size_t)2 * BS * 8;
        ci = rp + (csr ? ((size_t)(n + 1) * 4 + 15) / 16 * 16 : 0);
        red = ci + (csr ? ((size_t)nnz * 4 + 15) / 16 * 16 : 0);
        e = red + (size_t)kClWarps * 6 * 4;
        total = e + (size_t)groups * 8;
    }
};

__global__ void __launch_bounds__(kClThreads, 1) exact_cluster_kernel(ClusterTask tk) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int n = tk.n, BS = tk.BS, GS = tk.gs;
    const int groups = kClThreads / GS;
    extern __shared__ __align__(16) unsigned char smem[];
    const ClusterSmem L(n, BS, tk.nnz, tk.csr_smem != 0, groups);
    float2* P = reinterpret_cast<float2*>(smem + L.pos);
    float2* inbox = reinterpret_cast<float2*>(smem + L.inbox);
    int* s_rp = reinterpret_cast<int*>(smem + L.rp);
    int* s_ci = reinterpret_cast<int*>(smem + L.ci);
    float* s_red = reinterpret_cast<float*>(smem + L.red);
    double* s_e = reinterpret_cast<double*>(smem + L.e);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = tid / GS, tg = tid - grp * GS;
    const int* rowptr = tk.csr_smem ? s_rp : tk.rowptr;
    const int* colids = tk.csr_smem ? s_ci : tk.colids;
    const bool rn = tk.rn != 0;

    for (int i = tid; i < n; i += kClThreads) P[i] = tk.pos[i];
    if (tk.csr_smem) {
        for (int i = tid; i <= n; i += kClThreads) s_rp[i] = tk.rowptr[i];
        for (int e = tid; e < tk.nnz; e += kClThreads) s_ci[e] = tk.colids[e];
    }
    if (tid < groups) s_e[tid] = 0.0;
    cl.sync();   // every CTA is resident and loaded before anyone writes remotely

    // every CTA's inbox, as seen from this CTA (distributed shared memory)
    float2* remote[16];
#pragma unroll
    for (int c = 0; c < 16; c++)
        remote[c] = c < C ? cl.map_shared_rank(inbox, (unsigned)c) : nullptr;

    double step = tk.step0;
    for (int t = 0; t < tk.iters; t++) {
        const float stepf = (float)step;
        for (int b = 0; b < tk.B; b++) {
            const int r0 = b * BS, r1 = min(n, r0 + BS);
            float2* box = inbox + (size_t)(b & 1) * BS;
            const int mine = (r1 - r0 - rank + C - 1) / C;   // rows r0 + rank + C*m
            for (int m0 = 0; m0 < mine; m0 += groups) {
                const int m = m0 + grp;
                const bool have = m < mine;
                const int i = r0 + rank + C * m;
                float rx = 0.f, ry = 0.f, ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f;
                float2 me = make_float2(0.f, 0.f);
                if (have) {
                    me = P[i];
                    if (tk.kahan) {   // every term compensated (uniform branch)
                        float cx = 0.f, cy = 0.f;
#pragma unroll 4
                        for (int j = tg; j < n; j += GS) {
                            const float2 p = P[j];
                            float tx = 0.f, ty = 0.f;
                            rep_pair(me.x, me.y, p.x, p.y, tx, ty);   // j == i gives 0
                            kahan_add(rx, cx, tx);
                            kahan_add(ry, cy, ty);
                        }
                        rx -= cx;
                        ry -= cy;
                    } else {
#pragma unroll 4
                        for (int j = tg; j < n; j += GS) {
                            const float2 p = P[j];
                            rep_pair(me.x, me.y, p.x, p.y, rx, ry);   // j == i gives 0
                        }
                    }
                    const int e1 = rowptr[i + 1];
                    for (int e = rowptr[i] + tg; e < e1; e += GS)
                        edge_terms(me.x, me.y, P[colids[e]], tk.invK, tk.am, rn, ax, ay, qx, qy);
                }
                float v[6] = {rx, ry, ax, ay, qx, qy};
#pragma unroll
                for (int k = 0; k < 6; k++) v[k] = warp_sum(v[k]);
                // the warps of a group combine in order
                if (lane == 0)
#pragma unroll
                    for (int k = 0; k < 6; k++) s_red[warp * 6 + k] = v[k];
                __syncthreads();
                if (have && tg == 0) {
                    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    for (int w = grp * (GS / 32); w < (grp + 1) * (GS / 32); w++)
#pragma unroll
                        for (int k = 0; k < 6; k++) s[k] += s_red[w * 6 + k];
                    const float fx = fmaf(tk.negRK2, s[0] - s[4], s[2]);
                    const float fy = fmaf(tk.negRK2, s[1] - s[5], s[3]);
                    float nx = me.x, ny = me.y, gx = fx, gy = fy;
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
                    s_e[grp] += (double)fmaf(fx, fx, fy * fy);
                    const float2 np2 = make_float2(nx, ny);
                    const int slot = (b & 1) * BS + (i - r0);
                    for (int c = 0; c < C; c++) remote[c][slot] = np2;   // every CTA's inbox
                }
                if (m0 + groups < mine) __syncthreads();   // s_red is reused by the next round
            }
            cl.sync();   // the minibatch's new positions are in every inbox
            for (int r = r0 + tid; r < r1; r += kClThreads) P[r] = box[r - r0];
            __syncthreads();
        }
        if (tid == 0) {   // this CTA's energy of iteration t, groups in order
            double e = 0.0;
            for (int g = 0; g < groups; g++) {
                e += s_e[g];
                s_e[g] = 0.0;
            }
            if (tk.e_iter) tk.e_iter[(size_t)t * C + rank] = e;
        }
        __syncthreads();
        step *= 0.999;   // Algorithm 2: Step = Step * 0.999
    }
    if (rank == 0)
        for (int i = tid; i < n; i += kClThreads) tk.pos[i] = P[i];
    cl.sync();   // no CTA leaves while another may still write into its inbox
}

int cluster_size_cached = -1;

}  // namespace

// Largest cluster (16, else 8) the device can run with this kernel, 0 if none.
static int cluster_size_for(size_t smem) {
    cudaFuncSetAttribute(exact_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(exact_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, exact_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0)
            return c;
        cudaGetLastError();
    }
    return 0;
}

bool cluster_engine_fits(int n, int BS, int64_t nnz) {
    if (n < 2 || n > kClusterMaxN || BS > kMaxBatch) return false;
    const ClusterSmem L(n, BS, (int)std::min<int64_t>(nnz, 1 << 30), false, kClWarps);
    return L.total <= 200 * 1024;
}

bl_status cluster_run(const int* rowptr, const int* colids, int64_t nnz, int n, float2* pos, int iters, int BS,
                      double step0, float invK, float negRK2, int rn, int am, int kahan, double* e_iter_buf,
                      double* energy, cudaStream_t st, int* C_out) {
    const bool csr = (size_t)((n + 1) + nnz) * 4 + (size_t)n * 8 + (size_t)4 * BS * 8 + 4096 <= 200 * 1024;
    // threads per row group: the minibatch's rows per CTA spread over the CTA
    int C = cluster_size_cached;
    const ClusterSmem L0(n, BS, (int)nnz, csr, kClWarps);
    if (C < 0) C = cluster_size_cached = cluster_size_for(200 * 1024);
    if (C <= 0) return set_error(BL_ECUDA, "exact cluster engine: no cluster launch on this device");
    const int rows = (BS + C - 1) / C;
    int gs = kClThreads;
    while (gs > 32 && gs / 2 * rows >= kClThreads) gs /= 2;   // groups = 512/gs >= rows when possible
    const int groups = kClThreads / gs;
    const ClusterSmem L(n, BS, (int)nnz, csr, groups);
    (void)L0;
    ClusterTask tk{};
    tk.n = n;
    tk.BS = BS;
    tk.B = div_up(n, BS);
    tk.iters = iters;
    tk.nnz = (int)nnz;
    tk.rowptr = rowptr;
    tk.colids = colids;
    tk.pos = pos;
    tk.e_iter = e_iter_buf;
    tk.step0 = step0;
    tk.invK = invK;
    tk.negRK2 = negRK2;
    tk.rn = rn;
    tk.am = am;
    tk.kahan = kahan;
    tk.csr_smem = csr ? 1 : 0;
    tk.gs = gs;
    BL_CUDA_TRY(cudaFuncSetAttribute(exact_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)L.total));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BL_CUDA_TRY(cudaLaunchKernelEx(&cfg, exact_cluster_kernel, tk));
    if (energy) BL_TRY(energy_reduce(e_iter_buf, iters, C, energy, st));
    if (C_out) *C_out = C;
    return BL_OK;
}

}  // namespace bl
