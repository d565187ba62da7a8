/*
 * batchlayout.h -- C ABI of a GB300-native (sm_103a) implementation of
 * BatchLayout's force-directed layout iteration (Rahman, Sujon, Azad,
 * "BatchLayout: A Batch-Parallel Force-Directed Graph Layout Algorithm in
 * Shared Memory", arXiv 2002.08233).
 *
 * What one iteration computes (Section 2.2, Section 3.3, Algorithm 2):
 *   for each minibatch b of BS consecutive vertex ids, in order:
 *     for every i in b, from the same positions c:
 *       ct_i = sum_{(i,j) in E} (|c_j-c_i|^2 / K) u_ij
 *            + sum_{j != i, (i,j) not in E} (-R K^2 / |c_j-c_i|) u_ij,
 *       u_ij = (c_j - c_i)/|c_j - c_i|
 *     then c_i += Step * ct_i / |ct_i|  (no move when ct_i = 0),
 *          Energy += |ct_i|^2
 *   Step = 0.999^t for iteration t (Step starts at 1.0).
 * Barnes-Hut mode (Section 3.5, Algorithms S3-S5) replaces the repulsion sum
 * with a quadtree walk: the tree is built once per iteration over Morton-sorted
 * positions; a node passes the acceptance test when theta > D_node/|c_i - g|
 * and then acts with its vertex count at its centroid g.
 *
 * Conventions for every call:
 *   - Status codes are returned, never abort(). bl_last_error() gives the text
 *     of the calling thread's last failure.
 *   - Host pointers are copied in; the caller keeps ownership. Output buffers
 *     belong to the caller; their capacity is checked (BL_EINVAL if short).
 *   - Handles belong to the library until the matching *_free call.
 *   - Work is queued on the stream set by bl_set_stream (default: the legacy
 *     default stream). Calls that return host data synchronise that stream.
 *   - Positions are FP32, interleaved x,y (2n floats). All force arithmetic is
 *     FP32; energies and quality metrics are accumulated in FP64.
 *   - Device memory comes from the allocator set by bl_set_allocator
 *     (default: cudaMalloc/cudaFree).
 */
#ifndef BATCHLAYOUT_H
#define BATCHLAYOUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BL_OK = 0,
    BL_EINVAL = 1,      /* bad argument, malformed CSR, short output buffer */
    BL_ENOMEM = 2,      /* device or host allocation failed */
    BL_EBUDGET = 3,     /* a request can never fit the server's memory budget */
    BL_ECUDA = 4,       /* a CUDA runtime call or kernel launch failed */
    BL_ETIMEOUT = 5,    /* a bounded device-side wait gave up (status word set) */
    BL_EBUSY = 6,       /* object in use by queued work */
    BL_ENOTREADY = 7,   /* serving: the result is not done yet */
    BL_ECANCELED = 8    /* serving: the request was cancelled */
} bl_status;

typedef enum {
    BL_EXACT = 0,       /* all-pairs repulsion (Algorithm 2) */
    BL_BH = 1,          /* Barnes-Hut repulsion (Algorithm S5) */
    BL_AUTO = 2         /* serving only: exact below 50,000 vertices, else BH */
} bl_mode;

/* CSR clean-up flags for bl_graph_load_csr */
#define BL_CSR_SYMMETRIZE 1u   /* add (j,i) for every (i,j) */
#define BL_CSR_DEDUP 2u        /* drop duplicate entries and self-loops */
#define BL_CSR_SORT 4u         /* sort each row (implied by the two above) */

typedef struct bl_graph bl_graph;
typedef struct bl_layout bl_layout;
typedef struct bl_server bl_server;

/* Force model parameters (Section 2.2). K: optimal spring length; R: relative
 * strength of repulsion. repulse_neighbors = 0 (default) repels non-adjacent
 * pairs only, as the combined force f(i,c) states; 1 repels every pair j != i,
 * as Algorithm S5's tree repulsion does literally. kahan: 1 = compensated (Kahan)
 * FP32 repulsion sums, 0 = plain FP32 sums, -1 (default) = compensated from
 * 1,000,000 vertices on; other values give BL_EINVAL. What is compensated: the
 * whole-GPU exact engine adds each row's column-tile partial sums (256 columns
 * at minibatch 256) with compensation; the one-cluster engine compensates every
 * term of each lane's strided sum; the batched kernel each stripe's folds of 32
 * columns; Barnes-Hut every node and leaf term of the walk. energy_model
 * picks the (a,r)-energy model, attraction |c_i - c_j|^a / K with repulsion
 * R K^2 / |c_i - c_j| (r = -1): BL_MODEL_FR (a = 2, Fruchterman-Reingold, the
 * default and the paper's reported model), BL_MODEL_FA (a = 1, ForceAtlas),
 * BL_MODEL_LINLOG (a = 0) or BL_MODEL_A3 (a = 3). */
typedef enum { BL_MODEL_FR = 0, BL_MODEL_FA = 1, BL_MODEL_LINLOG = 2, BL_MODEL_A3 = 3 } bl_energy_model;
typedef struct {
    float K;
    float R;
    int32_t repulse_neighbors;
    int32_t kahan;
    int32_t energy_model;   /* bl_energy_model; 0 = Fruchterman-Reingold */
} bl_force_params;

typedef struct {
    int64_t iterations;          /* iterations done so far (t of the schedule) */
    double step;                 /* Step of the next iteration = 0.999^t */
    double energy;               /* sum |ct_i|^2 of the last iteration (FP64) */
    double pair_interactions;    /* exact mode: n(n-1) per iteration, cumulative */
    double vertex_updates;       /* n per iteration, cumulative */
    double bh_far_nodes;         /* BH: accepted far-field nodes, last tree walk */
    double bh_near_pairs;        /* BH: leaf vertices visited (each query's own
                                    vertex included), last tree walk */
    double last_run_ms;          /* device time of the last bl_layout_run */
} bl_stats_t;

/* ---- runtime configuration ------------------------------------------------ */

/* Stream for all subsequent work of the calling process (a cudaStream_t cast
 * to void*; NULL = legacy default stream). */
bl_status bl_set_stream(void *stream);

/* Device allocator hooks. alloc(bytes, ctx) returns device memory or NULL;
 * dealloc(ptr, ctx) releases it. Pass NULLs to restore cudaMalloc/cudaFree.
 * Objects keep the hooks they were created with. */
bl_status bl_set_allocator(void *(*alloc)(size_t bytes, void *ctx),
                           void (*dealloc)(void *ptr, void *ctx), void *ctx);

const char *bl_last_error(void);
const char *bl_version(void);

/* ---- graph (Section 2.1: CSR rowptr[n+1], colids[nnz]) --------------------- */

/* Validates and uploads an undirected graph. Without flags the CSR must be
 * clean: rowptr[0] = 0, non-decreasing, rowptr[n] = nnz; colids in [0,n),
 * strictly increasing within a row (no duplicates), no self-loops, symmetric.
 * Flags repair what they name. int32 ids; n >= 1. */
bl_status bl_graph_load_csr(int32_t n, int64_t nnz, const int32_t *rowptr,
                            const int32_t *colids, uint32_t flags, bl_graph **out);
bl_status bl_graph_info(const bl_graph *g, int32_t *n, int64_t *nnz);
void bl_graph_free(bl_graph *g);

/* ---- one layout ------------------------------------------------------------ */

/* Creates the layout state of graph g (the graph must outlive it). Initial
 * positions: xy (2n floats, host) when non-NULL, else uniform in [-1,1)^2 from
 * SplitMix64 at `seed` (24 random bits per coordinate; coordinate k = 2i for
 * x_i, 2i+1 for y_i). start_iter sets t, so Step = 0.999^start_iter (resume).
 * params may be NULL (K = R = 1, non-neighbour repulsion, kahan automatic). */
bl_status bl_layout_init(const bl_graph *g, const float *xy, uint64_t seed, int64_t start_iter,
                         const bl_force_params *params, bl_layout **out);

/* Greedy initialisation (Section 3.6, Algorithm 3): a layout whose positions
 * come from a depth-first placement starting at v0 = (0, 0): each vertex U taken
 * from the stack puts its not yet placed neighbours, in CSR order, on the unit
 * circle around U at angles 0, d, 2d, ... degrees, d = 360/deg(U) (PI = 3.1416
 * as the paper prints it), formed in double and stored as FP32. v0 < 0 draws the
 * start vertex as SplitMix64(seed) output 0 mod n. Vertices outside v0's
 * component keep the seeded random positions of bl_layout_init(seed). Host-side
 * (the walk's order defines the layout); synchronises. */
bl_status bl_layout_init_greedy(const bl_graph *g, int64_t v0, uint64_t seed,
                                const bl_force_params *params, bl_layout **out);

/* Replaces the positions (host, 2n floats) and the iteration counter. */
bl_status bl_layout_set_positions(bl_layout *L, const float *xy, int64_t start_iter);

/* Runs `iters` iterations with minibatch size `batch` (1 <= batch <= 8192)
 * in mode BL_EXACT or BL_BH (theta: MAC threshold, the paper uses 1.2) —
 * Algorithm 2 with Section 2.2's forces, Algorithm S5 for BL_BH. Continues the
 * step schedule from the layout's iteration counter; runs of k and m
 * iterations give the same positions and energies, bit for bit, as one run of
 * k + m. Synchronises; BL_ETIMEOUT if a bounded device-side wait gave up.
 * BL_BH takes graphs of at most 126,322,567 vertices (its quadtree reserves
 * 17 n + 1 nodes with 32-bit indices); larger ones give BL_EINVAL. A BL_EXACT
 * call runs at most 2^31 - 1 minibatch steps (iters * ceil(n / batch)); a
 * longer run is split over several calls, with the same result. On the
 * whole-GPU exact engine a call that continues the previous exact call (same
 * batch, positions not replaced since) picks up the per-row repulsion sums that
 * call left on the device (about 32 bytes per vertex, held by the layout)
 * instead of recomputing them from the start positions. */
bl_status bl_layout_run(bl_layout *L, int32_t iters, int32_t batch, bl_mode mode, float theta);

/* Runs at most max_iters iterations and stops after the first iteration whose
 * energy differs from the previous one by at most tol * max(E_prev, 1) (Section
 * 4.5 runs until the difference is below 1e-6; read relatively). The previous
 * one may come from the layout's last run. The result equals stopping there
 * exactly: iterations run in chunks, and a chunk in which the rule holds is
 * rolled back and re-run to that iteration. *iters_done receives the iterations
 * run, *converged 1 if the rule held (both may be NULL); bl_energy_history then
 * returns the call's whole history. Synchronises. */
bl_status bl_layout_run_until(bl_layout *L, int32_t max_iters, int32_t batch, bl_mode mode,
                              float theta, double tol, int32_t *iters_done, int32_t *converged);

/* Copies positions to host (2n floats; cap_floats >= 2n). Synchronises. */
bl_status bl_positions(const bl_layout *L, float *xy, int64_t cap_floats);

/* Device pointer of the live positions (float2[n]); valid until the next
 * bl_layout_run or bl_layout_free. New positions written through it before the
 * next run are honoured (that run does not continue the previous exact launch's
 * carried sums). */
bl_status bl_positions_device(const bl_layout *L, void **dptr);

/* Energy of each iteration of the last bl_layout_run (FP64, Section 2.2's
 * sum_i |f(i,c)|^2). Synchronises. *count = iterations of that run; with
 * out == NULL only the count is returned. */
bl_status bl_energy_history(const bl_layout *L, double *out, int64_t cap, int64_t *count);

bl_status bl_stats(const bl_layout *L, bl_stats_t *out);
/* Frees the layout after the library's stream (bl_set_stream) has drained. */
void bl_layout_free(bl_layout *L);

/* ---- quality (Section 3.7) --------------------------------------------------- */

/* Layout quality as Section 3.7 measures it, of the current positions, in FP64
 * on the GPU:
 *  - stress sum_{pairs} (s*x_ij - d_ij)^2 / d_ij^2 at the scale s* that
 *    minimises it (x = layout distance, d = BFS hop distance; unreachable pairs
 *    skipped). nsources <= 0 or >= n: all unordered pairs. Otherwise the BFS
 *    sources are a seeded sample (below) and the ordered-pair sum is scaled by
 *    n / (2 nsources).
 *  - neighbourhood preservation, 1-hop reading: for each query i with deg(i) > 0,
 *    L_i = the deg(i) vertices nearest to i in the layout (squared distance in
 *    FP64 as dx*dx + dy*dy, ties by smaller id); NP = mean of
 *    |N(i) & L_i| / |N(i) | L_i|. nqueries <= 0 or >= n: every vertex; otherwise
 *    a seeded sample drawn with seed ^ 0x5bd1e995.
 *  - edge uniformity sqrt(sum_e (l_e - mean)^2 / (|E| mean^2)), each undirected
 *    edge once.
 * Seeded sample of m of n vertices: partial Fisher-Yates over 0..n-1 whose step
 * k swaps entries k and k + (z_k mod (n-k)), z_k = SplitMix64 output k of the
 * stream with state `seed` (as bl_layout_init); the sample is entries 0..m-1.
 * out (cap >= 6 doubles) = {stress, s*, stress pairs, NP, NP queries with
 * deg > 0, edge uniformity}; with cap >= 7, out[6] = total NP intersection size.
 * Allocates scratch (O(n) for stress, 12 B x n per SM for NP) through the
 * library allocator. Synchronises. */
bl_status bl_quality(const bl_layout *L, int32_t nsources, int32_t nqueries, uint64_t seed,
                     double *out, int64_t cap);

/* ---- many small graphs in one persistent launch ------------------------------ */

/* Lays out `count` graphs with initial positions from seeds[k] (as
 * bl_layout_init), `iters` iterations each, exact mode (BL_EXACT; BL_BH is
 * accepted and run one graph at a time). outs[k] receives a layout handle
 * that holds the result. One persistent kernel works through a vertex-block
 * work list of all graphs, in chunks of iterations replayed from a captured
 * CUDA graph. */
bl_status bl_layout_batch(const bl_graph *const *gs, int32_t count, const uint64_t *seeds,
                          int32_t iters, int32_t batch, bl_mode mode, float theta,
                          bl_layout **outs);

/* Continues `count` existing layouts by `iters` exact-mode iterations each
 * (Algorithm 2 per layout, Step continuing from each layout's own t), in the same
 * batched launch as bl_layout_batch. Graphs of at most 16,384 vertices with
 * batch <= 256 whose n^2 is at most the total work / SMs share the persistent
 * kernel (one CTA per graph, positions in shared memory); the others run one at a
 * time on the whole GPU. A graph's positions do not depend on which other graphs
 * share the launch, nor on the launch shape the autotuner picks (first call per
 * shared-memory size class; environment BL_BATCH_SHAPE=0..3 fixes it). The
 * environment variable BL_BATCH_CHUNK sets the iterations per captured launch.
 * Synchronises. */
bl_status bl_layout_run_batch(bl_layout *const *Ls, int32_t count, int32_t iters, int32_t batch);

/* ---- continuous-batching server -------------------------------------------- */

/* The paper lays out one graph per run; serving many requests is this library's
 * addition. A server owns a worker thread and a stream on the device current at
 * creation, and admits requests against mem_budget_bytes of working memory
 * (positions, energies, Barnes-Hut trees; the graphs themselves belong to the
 * caller). Each tick the worker admits queued requests in arrival order while
 * they fit the budget (whole-GPU jobs also need one of 4 slots), then advances
 * every admitted request: exact requests of at most 16,384 vertices, batch
 * <= 256 and n^2 x iters <= 2.5e9 share one persistent batched launch (50
 * iterations per tick); the others (larger exact, and BH) run a chunk whose
 * length depends only on the request, each on a stream of its own, so the chunks
 * and the batched launch of a tick overlap on the device. A finished layout is
 * copied to host memory and its device memory
 * returns to the budget at once. A request's result does not depend on what
 * else is being served. Device memory comes from the library allocator
 * (bl_set_allocator) in force at each allocation. */
bl_status bl_server_create(size_t mem_budget_bytes, bl_server **out);

/* Queues a layout of g (which must stay alive until polled) with seeded initial
 * positions (as bl_layout_init), `iters` iterations of minibatch `batch`. mode
 * BL_AUTO picks exact below 50,000 vertices and BH otherwise. BL_EBUDGET if the
 * request could never fit the budget; BL_EINVAL for a BH request over BH's
 * vertex limit (bl_layout_run). *ticket identifies the request. */
bl_status bl_serve_submit(bl_server *S, const bl_graph *g, uint64_t seed, int32_t iters,
                          int32_t batch, bl_mode mode, float theta, uint64_t *ticket);

/* Non-blocking. BL_ENOTREADY while queued or running; once done, copies 2n
 * floats to xy (cap checked), the latency (submit -> done, seconds) to
 * *latency_s, and retires the ticket. A canceled request answers BL_ECANCELED
 * and a failed one its error (e.g. BL_ETIMEOUT), both retiring the ticket. */
bl_status bl_serve_poll(bl_server *S, uint64_t ticket, float *xy, int64_t cap, double *latency_s);

/* Cancels a queued request (BL_EBUSY once it is on the GPU or finished). */
bl_status bl_serve_cancel(bl_server *S, uint64_t ticket);

/* out[0..5] = {completed, in flight, queued, bytes in use, p50 s, p99 s} over
 * the requests completed so far; with cap >= 7, out[6] = peak bytes in use. */
bl_status bl_server_stats(bl_server *S, double *out, int64_t cap);

/* Stops the worker (requests still queued or running are dropped) and frees
 * the server. */
void bl_server_free(bl_server *S);

/* ---- exact run without device allocations ------------------------------------ */

/* The paper has no counterpart to this call; it exists for callers that cannot
 * call cudaMalloc (an engine that hands out all device memory from its own pool,
 * a serving loop that must not stall on an allocation's implicit
 * synchronisation, a process under a hard device-memory quota).
 * Runs `iters` exact-mode iterations on the whole-GPU engine (the one
 * bl_layout_run uses for BL_EXACT above 3,072 vertices; for smaller graphs
 * bl_layout_run picks the one-cluster engine, whose results agree within the
 * exact-mode tolerance, not bit for bit) on buffers the caller owns, all device
 * pointers: d_rowptr[n+1] and
 * d_colids[nnz] a CSR that already satisfies bl_graph_load_csr's rules (not
 * checked here), d_xy[2n] positions (in/out), d_energy[iters] per-iteration
 * energy (out, may be NULL). params may be NULL (defaults as bl_layout_init);
 * start_iter sets Step = 0.999^start_iter. Work goes to `stream` (a
 * cudaStream_t, NULL = legacy default stream); the call synchronises it before
 * returning and reports BL_ETIMEOUT from the device-side waits.
 * Allocates nothing: the engine's working memory lives in one file-scope
 * device array of about 2 MiB that every GPU loading the library holds until
 * exit. Limits: n <= 131072 and iters x (CTAs, at most one per SM) <= 131072;
 * larger requests return BL_EINVAL, as do K or R not positive and finite. The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), and so does the first call after that device's
 * context has changed (cudaDeviceReset); make that first call before any
 * stream capture. All calls share the array: calls that overlap on the GPU
 * (other host threads, other streams) race and must be serialised by the
 * caller. */
bl_status bl_layout_run_noalloc(int32_t n, const int32_t *d_rowptr, const int32_t *d_colids,
                                float *d_xy, int32_t iters, int32_t batch,
                                const bl_force_params *params, int64_t start_iter,
                                double *d_energy, void *stream);

/* ---- failure-detection hook --------------------------------------------------- */

/* Test hook (the paper has no counterpart): runs the engines' bounded grid
 * barrier in a 2-CTA cooperative kernel that expects 3 CTAs, so the barrier can
 * never complete; each wait gives up after limit_ms (1..2000) and the call
 * returns BL_ETIMEOUT with the context still usable. Synchronises. */
bl_status bl_debug_barrier_timeout(int32_t limit_ms);

/* ---- parity hooks ------------------------------------------------------------ */

/* One-snapshot forces ct_i (FP32, 2 floats per vertex) for i in [lo, hi) from
 * the current positions, without moving any vertex: the exact engine's column
 * and CSR phases (mode BL_EXACT) or the tree walk plus CSR attraction
 * (mode BL_BH). f_out holds 2*(hi-lo) floats. Synchronises. */
bl_status bl_debug_forces(bl_layout *L, bl_mode mode, float theta, int32_t lo, int32_t hi,
                          float *f_out);

/* The Barnes-Hut tree of the current positions (Section 3.5, Algorithm S3),
 * built by the GPU: Morton codes in sorted order, the sorting permutation and
 * the pre-order node arrays first/count/level/skip plus FP32 coordinate sums.
 * Arrays hold `cap` nodes; *nnodes receives the node count (BL_EINVAL when cap
 * is short, after writing *nnodes). box = {xmin, ymin, D}. Synchronises. */
bl_status bl_debug_bh_tree(bl_layout *L, uint32_t *codes, int32_t *perm, int32_t *first,
                           int32_t *count, int32_t *level, int32_t *skip, float *sumx,
                           float *sumy, int64_t cap, int64_t *nnodes, float *box);

/* The acceptance decisions of the Barnes-Hut walk (Section 3.5's MAC,
 * Algorithm S4) query by query, on the tree of the current positions: far[i] =
 * far-field nodes accepted on vertex i's walk, near[i] = leaf vertices it met
 * (its own included). Arrays of cap >= n int32, indexed by vertex id.
 * Synchronises. */
bl_status bl_debug_bh_counts(bl_layout *L, float theta, int32_t *far, int32_t *near, int64_t cap);

/* ---- profiling hooks ---------------------------------------------------------- */

/* Records device phase timestamps (global timer, ns) for the first max_steps
 * minibatch steps of the next exact-mode bl_layout_run (0 turns it off). Per
 * CTA and step, 12 slots: control warp {0 step start, 1 previous batch
 * published by all CTAs, 2 column tile in shared memory, 3 bulk warps done with
 * the previous step, 9 first critical rows' column pass summed, 11 their CSR
 * terms summed, 4 critical rows moved, 6 arrival posted}; bulk warps {7 step
 * start, 5 moved rows picked up, 10 neighbours staged, 8 step done}. In BH mode
 * (any max_steps > 0) the last iteration's sweep is traced instead: the start
 * time of each of its dependency levels, then its end; with max_steps >= 2 these
 * are followed by three stamps per sweep task, in the sweep's task order (levels
 * in order; inside a level first the later segments of long rows, each at the
 * level after its own columns' highest, then the rows and first segments, each
 * group in row id order): {task start, its first earlier-minibatch positions
 * gathered, task done}. */
bl_status bl_set_trace(bl_layout *L, int32_t max_steps);

/* Phase timing of Barnes-Hut runs (profiling; the paper has no counterpart).
 * With on != 0, every later BL_BH bl_layout_run of L records CUDA events between
 * its phases (a little host work per iteration). bl_get_phase_times then gives,
 * for the last such run, out[0..8] = device milliseconds summed over its
 * iterations of {bounding box + Morton codes, radix sort, tree + node sums,
 * theta-walk, wait for the edge pass, minibatch sweep (first level + dataflow),
 * energy, edge pass (side stream, overlapping the tree and walk), whole
 * iteration}, out[9] = nodes of the last tree, out[10] = node records read by the
 * queries of the last walk (one per node a query visits), out[11] = iterations
 * of that run (cap >= 12). */
bl_status bl_set_phase_timing(bl_layout *L, int32_t on);

/* Ceiling probes of the exact pair loop (profiling; the paper has no
 * counterpart). On every SM, `threads` threads (a multiple of 32 up to 512) each
 * run one row against a 256-column tile in shared memory with the exact engine's
 * packed pair loop, 400 times; with skip_sp0 != 0 the warps of sub-partition 0
 * (warp index % 4 == 0) sit out. Then 512 threads per SM run 8 independent chains
 * of rcp.approx(x/2 + 1). out[0] = pair interactions per clock per SM (longest warp's
 * clock64 span), out[1] = reciprocal lanes per clock per SM (CUDA events, at the
 * clock of out[3]), out[2] = the pair kernel's device milliseconds (CUDA events),
 * out[3] = the SM clock those imply (MHz). cap >= 4. Allocates and frees its
 * scratch; synchronises. */
bl_status bl_measure_pair_rate(int32_t threads, int32_t skip_sp0, double *out, int64_t cap);
bl_status bl_get_phase_times(const bl_layout *L, double *out, int64_t cap);

/* Copies the trace of the last traced run: [CTAs][max_steps][12] uint64
 * (exact mode) or [levels + 1] uint64, then [tasks][3] with max_steps >= 2
 * (BH mode).
 * *count = entries; with out == NULL only the count. Synchronises. */
bl_status bl_get_trace(const bl_layout *L, uint64_t *out, int64_t cap, int64_t *count);

#ifdef __cplusplus
}
#endif

#endif /* BATCHLAYOUT_H */
