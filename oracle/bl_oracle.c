/*
 * FP64 CPU oracle for BatchLayout (Rahman, Sujon, Azad; arXiv 2002.08233).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, sequential statement
 * of what the layout method computes. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the library's product path
 * never does. It shares no code, header or table with the CUDA sources.
 *
 * Passages followed (section / equation / algorithm of the paper):
 *   - force law f_a, f_r and the combined force f(i,c): Section 2.2
 *   - the sequential loop and step schedule: Algorithm 1
 *   - minibatch semantics, the update c_i += Step*ct_i/|ct_i|, the energy
 *     sum and Step *= 0.999: Section 3.3 and Algorithm 2
 *   - Barnes-Hut: quadtree and centroids (Section 3.5, Fig. 3), Morton order
 *     (Fig. 4), MAC theta > D/|c_i - c_j| (Section 3.5), theta = 1.2
 *     (Section 4.1), constructBHT / calcRepulsiveForce / BatchLayoutBH
 *     (Algorithms S3, S4, S5 of the supplement)
 *   - quality metrics: stress, edge uniformity, neighbourhood preservation
 *     (Section 3.7)
 *
 * Readings taken where the paper is silent, garbled or ambiguous:
 *   R1  FR model (2,-1): attraction magnitude d^2/K, repulsion magnitude
 *       R*K^2/d, directed along the unit vector; the printed exponent sign of
 *       f_r is garbled (with d^r, r=-1 repulsion would grow with d).
 *   R2  Repulsion set: by default non-neighbours only (Section 2.2, the else
 *       branch of Algorithm 2). repulse_neighbors=1 takes repulsion over all
 *       j != i, which is what Algorithm S5's tree repulsion does literally.
 *       In BH mode with repulse_neighbors=0 the exact neighbour terms, taken
 *       at the tree's snapshot positions, are removed from the tree sum.
 *   R3  K = R = 1 by default (parameters).
 *   R4  n not a multiple of BS: the last batch is partial.
 *   R5  |ct| = 0 -> no move; a pair at distance 0 (j != i) contributes 0.
 *   R6  Algorithm S5 omits Step *= 0.999: Algorithm 2's schedule is used.
 *   R7  BH tree built once per iteration from the snapshot S of the positions
 *       at iteration start (Algorithm S5 builds it before the batch loop);
 *       attraction uses the live positions.
 *   R8  Algorithm S5's bounding-box rescaling does not move vertices: the box only
 *       quantises positions to Morton codes; the root square has side
 *       D = max(xmax-xmin, ymax-ymin) anchored at (xmin, ymin).
 *   R9  Morton codes in FP32, no contraction: s = 65536/D;
 *       q = min(65535, floor((x - xmin) * s)); code = spread(qx)|spread(qy)<<1.
 *       D == 0 (or not finite) gives code 0 for every vertex. Stable sort by
 *       code (ties by vertex id).
 *   R10 A node exists for every non-empty cell whose parent is not a leaf; a
 *       node is a leaf iff it holds one vertex or sits at level 16. Nodes are
 *       listed in pre-order, children in code order.
 *   R11 Node coordinate sums are FP32: a leaf adds its vertices in sorted order
 *       starting from 0; an inner node adds its children's sums in child
 *       order starting from the first child's sum. Centroid = sum / count
 *       (FP32, correctly rounded). The far field of an accepted node is
 *       count * f_r towards the centroid (the "f_a" in Algorithm S4's MAC
 *       branch is read as f_r).
 *   R12 MAC in FP32: Dl = D * 2^-level, dx = gx - xi, dy = gy - yi,
 *       d2 = fmaf(dy, dy, dx*dx); accept iff Dl*Dl < (theta*theta)*d2.
 *       Leaves always sum their vertices directly (each with its own
 *       distance); vertex i itself is skipped by index. There is no
 *       containment test.
 *   R19 (a,r)-energy models (Section 2.2; Section 4.1 says the software has
 *       four variants from the ForceAtlas2 paper): attraction magnitude
 *       d^a / K for a in {0, 1, 2, 3}, repulsion as R1 (r = -1), i.e. LinLog
 *       (0,-1), ForceAtlas (1,-1), Fruchterman-Reingold (2,-1) and (3,-1).
 *       d^a is formed by repeated multiplication.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

#define ORC_EXACT 0
#define ORC_BH 1
#define ORC_LEVELS 16

/* -------------------------------------------------------------------------- */
/* Force law, Section 2.2 (reading R1)                                         */
/* -------------------------------------------------------------------------- */

/* f_a(i,j) * (c_j - c_i)/|c_i - c_j| with f_a = |c_i - c_j|^a / K (the
 * (a,r)-energy model of Section 2.2; a = 2 is Fruchterman-Reingold, R1/R19) */
static void attractive_term(double xi, double yi, double xj, double yj, double K, int a,
                            double *tx, double *ty)
{
    double dx = xj - xi, dy = yj - yi;
    double d = sqrt(dx * dx + dy * dy);
    if (d == 0.0) { *tx = 0.0; *ty = 0.0; return; }
    double fa = 1.0;
    for (int k = 0; k < a; k++) fa *= d;
    fa /= K;
    *tx = fa * dx / d;
    *ty = fa * dy / d;
}

/* f_r(i,j) * (c_j - c_i)/|c_i - c_j| with f_r = -R K^2 / |c_i - c_j| */
static void repulsive_term(double xi, double yi, double xj, double yj, double K, double R,
                           double *tx, double *ty)
{
    double dx = xj - xi, dy = yj - yi;
    double d = sqrt(dx * dx + dy * dy);
    if (d == 0.0) { *tx = 0.0; *ty = 0.0; return; }
    double fr = -R * K * K / d;
    *tx = fr * dx / d;
    *ty = fr * dy / d;
}

/* -------------------------------------------------------------------------- */
/* Exact combined force f(i,c) (Section 2.2; Algorithm 2's inner loops)        */
/* -------------------------------------------------------------------------- */

static void exact_force(int i, int n, const int *rowptr, const int *colids, const double *xy,
                        double K, double R, int a, int repulse_neighbors,
                        double *fx, double *fy, double *mag)
{
    double sx = 0.0, sy = 0.0, m = 0.0, tx, ty;
    int k = rowptr[i], kend = rowptr[i + 1];
    double xi = xy[2 * i], yi = xy[2 * i + 1];
    for (int j = 0; j < n; j++) {
        int is_edge = 0;
        if (k < kend && colids[k] == j) { is_edge = 1; k++; }   /* merge of sorted colids */
        if (is_edge) {
            attractive_term(xi, yi, xy[2 * j], xy[2 * j + 1], K, a, &tx, &ty);
            sx += tx; sy += ty; m += sqrt(tx * tx + ty * ty);
        }
        if (j != i && (!is_edge || repulse_neighbors)) {
            repulsive_term(xi, yi, xy[2 * j], xy[2 * j + 1], K, R, &tx, &ty);
            sx += tx; sy += ty; m += sqrt(tx * tx + ty * ty);
        }
    }
    *fx = sx; *fy = sy;
    if (mag) *mag = m;
}

/* -------------------------------------------------------------------------- */
/* Barnes-Hut: Morton codes (R8, R9), tree (Algorithm S3, R10, R11)            */
/* -------------------------------------------------------------------------- */

typedef struct {
    float xmin, ymin, D;
} orc_box;

static uint32_t spread16(uint32_t v)
{
    /* bit b of v goes to bit 2b of the result */
    uint32_t r = 0;
    for (int b = 0; b < 16; b++) r |= ((v >> b) & 1u) << (2 * b);
    return r;
}

static orc_box morton_codes(int n, const float *xf, const float *yf, uint32_t *codes)
{
    orc_box box = {0.0f, 0.0f, 0.0f};
    if (n <= 0) return box;
    float xmin = xf[0], xmax = xf[0], ymin = yf[0], ymax = yf[0];
    for (int i = 1; i < n; i++) {
        if (xf[i] < xmin) xmin = xf[i];
        if (xf[i] > xmax) xmax = xf[i];
        if (yf[i] < ymin) ymin = yf[i];
        if (yf[i] > ymax) ymax = yf[i];
    }
    float dxr = xmax - xmin, dyr = ymax - ymin;
    float D = dxr > dyr ? dxr : dyr;
    box.xmin = xmin; box.ymin = ymin; box.D = D;
    if (!(D > 0.0f) || !isfinite(D)) {
        for (int i = 0; i < n; i++) codes[i] = 0u;
        return box;
    }
    float s = 65536.0f / D;
    for (int i = 0; i < n; i++) {
        float tx = (xf[i] - xmin) * s;
        float ty = (yf[i] - ymin) * s;
        uint32_t qx = (uint32_t)floorf(tx);
        uint32_t qy = (uint32_t)floorf(ty);
        if (qx > 65535u) qx = 65535u;
        if (qy > 65535u) qy = 65535u;
        codes[i] = spread16(qx) | (spread16(qy) << 1);
    }
    return box;
}

typedef struct {
    uint32_t code;
    int id;
} keyed;

static int cmp_keyed(const void *a, const void *b)
{
    const keyed *p = (const keyed *)a, *q = (const keyed *)b;
    if (p->code != q->code) return p->code < q->code ? -1 : 1;
    return (p->id > q->id) - (p->id < q->id);
}

typedef struct {
    int first, count, level, skip;
    int nchild, child[4];
    float sx, sy;      /* FP32 coordinate sums (R11) */
    float gx, gy;      /* FP32 centroid */
} onode;

typedef struct {
    int n, nnodes, cap;
    onode *nodes;
    int *perm;          /* sorted position -> vertex id */
    uint32_t *scodes;   /* sorted codes */
    const float *xf, *yf;
    orc_box box;
} otree;

static int tree_push(otree *t)
{
    if (t->nnodes == t->cap) {
        int nc = t->cap ? 2 * t->cap : 64;
        onode *p = (onode *)realloc(t->nodes, (size_t)nc * sizeof(onode));
        if (!p) return -1;
        t->nodes = p; t->cap = nc;
    }
    memset(&t->nodes[t->nnodes], 0, sizeof(onode));
    return t->nnodes++;
}

/* constructBHT (Algorithm S3): the cell holding sorted positions [lo, hi) at
 * `level`; split into the four quadrants of the next level in code order. */
static int construct(otree *t, int lo, int hi, int level)
{
    int v = tree_push(t);
    if (v < 0) return -1;
    t->nodes[v].first = lo;
    t->nodes[v].count = hi - lo;
    t->nodes[v].level = level;
    if (hi - lo == 1 || level == ORC_LEVELS) {
        float sx = 0.0f, sy = 0.0f;
        for (int k = lo; k < hi; k++) {
            sx = sx + t->xf[t->perm[k]];
            sy = sy + t->yf[t->perm[k]];
        }
        t->nodes[v].sx = sx;
        t->nodes[v].sy = sy;
    } else {
        int shift = 30 - 2 * level;          /* bits of the quadrant at level+1 */
        int a = lo;
        int kids[4], nk = 0;
        for (uint32_t q = 0; q < 4; q++) {
            int b = a;
            while (b < hi && ((t->scodes[b] >> shift) & 3u) == q) b++;
            if (b > a) {
                int c = construct(t, a, b, level + 1);
                if (c < 0) return -1;
                kids[nk++] = c;
            }
            a = b;
        }
        /* construct() may have moved t->nodes */
        t->nodes[v].nchild = nk;
        float sx = t->nodes[kids[0]].sx, sy = t->nodes[kids[0]].sy;
        for (int c = 1; c < nk; c++) {
            sx = sx + t->nodes[kids[c]].sx;
            sy = sy + t->nodes[kids[c]].sy;
        }
        for (int c = 0; c < nk; c++) t->nodes[v].child[c] = kids[c];
        t->nodes[v].sx = sx;
        t->nodes[v].sy = sy;
    }
    t->nodes[v].gx = t->nodes[v].sx / (float)t->nodes[v].count;
    t->nodes[v].gy = t->nodes[v].sy / (float)t->nodes[v].count;
    t->nodes[v].skip = t->nnodes;
    return v;
}

static void tree_free(otree *t)
{
    free(t->nodes); free(t->perm); free(t->scodes);
    memset(t, 0, sizeof(*t));
}

static int tree_build(otree *t, int n, const float *xf, const float *yf)
{
    memset(t, 0, sizeof(*t));
    t->n = n; t->xf = xf; t->yf = yf;
    if (n <= 0) return ORC_OK;
    uint32_t *codes = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    keyed *kv = (keyed *)malloc((size_t)n * sizeof(keyed));
    t->perm = (int *)malloc((size_t)n * sizeof(int));
    t->scodes = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!codes || !kv || !t->perm || !t->scodes) { free(codes); free(kv); tree_free(t); return ORC_ENOMEM; }
    t->box = morton_codes(n, xf, yf, codes);
    for (int i = 0; i < n; i++) { kv[i].code = codes[i]; kv[i].id = i; }
    qsort(kv, (size_t)n, sizeof(keyed), cmp_keyed);
    for (int k = 0; k < n; k++) { t->perm[k] = kv[k].id; t->scodes[k] = kv[k].code; }
    free(codes); free(kv);
    if (construct(t, 0, n, 0) < 0) { tree_free(t); return ORC_ENOMEM; }
    return ORC_OK;
}

/* MAC (Section 3.5; R12), evaluated in FP32 */
static int mac_accept(const otree *t, const onode *v, float xi, float yi, float theta)
{
    float Dl = ldexpf(t->box.D, -v->level);
    float dx = v->gx - xi;
    float dy = v->gy - yi;
    float d2 = fmaf(dy, dy, dx * dx);
    float th2 = theta * theta;
    return (Dl * Dl) < (th2 * d2);
}

/* calcRepulsiveForce (Algorithm S4): repulsion on vertex i from the subtree v. */
static void tree_repulsion(const otree *t, int v, int i, double xi, double yi, float xif, float yif,
                           float theta, double K, double R, double *fx, double *fy, double *mag)
{
    const onode *nd = &t->nodes[v];
    double tx, ty;
    int leaf = (nd->count == 1 || nd->level == ORC_LEVELS);
    if (leaf) {
        for (int k = nd->first; k < nd->first + nd->count; k++) {
            int j = t->perm[k];
            if (j == i) continue;
            repulsive_term(xi, yi, (double)t->xf[j], (double)t->yf[j], K, R, &tx, &ty);
            *fx += tx; *fy += ty; *mag += sqrt(tx * tx + ty * ty);
        }
        return;
    }
    if (mac_accept(t, nd, xif, yif, theta)) {
        repulsive_term(xi, yi, (double)nd->gx, (double)nd->gy, K, R, &tx, &ty);
        tx *= (double)nd->count; ty *= (double)nd->count;
        *fx += tx; *fy += ty; *mag += sqrt(tx * tx + ty * ty);
        return;
    }
    for (int c = 0; c < nd->nchild; c++)
        tree_repulsion(t, nd->child[c], i, xi, yi, xif, yif, theta, K, R, fx, fy, mag);
}

/* BH force on i: attraction at positions `live`; repulsion from the tree built
 * on the snapshot, minus exact neighbour terms at the snapshot unless
 * repulse_neighbors (R2, R7). */
static void bh_force(int i, const int *rowptr, const int *colids, const double *live,
                     const otree *t, float theta, double K, double R, int a, int repulse_neighbors,
                     double *fx, double *fy, double *mag)
{
    double sx = 0.0, sy = 0.0, m = 0.0, tx, ty;
    double xi = live[2 * i], yi = live[2 * i + 1];
    for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
        int j = colids[k];
        attractive_term(xi, yi, live[2 * j], live[2 * j + 1], K, a, &tx, &ty);
        sx += tx; sy += ty; m += sqrt(tx * tx + ty * ty);
    }
    double rx = 0.0, ry = 0.0, rm = 0.0;
    double sxi = (double)t->xf[i], syi = (double)t->yf[i];
    if (t->nnodes > 0)
        tree_repulsion(t, 0, i, sxi, syi, t->xf[i], t->yf[i], theta, K, R, &rx, &ry, &rm);
    if (!repulse_neighbors) {
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int j = colids[k];
            repulsive_term(sxi, syi, (double)t->xf[j], (double)t->yf[j], K, R, &tx, &ty);
            rx -= tx; ry -= ty;
        }
    }
    *fx = sx + rx; *fy = sy + ry;
    if (mag) *mag = m + rm;
}

/* -------------------------------------------------------------------------- */
/* Public entry points                                                         */
/* -------------------------------------------------------------------------- */

static int check_csr(int n, const int *rowptr, const int *colids)
{
    if (n < 0 || !rowptr) return ORC_EINVAL;
    if (rowptr[0] != 0) return ORC_EINVAL;
    for (int i = 0; i < n; i++) {
        if (rowptr[i + 1] < rowptr[i]) return ORC_EINVAL;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            if (colids[k] < 0 || colids[k] >= n) return ORC_EINVAL;
            if (k > rowptr[i] && colids[k] <= colids[k - 1]) return ORC_EINVAL;
        }
    }
    return ORC_OK;
}

/* One-snapshot forces f(i, c) for i in [lo, hi), all from the same positions xy
 * (FP64, interleaved x,y). f_out[2*(i-lo)+{0,1}]; mag_out[i-lo] = sum of the
 * magnitudes of the terms that make up f(i,c). mode 0: exact, 1: BH (tree on
 * the FP32-rounded positions). nthreads > 1 spreads the vertices over OpenMP
 * threads; results do not depend on it. */
int orc_forces(int n, const int *rowptr, const int *colids, const double *xy,
               double K, double R, int a, int repulse_neighbors, int mode, double theta,
               int lo, int hi, int nthreads, double *f_out, double *mag_out)
{
    if (a < 0 || a > 3) return ORC_EINVAL;
    if (check_csr(n, rowptr, colids) != ORC_OK) return ORC_EINVAL;
    if (lo < 0 || hi > n || lo > hi) return ORC_EINVAL;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    if (mode == ORC_EXACT) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) if (nthreads > 1)
#endif
        for (int i = lo; i < hi; i++)
            exact_force(i, n, rowptr, colids, xy, K, R, a, repulse_neighbors,
                        &f_out[2 * (i - lo)], &f_out[2 * (i - lo) + 1], mag_out ? &mag_out[i - lo] : NULL);
        return ORC_OK;
    }
    float *xf = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    float *yf = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    if (!xf || !yf) { free(xf); free(yf); return ORC_ENOMEM; }
    for (int i = 0; i < n; i++) { xf[i] = (float)xy[2 * i]; yf[i] = (float)xy[2 * i + 1]; }
    otree t;
    int rc = tree_build(&t, n, xf, yf);
    if (rc == ORC_OK) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) if (nthreads > 1)
#endif
        for (int i = lo; i < hi; i++)
            bh_force(i, rowptr, colids, xy, &t, (float)theta, K, R, a, repulse_neighbors,
                     &f_out[2 * (i - lo)], &f_out[2 * (i - lo) + 1], mag_out ? &mag_out[i - lo] : NULL);
    }
    tree_free(&t);
    free(xf); free(yf);
    return rc;
}

/* Algorithm 2 (exact) / Algorithm S5 (BH): `iters` iterations of minibatches of
 * size BS in vertex-id order on positions xy (FP64, updated in place). The
 * step starts at 0.999^start_iter (Step = 1.0 then Step *= 0.999 per
 * iteration). energy_out[t] (may be NULL) receives sum_i |ct_i|^2 of iteration t.
 * nthreads > 1 parallelises the force loop of each minibatch (Algorithm 2's
 * ParFor); results do not depend on it. */
int orc_run(int n, const int *rowptr, const int *colids, double *xy,
            int iters, int BS, int mode, double theta, double K, double R, int a,
            int repulse_neighbors, long long start_iter, int nthreads, double *energy_out)
{
    if (a < 0 || a > 3) return ORC_EINVAL;
    if (check_csr(n, rowptr, colids) != ORC_OK) return ORC_EINVAL;
    if (iters < 0 || BS <= 0 || start_iter < 0) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    double step = 1.0;
    for (long long s = 0; s < start_iter; s++) step *= 0.999;
    double *ct = (double *)malloc((size_t)2 * (size_t)(BS < n ? BS : n) * sizeof(double));
    float *xf = (float *)malloc((size_t)n * sizeof(float));
    float *yf = (float *)malloc((size_t)n * sizeof(float));
    if (!ct || !xf || !yf) { free(ct); free(xf); free(yf); return ORC_ENOMEM; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int rc = ORC_OK;
    for (int t = 0; t < iters && rc == ORC_OK; t++) {
        double energy = 0.0;
        otree tree;
        memset(&tree, 0, sizeof(tree));
        if (mode == ORC_BH) {
            /* snapshot S of iteration start, rounded to FP32 for the tree (R7) */
            for (int i = 0; i < n; i++) { xf[i] = (float)xy[2 * i]; yf[i] = (float)xy[2 * i + 1]; }
            rc = tree_build(&tree, n, xf, yf);
            if (rc != ORC_OK) break;
        }
        int nb = (n + BS - 1) / BS;
        for (int b = 0; b < nb; b++) {
            int lo = b * BS, hi = lo + BS < n ? lo + BS : n;
            /* forces of the whole minibatch from the same positions */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (nthreads > 1)
#endif
            for (int i = lo; i < hi; i++) {
                if (mode == ORC_EXACT)
                    exact_force(i, n, rowptr, colids, xy, K, R, a, repulse_neighbors,
                                &ct[2 * (i - lo)], &ct[2 * (i - lo) + 1], NULL);
                else
                    bh_force(i, rowptr, colids, xy, &tree, (float)theta, K, R, a, repulse_neighbors,
                             &ct[2 * (i - lo)], &ct[2 * (i - lo) + 1], NULL);
            }
            /* then the update of the minibatch */
            for (int i = lo; i < hi; i++) {
                double fx = ct[2 * (i - lo)], fy = ct[2 * (i - lo) + 1];
                double nf = sqrt(fx * fx + fy * fy);
                if (nf > 0.0) {
                    xy[2 * i] += step * fx / nf;
                    xy[2 * i + 1] += step * fy / nf;
                }
                energy += nf * nf;
            }
        }
        if (mode == ORC_BH) tree_free(&tree);
        if (energy_out) energy_out[t] = energy;
        step *= 0.999;
    }
    free(ct); free(xf); free(yf);
    return rc;
}

/* Morton codes of FP32 positions (R9). box_out = {xmin, ymin, D}. */
int orc_morton(int n, const float *xf, const float *yf, uint32_t *codes, float *box_out)
{
    if (n < 0) return ORC_EINVAL;
    orc_box b = morton_codes(n, xf, yf, codes);
    if (box_out) { box_out[0] = b.xmin; box_out[1] = b.ymin; box_out[2] = b.D; }
    return ORC_OK;
}

/* The quadtree of Algorithm S3 on FP32 positions, flattened in pre-order.
 * perm[k] = vertex at sorted position k; scodes[k] its code. Node arrays hold
 * up to `cap` nodes; *nnodes receives the count (ORC_EINVAL when cap is short). */
int orc_bh_tree(int n, const float *xf, const float *yf, int *perm, uint32_t *scodes,
                int cap, int *first, int *count, int *level, int *skip,
                float *sumx, float *sumy, int *nnodes)
{
    otree t;
    int rc = tree_build(&t, n, xf, yf);
    if (rc != ORC_OK) return rc;
    *nnodes = t.nnodes;
    if (t.nnodes > cap) { tree_free(&t); return ORC_EINVAL; }
    for (int k = 0; k < n; k++) { perm[k] = t.perm[k]; scodes[k] = t.scodes[k]; }
    for (int v = 0; v < t.nnodes; v++) {
        first[v] = t.nodes[v].first; count[v] = t.nodes[v].count;
        level[v] = t.nodes[v].level; skip[v] = t.nodes[v].skip;
        sumx[v] = t.nodes[v].sx; sumy[v] = t.nodes[v].sy;
    }
    tree_free(&t);
    return ORC_OK;
}

/* Per-query MAC statistics of the BH walk at theta: accepted far-field nodes
 * and directly summed leaf vertices (for reporting interactions). */
static void walk_counts(const otree *t, int v, float xif, float yif, float theta,
                        long long *far_nodes, long long *near_pairs)
{
    const onode *nd = &t->nodes[v];
    int leaf = (nd->count == 1 || nd->level == ORC_LEVELS);
    if (leaf) { *near_pairs += nd->count; return; }
    if (mac_accept(t, nd, xif, yif, theta)) { (*far_nodes)++; return; }
    for (int c = 0; c < nd->nchild; c++) walk_counts(t, nd->child[c], xif, yif, theta, far_nodes, near_pairs);
}

int orc_bh_interactions(int n, const float *xf, const float *yf, double theta,
                        long long *far_nodes, long long *near_pairs)
{
    otree t;
    int rc = tree_build(&t, n, xf, yf);
    if (rc != ORC_OK) return rc;
    *far_nodes = 0; *near_pairs = 0;
    for (int i = 0; i < n && t.nnodes > 0; i++)
        walk_counts(&t, 0, xf[i], yf[i], (float)theta, far_nodes, near_pairs);
    tree_free(&t);
    return ORC_OK;
}

/* The same MAC decisions query by query: far_out[i] = far-field nodes accepted on
 * vertex i's walk, near_out[i] = leaf vertices it met (its own included). */
int orc_bh_query_counts(int n, const float *xf, const float *yf, double theta,
                        int *far_out, int *near_out)
{
    otree t;
    int rc = tree_build(&t, n, xf, yf);
    if (rc != ORC_OK) return rc;
    for (int i = 0; i < n; i++) {
        long long f = 0, m = 0;
        if (t.nnodes > 0) walk_counts(&t, 0, xf[i], yf[i], (float)theta, &f, &m);
        far_out[i] = (int)f;
        near_out[i] = (int)m;
    }
    tree_free(&t);
    return ORC_OK;
}

/* -------------------------------------------------------------------------- */
/* Quality metrics, Section 3.7                                                */
/* -------------------------------------------------------------------------- */

static int bfs(int n, const int *rowptr, const int *colids, int src, int *dist, int *queue)
{
    for (int i = 0; i < n; i++) dist[i] = -1;
    int head = 0, tail = 0;
    dist[src] = 0; queue[tail++] = src;
    while (head < tail) {
        int u = queue[head++];
        for (int k = rowptr[u]; k < rowptr[u + 1]; k++) {
            int v = colids[k];
            if (dist[v] < 0) { dist[v] = dist[u] + 1; queue[tail++] = v; }
        }
    }
    return tail;
}

/* Stress: sum over pairs with finite hop distance d of w (|c_i - c_j| - d)^2,
 * w = d^-2, minimised over a uniform scale s of the layout. With x = |c_i-c_j|:
 * stress(s) = sum (s x/d - 1)^2, minimised at s* = sum(x/d) / sum(x^2/d^2).
 * Sources: all vertices when srcs == NULL (pairs i<j), else the listed sources,
 * each against every j != src (ordered pairs from the samples, scaled by
 * n / nsrc / 2 to the unordered all-pairs estimate).
 * out = {stress at s*, s*, number of pairs used}. Positions are FP32. */
int orc_stress(int n, const int *rowptr, const int *colids, const float *xy,
               int nsrc, const int *srcs, double *out)
{
    if (check_csr(n, rowptr, colids) != ORC_OK) return ORC_EINVAL;
    int *dist = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    int *queue = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    if (!dist || !queue) { free(dist); free(queue); return ORC_ENOMEM; }
    double a = 0.0, b = 0.0, pairs = 0.0;   /* a = sum x/d, b = sum x^2/d^2 */
    int ns = srcs ? nsrc : n;
    for (int s = 0; s < ns; s++) {
        int src = srcs ? srcs[s] : s;
        bfs(n, rowptr, colids, src, dist, queue);
        for (int j = 0; j < n; j++) {
            if (j == src || dist[j] <= 0) continue;
            if (!srcs && j < src) continue;
            double dx = (double)xy[2 * j] - (double)xy[2 * src];
            double dy = (double)xy[2 * j + 1] - (double)xy[2 * src + 1];
            double x = sqrt(dx * dx + dy * dy);
            double d = (double)dist[j];
            a += x / d;
            b += (x / d) * (x / d);
            pairs += 1.0;
        }
    }
    free(dist); free(queue);
    double sstar = b > 0.0 ? a / b : 0.0;
    double stress = pairs - (b > 0.0 ? a * a / b : 0.0);
    if (srcs && ns > 0) { stress *= (double)n / (double)ns / 2.0; }
    out[0] = stress; out[1] = sstar; out[2] = pairs;
    return ORC_OK;
}

/* Edge uniformity: sqrt( sum_e (l_e - l_mu)^2 / (|E| l_mu^2) ), each undirected
 * edge once (i < j). */
int orc_edge_uniformity(int n, const int *rowptr, const int *colids, const float *xy, double *out)
{
    if (check_csr(n, rowptr, colids) != ORC_OK) return ORC_EINVAL;
    double sum = 0.0; long long m = 0;
    for (int i = 0; i < n; i++)
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int j = colids[k];
            if (j <= i) continue;
            double dx = (double)xy[2 * j] - (double)xy[2 * i];
            double dy = (double)xy[2 * j + 1] - (double)xy[2 * i + 1];
            sum += sqrt(dx * dx + dy * dy); m++;
        }
    if (m == 0) { out[0] = 0.0; return ORC_OK; }
    double mu = sum / (double)m, var = 0.0;
    for (int i = 0; i < n; i++)
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int j = colids[k];
            if (j <= i) continue;
            double dx = (double)xy[2 * j] - (double)xy[2 * i];
            double dy = (double)xy[2 * j + 1] - (double)xy[2 * i + 1];
            double l = sqrt(dx * dx + dy * dy);
            var += (l - mu) * (l - mu);
        }
    out[0] = sqrt(var / ((double)m * mu * mu));
    return ORC_OK;
}

typedef struct { double d2; int id; } dist_id;

static int cmp_dist_id(const void *a, const void *b)
{
    const dist_id *p = (const dist_id *)a, *q = (const dist_id *)b;
    if (p->d2 != q->d2) return p->d2 < q->d2 ? -1 : 1;
    return (p->id > q->id) - (p->id < q->id);
}

/* Neighbourhood preservation, 1-hop reading: for each query i with deg(i) > 0,
 * L_i = the deg(i) layout-nearest vertices j != i (squared distance in FP64,
 * ties by id); J_i = |N(i) & L_i| / |N(i) | L_i|; NP = mean of J_i.
 * Queries: all vertices (queries == NULL) or the listed ones.
 * out = {NP, number of queries with deg > 0, sum of intersections}. */
int orc_neighborhood_preservation(int n, const int *rowptr, const int *colids, const float *xy,
                                  int nq, const int *queries, double *out)
{
    if (check_csr(n, rowptr, colids) != ORC_OK) return ORC_EINVAL;
    dist_id *buf = (dist_id *)malloc((size_t)(n > 0 ? n : 1) * sizeof(dist_id));
    char *mark = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!buf || !mark) { free(buf); free(mark); return ORC_ENOMEM; }
    double acc = 0.0, inter_total = 0.0; long long used = 0;
    int total = queries ? nq : n;
    for (int q = 0; q < total; q++) {
        int i = queries ? queries[q] : q;
        int deg = rowptr[i + 1] - rowptr[i];
        if (deg == 0) continue;
        int m = 0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = (double)xy[2 * j] - (double)xy[2 * i];
            double dy = (double)xy[2 * j + 1] - (double)xy[2 * i + 1];
            buf[m].d2 = dx * dx + dy * dy; buf[m].id = j; m++;
        }
        qsort(buf, (size_t)m, sizeof(dist_id), cmp_dist_id);
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) mark[colids[k]] = 1;
        int inter = 0;
        for (int k = 0; k < deg && k < m; k++) inter += mark[buf[k].id];
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) mark[colids[k]] = 0;
        int uni = deg + (deg < m ? deg : m) - inter;
        acc += (double)inter / (double)uni;
        inter_total += inter;
        used++;
    }
    free(buf); free(mark);
    out[0] = used ? acc / (double)used : 0.0;
    out[1] = (double)used;
    out[2] = inter_total;
    return ORC_OK;
}

/* -------------------------------------------------------------------------- */
/* Greedy initialisation, Algorithm 3                                          */
/* -------------------------------------------------------------------------- */

/* DFS with an explicit stack from vertex v0 placed at (0,0): a popped vertex U
 * places its unvisited neighbours on the unit circle around U at angles
 * 0, d, 2d, ... degrees with d = 360/deg(U). PI is the paper's 3.1416.
 * Vertices not reached from v0 keep the positions already in xy. */
int orc_greedy_init(int n, const int *rowptr, const int *colids, int v0, double *xy)
{
    if (check_csr(n, rowptr, colids) != ORC_OK) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    if (v0 < 0 || v0 >= n) return ORC_EINVAL;
    char *visited = (char *)calloc((size_t)n, 1);
    int *stack = (int *)malloc((size_t)n * sizeof(int));
    if (!visited || !stack) { free(visited); free(stack); return ORC_ENOMEM; }
    const double PI = 3.1416;
    int top = 0;
    xy[2 * v0] = 0.0; xy[2 * v0 + 1] = 0.0;
    stack[top++] = v0; visited[v0] = 1;
    while (top > 0) {
        int u = stack[--top];
        int deg = rowptr[u + 1] - rowptr[u];
        double d = deg > 0 ? 360.0 / (double)deg : 0.0;
        double D = 0.0;
        for (int k = rowptr[u]; k < rowptr[u + 1]; k++) {
            int w = colids[k];
            if (visited[w]) continue;
            xy[2 * w] = xy[2 * u] + cos(PI * D / 180.0);
            xy[2 * w + 1] = xy[2 * u + 1] + sin(PI * D / 180.0);
            visited[w] = 1;
            stack[top++] = w;
            D += d;
        }
    }
    free(visited); free(stack);
    return ORC_OK;
}
