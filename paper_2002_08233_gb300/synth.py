"""Seeded synthetic inputs: graphs in CSR form and initial layouts.

This module holds no part of the layout method's arithmetic. It only draws
graphs and starting positions, so that the CUDA path and the FP64 oracle can
be fed identical inputs. Every generator is deterministic in its seed.

Graph families stand in for the paper's datasets (Section 4.2, Table I: meshes,
scale-free and social graphs from SuiteSparse, LFR benchmark graphs), which are
not available here:

* ``grid2d``        -- 2-D grid (mesh-like, like 3elt_dual / fe_4elt2)
* ``barabasi_albert`` -- preferential attachment (scale-free, like ba_network)
* ``rmat``          -- recursive-matrix graph (power-law, like comYoutube)
* ``binary_tree``, ``erdos_renyi``, ``tri_mesh`` -- small-graph mixes

Every graph is undirected: ``csr_from_edges`` symmetrises the edge list, drops
self-loops and duplicates and sorts each row, since the method walks sorted
neighbour lists (Section 2.1, Algorithm 2's merge of colids).

Initial positions (Section 4.3.1 uses random coordinates in [-MAXMIN, MAXMIN])
come from ``uniform_positions``: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
evaluated as a counter-based generator, 24 random bits per coordinate, mapped to
[-1, 1). The values are exact in FP32, so both sides start from the same layout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclass
class CSR:
    """Undirected graph in CSR form (int32 rowptr[n+1], int32 colids[nnz])."""

    n: int
    rowptr: np.ndarray
    colids: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colids.shape[0])

    @property
    def n_edges(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)


# ----------------------------------------------------------------------------
# counter-based SplitMix64
# ----------------------------------------------------------------------------

def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream whose state
    starts at ``seed``: output k = mix(seed + (k+1)*0x9E3779B97F4A7C15)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def seeded_sample(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct vertices of 0..n-1: entries 0..m-1 after a partial
    Fisher-Yates shuffle whose step k swaps entries k and k + (z_k mod (n-k)),
    z_k = SplitMix64 output k of the stream with state ``seed``."""
    idx = np.arange(n, dtype=np.int64)
    z = splitmix64(seed, m)
    for k in range(m):
        j = k + int(z[k] % np.uint64(n - k))
        idx[k], idx[j] = idx[j], idx[k]
    return idx[:m].astype(np.int32)


def uniform_positions(n: int, seed: int = 0) -> np.ndarray:
    """float32[n, 2] uniform in [-1, 1): coordinate k (x of vertex i is k=2i,
    y is k=2i+1) is ((z_k >> 40) * 2^-24) * 2 - 1 for SplitMix64 output z_k."""
    z = splitmix64(seed, 2 * n)
    u = (z >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))
    return (u * 2.0 - 1.0).astype(np.float32).reshape(n, 2)


# ----------------------------------------------------------------------------
# CSR assembly
# ----------------------------------------------------------------------------

def _sorted_unique(key: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent difference)."""
    key = np.sort(key, kind="stable")
    if key.size == 0:
        return key
    keep = np.empty(key.size, dtype=bool)
    keep[0] = True
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    return key[keep]


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, name: str = "") -> CSR:
    """Symmetrise, drop self-loops and duplicates, sort rows."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.concatenate([u, v])
    b = np.concatenate([v, u])
    key = _sorted_unique(a * np.int64(n) + b)
    rows = (key // n).astype(np.int64)
    cols = (key % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph too large for int32 CSR")
    return CSR(n=n, rowptr=rowptr.astype(np.int32), colids=cols, name=name)


# ----------------------------------------------------------------------------
# graph families
# ----------------------------------------------------------------------------

def grid2d(rows: int, cols: int) -> CSR:
    """rows x cols 4-neighbour grid; vertex id = r*cols + c."""
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    u = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    v = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    return csr_from_edges(rows * cols, u, v, name=f"grid{rows}x{cols}")


def path_graph(n: int) -> CSR:
    i = np.arange(n - 1, dtype=np.int64)
    return csr_from_edges(n, i, i + 1, name=f"path{n}")


def cycle_graph(n: int) -> CSR:
    i = np.arange(n, dtype=np.int64)
    return csr_from_edges(n, i, (i + 1) % n, name=f"cycle{n}")


def from_edge_list(n: int, edges) -> CSR:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return csr_from_edges(n, e[:, 0], e[:, 1], name=f"edges{n}")


def barabasi_albert(n: int, m: int = 4, seed: int = 1) -> CSR:
    """Preferential attachment: a (m+1)-clique seed, then each new vertex links to
    m distinct earlier vertices drawn with probability proportional to degree
    (sampling uniformly from the list of edge endpoints, without repeats)."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    if n <= m0:
        iu, ju = np.triu_indices(n, 1)
        return csr_from_edges(n, iu, ju, name=f"ba{n}")
    iu, ju = np.triu_indices(m0, 1)
    n_edges = len(iu) + (n - m0) * m
    src = np.empty(n_edges, dtype=np.int64)
    dst = np.empty(n_edges, dtype=np.int64)
    src[: len(iu)] = iu
    dst[: len(iu)] = ju
    ends = np.empty(2 * n_edges, dtype=np.int64)
    ends[0: 2 * len(iu): 2] = iu
    ends[1: 2 * len(iu): 2] = ju
    n_ends = 2 * len(iu)
    e = len(iu)
    # draw candidates in blocks to keep the Python loop light
    block = rng.random(size=(n - m0, 4 * m))
    for idx, v in enumerate(range(m0, n)):
        chosen = []
        r = block[idx]
        k = 0
        while len(chosen) < m:
            if k < r.shape[0]:
                x = r[k]
                k += 1
            else:
                x = rng.random()
            t = int(ends[int(x * n_ends)])
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            src[e] = v
            dst[e] = t
            ends[n_ends] = v
            ends[n_ends + 1] = t
            n_ends += 2
            e += 1
    return csr_from_edges(n, src, dst, name=f"ba{n}_m{m}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 3, n: int | None = None) -> CSR:
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004): 2^scale * edge_factor samples,
    each choosing one quadrant per level with probabilities (a, b, c, d). With
    ``n`` given (< 2^scale), endpoints are folded into [0, n) by modulo."""
    rng = np.random.default_rng(seed)
    nv = 1 << scale
    m = nv * edge_factor
    u = np.zeros(m, dtype=np.int64)
    v = np.zeros(m, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    chunk = 1 << 22
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        uu = np.zeros(hi - lo, dtype=np.int64)
        vv = np.zeros(hi - lo, dtype=np.int64)
        for lev in range(scale):
            r = rng.random(hi - lo)
            ubit = r >= ab
            vbit = ((r >= a) & (r < ab)) | (r >= abc)
            bit = np.int64(1 << (scale - 1 - lev))
            uu |= np.where(ubit, bit, 0)
            vv |= np.where(vbit, bit, 0)
        u[lo:hi] = uu
        v[lo:hi] = vv
    if n is not None and n < nv:
        u %= n
        v %= n
        nv = n
    return csr_from_edges(nv, u, v, name=f"rmat{scale}_ef{edge_factor}")


def binary_tree(n: int, seed: int) -> CSR:
    """Random binary tree: vertex i >= 1 attaches to a uniformly chosen earlier
    vertex that still has fewer than two children."""
    rng = np.random.default_rng(seed)
    open_slots = [0, 0]  # each entry = a free child slot of that parent
    u = np.empty(max(n - 1, 0), dtype=np.int64)
    v = np.empty(max(n - 1, 0), dtype=np.int64)
    for i in range(1, n):
        k = int(rng.integers(len(open_slots)))
        p = open_slots[k]
        open_slots[k] = open_slots[-1]
        open_slots.pop()
        u[i - 1] = p
        v[i - 1] = i
        open_slots.append(i)
        open_slots.append(i)
    return csr_from_edges(n, u, v, name=f"bintree{n}")


def erdos_renyi(n: int, mean_degree: float, seed: int) -> CSR:
    """G(n, M) with M = round(n * mean_degree / 2) distinct uniform edges."""
    rng = np.random.default_rng(seed)
    target = int(round(n * mean_degree / 2))
    target = min(target, n * (n - 1) // 2)
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < target:
        need = target - keys.shape[0]
        a = rng.integers(0, n, size=2 * need + 16)
        b = rng.integers(0, n, size=2 * need + 16)
        lo = np.minimum(a, b)
        hi = np.maximum(a, b)
        ok = lo != hi
        cand = lo[ok] * np.int64(n) + hi[ok]
        keys = _sorted_unique(np.concatenate([keys, cand]))
    if keys.shape[0] > target:
        keys = rng.permutation(keys)[:target]
    return csr_from_edges(n, keys // n, keys % n, name=f"er{n}")


def tri_mesh(rows: int, cols: int, seed: int) -> CSR:
    """Triangulated grid: 4-neighbour grid plus one diagonal per cell, the
    diagonal's orientation drawn per cell."""
    rng = np.random.default_rng(seed)
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    u = [ids[:, :-1].ravel(), ids[:-1, :].ravel()]
    v = [ids[:, 1:].ravel(), ids[1:, :].ravel()]
    flip = rng.random((rows - 1, cols - 1)) < 0.5
    tl, tr = ids[:-1, :-1], ids[:-1, 1:]
    bl, br = ids[1:, :-1], ids[1:, 1:]
    u.append(np.where(flip, tr, tl).ravel())
    v.append(np.where(flip, bl, br).ravel())
    return csr_from_edges(rows * cols, np.concatenate(u), np.concatenate(v),
                          name=f"trimesh{rows}x{cols}")


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------

def grid_32x32() -> CSR:
    """32x32 grid: 1,024 vertices, 1,984 undirected edges."""
    return grid2d(32, 32)


def ba_65536() -> CSR:
    """Barabasi-Albert n=65,536, m=4 (262,134 undirected edges)."""
    return barabasi_albert(65536, 4, seed=1)


def rmat_scale20() -> CSR:
    """R-MAT scale 20, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), seed 3."""
    return rmat(20, 16, 0.57, 0.19, 0.19, seed=3)


def _near_grid(n: int) -> CSR:
    r = max(1, int(round(math.sqrt(n))))
    c = max(1, int(round(n / r)))
    return grid2d(r, c)


def small_graph_mix(count: int = 4096, n_lo: int = 50, n_hi: int = 5000,
                    seed: int = 4) -> list[CSR]:
    """Sizes log-uniform in [n_lo, n_hi]; kind cycles over grid / random binary
    tree / Erdos-Renyi (mean degree uniform in [4, 8])."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))
    kinds = rng.integers(0, 3, size=count)
    degs = rng.uniform(4.0, 8.0, size=count)
    out = []
    for k in range(count):
        n = int(round(sizes[k]))
        if kinds[k] == 0:
            g = _near_grid(n)
        elif kinds[k] == 1:
            g = binary_tree(n, seed * 100003 + k)
        else:
            g = erdos_renyi(n, float(degs[k]), seed * 100003 + k)
        out.append(g)
    return out


@dataclass
class Request:
    arrival_s: float
    graph: CSR
    seed: int


def _stream_graph(args) -> CSR:
    """Graph k of a serving stream: R-MAT (edge factor 8, folded into n vertices)
    or a triangulated mesh of about n vertices, from its own seed."""
    kind, n, gseed = args
    if kind == 0:
        scale = max(1, int(math.ceil(math.log2(n))))
        return rmat(scale, 8, seed=gseed, n=n)
    r = max(2, int(round(math.sqrt(n))))
    return tri_mesh(r, max(2, int(round(n / r))), gseed)


def serving_stream_plan(count: int, rate_per_s: float, n_lo: int, n_hi: int, seed: int = 5):
    """Arrival times and each request's graph recipe (kind, n, graph seed)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))
    kinds = rng.integers(0, 2, size=count)
    recipes = [(int(kinds[k]), int(round(sizes[k])), seed * 1000003 + k) for k in range(count)]
    return [float(x) for x in t], recipes


def serving_stream(count: int, rate_per_s: float, n_lo: int, n_hi: int,
                   seed: int = 5, workers: int = 1):
    """Poisson arrivals; sizes log-uniform in [n_lo, n_hi]; half R-MAT (edge
    factor 8, folded into n vertices), half triangulated meshes. With workers > 1
    the graphs are drawn by a pool of processes started with "spawn" (each graph
    depends only on its own recipe, so the stream is the same) and the requests
    are yielded in order as they are ready; otherwise a list is returned."""
    times, recipes = serving_stream_plan(count, rate_per_s, n_lo, n_hi, seed)
    if workers <= 1:
        return [Request(arrival_s=times[k], graph=_stream_graph(recipes[k]), seed=k) for k in range(count)]

    def gen():
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            for k, g in enumerate(pool.imap(_stream_graph, recipes, chunksize=1)):
                yield Request(arrival_s=times[k], graph=g, seed=k)
    return gen()
