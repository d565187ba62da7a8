"""Thin ctypes binding of the C ABI in include/batchlayout.h.

Argument marshalling only: every step of the layout runs in the CUDA library
(lib/libbatchlayout.so). PyTorch supplies the device memory (through the
allocator hooks) and the stream. There is no CPU fallback: when the library
or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libbatchlayout.so")

BL_OK, BL_EINVAL, BL_ENOMEM, BL_EBUDGET, BL_ECUDA, BL_ETIMEOUT, BL_EBUSY, BL_ENOTREADY, \
    BL_ECANCELED = range(9)
STATUS_NAMES = ["BL_OK", "BL_EINVAL", "BL_ENOMEM", "BL_EBUDGET", "BL_ECUDA", "BL_ETIMEOUT",
                "BL_EBUSY", "BL_ENOTREADY", "BL_ECANCELED"]
MODES = {"exact": 0, "bh": 1, "auto": 2}
# (a,r)-energy models: attraction d^a / K, repulsion R K^2 / d
ENERGY_MODELS = {"fr": 0, "fa": 1, "linlog": 2, "a3": 3}
MODEL_EXPONENT = {"fr": 2, "fa": 1, "linlog": 0, "a3": 3}
CSR_SYMMETRIZE, CSR_DEDUP, CSR_SORT = 1, 2, 4
THETA_DEFAULT = 1.2   # Section 4.1: the MAC threshold used with ForceAtlas2BH


class BatchLayoutError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class ForceParams(ctypes.Structure):
    _fields_ = [("K", ctypes.c_float), ("R", ctypes.c_float),
                ("repulse_neighbors", ctypes.c_int32), ("kahan", ctypes.c_int32),
                ("energy_model", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("step", ctypes.c_double),
                ("energy", ctypes.c_double), ("pair_interactions", ctypes.c_double),
                ("vertex_updates", ctypes.c_double), ("bh_far_nodes", ctypes.c_double),
                ("bh_near_pairs", ctypes.c_double), ("last_run_ms", ctypes.c_double)]


_lib = None
_lib_lock = threading.Lock()
_hooks = {}


@atexit.register
def _closing():
    _hooks["closing"] = True


def _declare(lib):
    P, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                             ctypes.c_uint64)
    f32, f64, sz = ctypes.c_float, ctypes.c_double, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "bl_set_stream": [P],
        "bl_set_allocator": [P, P, P],
        "bl_graph_load_csr": [i32, i64, P, P, u32, PP],
        "bl_graph_info": [P, P, P],
        "bl_layout_init": [P, P, u64, i64, P, PP],
        "bl_layout_set_positions": [P, P, i64],
        "bl_layout_run": [P, i32, i32, ctypes.c_int, f32],
        "bl_positions": [P, P, i64],
        "bl_positions_device": [P, PP],
        "bl_energy_history": [P, P, i64, P],
        "bl_stats": [P, P],
        "bl_quality": [P, i32, i32, u64, P, i64],
        "bl_layout_batch": [P, i32, P, i32, i32, ctypes.c_int, f32, P],
        "bl_server_create": [sz, PP],
        "bl_serve_submit": [P, P, u64, i32, i32, ctypes.c_int, f32, P],
        "bl_serve_poll": [P, u64, P, i64, P],
        "bl_serve_cancel": [P, u64],
        "bl_server_stats": [P, P, i64],
        "bl_debug_forces": [P, ctypes.c_int, f32, i32, i32, P],
        "bl_debug_bh_tree": [P, P, P, P, P, P, P, P, P, i64, P, P],
        "bl_debug_bh_counts": [P, f32, P, P, i64],
        "bl_set_trace": [P, i32],
        "bl_set_phase_timing": [P, i32],
        "bl_get_phase_times": [P, P, i64],
        "bl_measure_pair_rate": [i32, i32, P, i64],
        "bl_get_trace": [P, P, i64, P],
        "bl_layout_run_noalloc": [i32, P, P, P, i32, i32, P, i64, P, P],
        "bl_layout_run_batch": [P, i32, i32, i32],
        "bl_debug_barrier_timeout": [i32],
        "bl_layout_init_greedy": [P, i64, u64, P, PP],
        "bl_layout_run_until": [P, i32, i32, ctypes.c_int, f32, f64, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.argtypes = args
        fn.restype = ctypes.c_int
    for name in ("bl_graph_free", "bl_layout_free", "bl_server_free"):
        fn = getattr(lib, name, None)
        if fn is not None:
            fn.argtypes = [P]
            fn.restype = None
    lib.bl_last_error.restype = ctypes.c_char_p
    lib.bl_version.restype = ctypes.c_char_p


def load(require_gpu: bool = True):
    """Loads lib/libbatchlayout.so. Raises when it is missing (build it with
    ``python -m paper_2002_08233_gb300.build``) or, with require_gpu, when no
    CUDA device is visible."""
    global _lib
    with _lib_lock:
        if _lib is None:
            try:
                import torch  # noqa: F401  -- share PyTorch's CUDA runtime
            except ImportError:
                pass
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"CUDA library not built: {LIB_PATH} is missing")
            lib = ctypes.CDLL(LIB_PATH)
            _declare(lib)
            _lib = lib
    if require_gpu:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("batchlayout needs a CUDA GPU; none is visible")
    return _lib


def _check(status: int):
    if status != BL_OK:
        raise BatchLayoutError(status, _lib.bl_last_error().decode(errors="replace"))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def use_torch(stream=None, allocator: bool = True):
    """Routes the library's device memory through PyTorch's caching allocator and
    its work onto `stream` (default: torch's current stream)."""
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib.bl_set_stream(ctypes.c_void_p(stream.cuda_stream)))
    if allocator and "alloc" not in _hooks:
        ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
        dev = torch.cuda.current_device()

        def _alloc(nbytes, _ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))
            except Exception:   # out of memory: the library reports BL_ENOMEM
                return None

        def _free(p, _ctx):
            if _hooks.get("closing"):
                return      # interpreter shutdown: torch may already be gone
            torch.cuda.caching_allocator_delete(int(p))

        _hooks["alloc"] = ALLOC(_alloc)
        _hooks["free"] = FREE(_free)
        _check(lib.bl_set_allocator(ctypes.cast(_hooks["alloc"], ctypes.c_void_p),
                                    ctypes.cast(_hooks["free"], ctypes.c_void_p), None))
    return stream


def set_stream(stream_handle: int | None):
    lib = load()
    _check(lib.bl_set_stream(ctypes.c_void_p(stream_handle) if stream_handle else None))


class Graph:
    """A validated undirected CSR graph resident on the GPU (bl_graph)."""

    def __init__(self, csr=None, *, n=None, rowptr=None, colids=None, flags: int = 0):
        lib = load()
        if csr is not None:
            n, rowptr, colids = csr.n, csr.rowptr, csr.colids
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colids, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.bl_graph_load_csr(int(n), int(ci.size), _ptr(rp), _ptr(ci) if ci.size else None,
                                     flags, ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        nn = ctypes.c_int32(0)
        nz = ctypes.c_int64(0)
        _check(lib.bl_graph_info(h, ctypes.byref(nn), ctypes.byref(nz)))
        self.nnz = int(nz.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.bl_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Layout:
    """Layout state of one graph (bl_layout)."""

    def __init__(self, graph: Graph, xy=None, seed: int = 0, start_iter: int = 0, K: float = 1.0,
                 R: float = 1.0, repulse_neighbors: bool = False, kahan: int = -1, model: str = "fr",
                 _handle=None):
        lib = load()
        self.graph = graph
        if _handle is not None:
            self._h = _handle
            return
        prm = ForceParams(K, R, int(repulse_neighbors), int(kahan), ENERGY_MODELS[model])
        h = ctypes.c_void_p()
        arr = None
        if xy is not None:
            arr = np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(graph.n, 2))
        _check(lib.bl_layout_init(graph.handle, _ptr(arr), ctypes.c_uint64(seed), int(start_iter),
                                  ctypes.byref(prm), ctypes.byref(h)))
        self._h = h

    def run(self, iters: int, batch: int = 256, mode: str = "exact", theta: float = THETA_DEFAULT):
        _check(_lib.bl_layout_run(self._h, int(iters), int(batch), MODES[mode], float(theta)))
        return self

    def run_until(self, max_iters: int, batch: int = 256, mode: str = "exact",
                  theta: float = THETA_DEFAULT, tol: float = 1e-6):
        """Runs until the relative energy change falls to tol (bl_layout_run_until).
        Returns (iterations run, converged)."""
        it = ctypes.c_int32(0)
        cv = ctypes.c_int32(0)
        _check(_lib.bl_layout_run_until(self._h, int(max_iters), int(batch), MODES[mode], float(theta),
                                        float(tol), ctypes.byref(it), ctypes.byref(cv)))
        return it.value, bool(cv.value)

    def set_positions(self, xy, start_iter: int = 0):
        arr = np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(self.graph.n, 2))
        _check(_lib.bl_layout_set_positions(self._h, _ptr(arr), int(start_iter)))

    def positions(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((self.graph.n, 2), dtype=np.float32)
        _check(_lib.bl_positions(self._h, _ptr(out), out.size))
        return out

    def device_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check(_lib.bl_positions_device(self._h, ctypes.byref(p)))
        return int(p.value or 0)

    def energy_history(self) -> np.ndarray:
        cnt = ctypes.c_int64(0)
        _check(_lib.bl_energy_history(self._h, None, 0, ctypes.byref(cnt)))
        out = np.zeros(max(cnt.value, 0), dtype=np.float64)
        if cnt.value:
            _check(_lib.bl_energy_history(self._h, _ptr(out), out.size, ctypes.byref(cnt)))
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(_lib.bl_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def quality(self, nsources: int = 0, nqueries: int = 0, seed: int = 0) -> dict:
        out = np.zeros(7, dtype=np.float64)
        _check(_lib.bl_quality(self._h, int(nsources), int(nqueries), ctypes.c_uint64(seed),
                               _ptr(out), out.size))
        return {"stress": out[0], "scale": out[1], "stress_pairs": out[2], "np": out[3],
                "np_queries": out[4], "edge_uniformity": out[5], "np_intersections": out[6]}

    def debug_forces(self, mode: str = "exact", theta: float = THETA_DEFAULT, lo: int = 0,
                     hi: int | None = None) -> np.ndarray:
        hi = self.graph.n if hi is None else hi
        out = np.zeros((max(hi - lo, 0), 2), dtype=np.float32)
        _check(_lib.bl_debug_forces(self._h, MODES[mode], float(theta), int(lo), int(hi),
                                    _ptr(out) if out.size else _ptr(np.zeros(2, np.float32))))
        return out

    def debug_bh_tree(self) -> dict:
        n = self.graph.n
        cap = 17 * n + 16
        codes = np.zeros(n, dtype=np.uint32)
        perm = np.zeros(n, dtype=np.int32)
        arrs = {k: np.zeros(cap, dtype=np.int32) for k in ("first", "count", "level", "skip")}
        sx = np.zeros(cap, dtype=np.float32)
        sy = np.zeros(cap, dtype=np.float32)
        box = np.zeros(3, dtype=np.float32)
        nn = ctypes.c_int64(0)
        _check(_lib.bl_debug_bh_tree(self._h, _ptr(codes), _ptr(perm), _ptr(arrs["first"]),
                                     _ptr(arrs["count"]), _ptr(arrs["level"]), _ptr(arrs["skip"]),
                                     _ptr(sx), _ptr(sy), cap, ctypes.byref(nn), _ptr(box)))
        m = int(nn.value)
        out = {k: v[:m] for k, v in arrs.items()}
        out.update(codes=codes, perm=perm, sumx=sx[:m], sumy=sy[:m], nnodes=m,
                   box=tuple(float(b) for b in box))
        return out

    def debug_bh_counts(self, theta: float = THETA_DEFAULT):
        """Per vertex: (far-field nodes accepted, leaf vertices met) on its walk."""
        n = self.graph.n
        far = np.zeros(n, dtype=np.int32)
        near = np.zeros(n, dtype=np.int32)
        _check(_lib.bl_debug_bh_counts(self._h, float(theta), _ptr(far), _ptr(near), n))
        return far, near

    PHASES = ("bbox_morton", "radix_sort", "tree", "walk", "edge_pass_wait", "sweep", "energy",
              "edge_pass", "iteration")

    def set_phase_timing(self, on: bool = True):
        _check(_lib.bl_set_phase_timing(self._h, int(bool(on))))

    def phase_times(self) -> dict:
        """Barnes-Hut phase times of the last timed run (ms summed over its
        iterations), the last tree's nodes and the walk's node-record reads."""
        out = np.zeros(12, dtype=np.float64)
        _check(_lib.bl_get_phase_times(self._h, _ptr(out), out.size))
        d = {k: float(out[q]) for q, k in enumerate(self.PHASES)}
        d.update(nodes=int(out[9]), walk_node_visits=int(out[10]), iterations=int(out[11]))
        return d

    def set_trace(self, max_steps: int):
        _check(_lib.bl_set_trace(self._h, int(max_steps)))

    def trace(self) -> np.ndarray:
        """Phase timestamps of the last traced run, uint64 [CTAs*steps*8]."""
        cnt = ctypes.c_int64(0)
        _check(_lib.bl_get_trace(self._h, None, 0, ctypes.byref(cnt)))
        out = np.zeros(cnt.value, dtype=np.uint64)
        if cnt.value:
            _check(_lib.bl_get_trace(self._h, _ptr(out), out.size, ctypes.byref(cnt)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.bl_layout_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_pair_rate(threads: int = 512, skip_sp0: bool = False) -> dict:
    """Ceiling probes of the exact pair loop and of the SFU reciprocal (profiling)."""
    out = np.zeros(4, dtype=np.float64)
    _check(load().bl_measure_pair_rate(int(threads), int(bool(skip_sp0)), _ptr(out), out.size))
    return {"pairs_per_clk_per_sm": float(out[0]), "rcp_lanes_per_clk_per_sm": float(out[1]),
            "pair_kernel_ms": float(out[2]), "sm_mhz_implied": float(out[3])}


def greedy_layout(graph: Graph, v0: int = -1, seed: int = 0, K: float = 1.0, R: float = 1.0,
                  repulse_neighbors: bool = False, model: str = "fr") -> Layout:
    """A layout initialised by the greedy placement (bl_layout_init_greedy)."""
    prm = ForceParams(K, R, int(repulse_neighbors), -1, ENERGY_MODELS[model])
    h = ctypes.c_void_p()
    _check(load().bl_layout_init_greedy(graph.handle, int(v0), ctypes.c_uint64(seed), ctypes.byref(prm),
                                        ctypes.byref(h)))
    return Layout(graph, _handle=h)


def layout_run_noalloc(n: int, d_rowptr: int, d_colids: int, d_xy: int, iters: int, batch: int = 256,
                       K: float = 1.0, R: float = 1.0, repulse_neighbors: bool = False,
                       start_iter: int = 0, d_energy: int = 0, stream: int = 0, model: str = "fr") -> None:
    """bl_layout_run_noalloc on device buffers the caller owns (raw device
    addresses): for callers that cannot allocate device memory. The library
    keeps its working memory in a fixed device array; calls that overlap on the
    GPU race on it."""
    prm = ForceParams(K, R, int(repulse_neighbors), -1, ENERGY_MODELS[model])
    _check(load().bl_layout_run_noalloc(int(n), d_rowptr, d_colids, d_xy, int(iters), int(batch),
                                        ctypes.byref(prm), int(start_iter), d_energy or None,
                                        stream or None))


def layout_batch(graphs, seeds, iters: int, batch: int = 64, mode: str = "exact",
                 theta: float = THETA_DEFAULT) -> list:
    """Many graphs in one persistent launch (bl_layout_batch)."""
    lib = load()
    cnt = len(graphs)
    hs = (ctypes.c_void_p * cnt)(*[g.handle for g in graphs])
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    outs = (ctypes.c_void_p * cnt)()
    _check(lib.bl_layout_batch(hs, cnt, _ptr(sd), int(iters), int(batch), MODES[mode],
                               float(theta), outs))
    return [Layout(g, _handle=ctypes.c_void_p(outs[k])) for k, g in enumerate(graphs)]


def run_batch(layouts, iters: int, batch: int = 64) -> None:
    """Continues existing layouts in one batched launch (bl_layout_run_batch)."""
    lib = load()
    cnt = len(layouts)
    hs = (ctypes.c_void_p * cnt)(*[L._h for L in layouts])
    _check(lib.bl_layout_run_batch(hs, cnt, int(iters), int(batch)))


class Server:
    """Continuous-batching layout server (bl_server_*)."""

    def __init__(self, mem_budget_bytes: int):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.bl_server_create(ctypes.c_size_t(mem_budget_bytes), ctypes.byref(h)))
        self._h = h

    def submit(self, graph: Graph, seed: int, iters: int, batch: int = 256, mode: str = "auto",
               theta: float = THETA_DEFAULT) -> int:
        t = ctypes.c_uint64(0)
        _check(_lib.bl_serve_submit(self._h, graph.handle, ctypes.c_uint64(seed), int(iters),
                                    int(batch), MODES[mode], float(theta), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, n: int):
        """Returns (positions, latency_s) or None while not ready."""
        out = np.empty((n, 2), dtype=np.float32)
        lat = ctypes.c_double(0.0)
        st = _lib.bl_serve_poll(self._h, ctypes.c_uint64(ticket), _ptr(out), out.size,
                                ctypes.byref(lat))
        if st == BL_ENOTREADY:
            return None
        _check(st)
        return out, lat.value

    def cancel(self, ticket: int):
        _check(_lib.bl_serve_cancel(self._h, ctypes.c_uint64(ticket)))

    def stats(self) -> dict:
        out = np.zeros(7, dtype=np.float64)
        _check(_lib.bl_server_stats(self._h, _ptr(out), out.size))
        return {"completed": out[0], "in_flight": out[1], "queued": out[2], "bytes": out[3],
                "p50_s": out[4], "p99_s": out[5], "peak_bytes": out[6]}

    def close(self):
        if getattr(self, "_h", None):
            _lib.bl_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
