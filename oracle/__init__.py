"""FP64 CPU oracle for BatchLayout -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The library's product path never does:
the CUDA path and this oracle share no code, and neither imports the other.

The arithmetic lives in ``bl_oracle.c`` (plain sequential C, FP64 except where
the paper's Barnes-Hut rules are pinned to FP32: Morton quantisation, node
centroids and the acceptance test). This module compiles it with gcc on first
use and marshals numpy arrays. Each function names the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbl_oracle.so")
_lock = threading.Lock()
_lib = None

EXACT = 0
BH = 1
THETA_DEFAULT = 1.2  # Section 4.1: same MAC threshold as ForceAtlas2BH


def build(force: bool = False) -> str:
    """Compile bl_oracle.c into _build/libbl_oracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, f64, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            lib.orc_forces.argtypes = [i32, P, P, P, f64, f64, i32, i32, i32, f64, i32, i32, i32, P, P]
            lib.orc_run.argtypes = [i32, P, P, P, i32, i32, i32, f64, f64, f64, i32, i32, i64, i32, P]
            lib.orc_morton.argtypes = [i32, P, P, P, P]
            lib.orc_bh_tree.argtypes = [i32, P, P, P, P, i32, P, P, P, P, P, P, P]
            lib.orc_bh_interactions.argtypes = [i32, P, P, f64, P, P]
            lib.orc_bh_query_counts.argtypes = [i32, P, P, f64, P, P]
            lib.orc_stress.argtypes = [i32, P, P, P, i32, P, P]
            lib.orc_edge_uniformity.argtypes = [i32, P, P, P, P]
            lib.orc_neighborhood_preservation.argtypes = [i32, P, P, P, i32, P, P]
            lib.orc_greedy_init.argtypes = [i32, P, P, i32, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.colids, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    return rp, ci


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def forces(g, xy, K=1.0, R=1.0, repulse_neighbors=False, mode=EXACT, theta=THETA_DEFAULT,
           lo=0, hi=None, nthreads=1, a=2):
    """One-snapshot combined forces f(i, c) for i in [lo, hi) (Section 2.2;
    BH repulsion per Algorithms S3/S4; attraction d^a/K, a = 2 by default).
    Returns (f[hi-lo, 2], mag[hi-lo]) where mag_i is the sum of the magnitudes
    of the terms that make up f(i, c)."""
    lib = _load()
    n = g.n
    hi = n if hi is None else hi
    rp, ci = _csr(g)
    x = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(n, 2))
    f = np.zeros((max(hi - lo, 0), 2), dtype=np.float64)
    mag = np.zeros(max(hi - lo, 0), dtype=np.float64)
    rc = lib.orc_forces(n, _ptr(rp), _ptr(ci), _ptr(x), K, R, int(a), int(repulse_neighbors), mode,
                        theta, lo, hi, nthreads, _ptr(f) if f.size else None, _ptr(mag) if mag.size else None)
    _check(rc, "forces")
    return f, mag


def run(g, xy, iters, batch, mode=EXACT, theta=THETA_DEFAULT, K=1.0, R=1.0,
        repulse_neighbors=False, start_iter=0, nthreads=1, a=2):
    """Algorithm 2 (exact) or Algorithm S5 (BH) with attraction d^a/K: returns
    (positions float64[n,2], energy per iteration float64[iters])."""
    lib = _load()
    n = g.n
    rp, ci = _csr(g)
    x = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(n, 2)).copy()
    e = np.zeros(max(iters, 1), dtype=np.float64)
    rc = lib.orc_run(n, _ptr(rp), _ptr(ci), _ptr(x), iters, batch, mode, theta, K, R, int(a),
                     int(repulse_neighbors), start_iter, nthreads, _ptr(e))
    _check(rc, "run")
    return x, e[:iters]


def morton(xy):
    """Morton codes of FP32 positions (Section 3.5, Fig. 4). Returns
    (codes uint32[n], (xmin, ymin, D))."""
    lib = _load()
    a = np.asarray(xy, dtype=np.float32).reshape(-1, 2)
    n = a.shape[0]
    xf = np.ascontiguousarray(a[:, 0])
    yf = np.ascontiguousarray(a[:, 1])
    codes = np.zeros(max(n, 1), dtype=np.uint32)
    box = np.zeros(3, dtype=np.float32)
    _check(lib.orc_morton(n, _ptr(xf), _ptr(yf), _ptr(codes), _ptr(box)), "morton")
    return codes[:n], tuple(float(v) for v in box)


def bh_tree(xy):
    """Quadtree of Algorithm S3 in pre-order. Returns a dict with perm, codes
    (sorted), first, count, level, skip, sumx, sumy (FP32)."""
    lib = _load()
    a = np.asarray(xy, dtype=np.float32).reshape(-1, 2)
    n = a.shape[0]
    xf = np.ascontiguousarray(a[:, 0])
    yf = np.ascontiguousarray(a[:, 1])
    cap = max(16, 17 * n + 1)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    codes = np.zeros(max(n, 1), dtype=np.uint32)
    arrs = {k: np.zeros(cap, dtype=np.int32) for k in ("first", "count", "level", "skip")}
    sx = np.zeros(cap, dtype=np.float32)
    sy = np.zeros(cap, dtype=np.float32)
    nn = ctypes.c_int(0)
    rc = lib.orc_bh_tree(n, _ptr(xf), _ptr(yf), _ptr(perm), _ptr(codes), cap,
                         _ptr(arrs["first"]), _ptr(arrs["count"]), _ptr(arrs["level"]),
                         _ptr(arrs["skip"]), _ptr(sx), _ptr(sy), ctypes.byref(nn))
    _check(rc, "bh_tree")
    m = nn.value
    out = {k: v[:m].copy() for k, v in arrs.items()}
    out.update(perm=perm[:n].copy(), codes=codes[:n].copy(), sumx=sx[:m].copy(),
               sumy=sy[:m].copy(), nnodes=m)
    return out


def bh_interactions(xy, theta=THETA_DEFAULT):
    """(accepted far-field nodes, directly summed leaf vertices) over all queries."""
    lib = _load()
    a = np.asarray(xy, dtype=np.float32).reshape(-1, 2)
    xf = np.ascontiguousarray(a[:, 0])
    yf = np.ascontiguousarray(a[:, 1])
    far = ctypes.c_longlong(0)
    near = ctypes.c_longlong(0)
    _check(lib.orc_bh_interactions(a.shape[0], _ptr(xf), _ptr(yf), theta, ctypes.byref(far),
                                   ctypes.byref(near)), "bh_interactions")
    return far.value, near.value


def bh_query_counts(xy, theta=THETA_DEFAULT):
    """Per vertex: (accepted far-field nodes, leaf vertices met, its own included)
    on its walk of the quadtree (Section 3.5's MAC, Algorithm S4)."""
    lib = _load()
    a = np.asarray(xy, dtype=np.float32).reshape(-1, 2)
    n = a.shape[0]
    xf = np.ascontiguousarray(a[:, 0])
    yf = np.ascontiguousarray(a[:, 1])
    far = np.zeros(max(n, 1), dtype=np.int32)
    near = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib.orc_bh_query_counts(n, _ptr(xf), _ptr(yf), theta, _ptr(far), _ptr(near)),
           "bh_query_counts")
    return far[:n].copy(), near[:n].copy()


def stress(g, xy, sources=None):
    """Stress (Section 3.7) minimised over the layout scale. Returns
    (stress, s_star, pairs)."""
    lib = _load()
    rp, ci = _csr(g)
    x = np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(g.n, 2))
    out = np.zeros(3, dtype=np.float64)
    if sources is None:
        rc = lib.orc_stress(g.n, _ptr(rp), _ptr(ci), _ptr(x), 0, None, _ptr(out))
    else:
        s = np.ascontiguousarray(sources, dtype=np.int32)
        rc = lib.orc_stress(g.n, _ptr(rp), _ptr(ci), _ptr(x), s.size, _ptr(s), _ptr(out))
    _check(rc, "stress")
    return float(out[0]), float(out[1]), float(out[2])


def edge_uniformity(g, xy):
    """Edge uniformity (Section 3.7)."""
    lib = _load()
    rp, ci = _csr(g)
    x = np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(g.n, 2))
    out = np.zeros(1, dtype=np.float64)
    _check(lib.orc_edge_uniformity(g.n, _ptr(rp), _ptr(ci), _ptr(x), _ptr(out)), "eu")
    return float(out[0])


def neighborhood_preservation(g, xy, queries=None):
    """Neighbourhood preservation (Section 3.7), 1-hop Jaccard reading.
    Returns (NP, queries used, total intersection size)."""
    lib = _load()
    rp, ci = _csr(g)
    x = np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(g.n, 2))
    out = np.zeros(3, dtype=np.float64)
    if queries is None:
        rc = lib.orc_neighborhood_preservation(g.n, _ptr(rp), _ptr(ci), _ptr(x), 0, None, _ptr(out))
    else:
        q = np.ascontiguousarray(queries, dtype=np.int32)
        rc = lib.orc_neighborhood_preservation(g.n, _ptr(rp), _ptr(ci), _ptr(x), q.size, _ptr(q),
                                               _ptr(out))
    _check(rc, "np")
    return float(out[0]), int(out[1]), int(out[2])


def greedy_init(g, xy, v0=0):
    """Greedy initialisation (Algorithm 3). Returns float64[n, 2]."""
    lib = _load()
    rp, ci = _csr(g)
    x = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(g.n, 2)).copy()
    _check(lib.orc_greedy_init(g.n, _ptr(rp), _ptr(ci), v0, _ptr(x)), "greedy_init")
    return x
