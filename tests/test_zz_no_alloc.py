"""bl_layout_run_noalloc: the exact-mode run for callers that cannot call
cudaMalloc (their device memory comes from a pool they own, or an allocation's
implicit synchronisation is not acceptable where they run). It keeps its working
memory in a fixed device array inside the library. These tests check, through
the C ABI, that two calls in a row give bit for bit what bl_layout_run gives on
the same inputs with the same (whole-GPU) engine, that a small graph matches the
FP64 oracle, that the calls allocate no device memory, and that sizes beyond the
array are refused.

Collected last on purpose (file name): a failure here leaves every other test
already run."""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import TOL_POS_EXACT, assert_positions, oracle_sensitivity

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def _noalloc_fn(lib):
    fn = lib.bl_layout_run_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int64, P, P]
    fn.restype = ctypes.c_int
    return fn


def _whole_gpu_reference(core, g, xy, runs):
    """bl_layout_run on the whole-GPU engine (forced, so small graphs do not take
    the one-cluster engine): positions and energies after each run of `runs`."""
    os.environ["BL_EXACT_ENGINE"] = "grid"
    try:
        L = core.Layout(core.Graph(g), xy=xy)
        out = []
        for it in runs:
            L.run(it, 256, "exact")
            out.append((L.positions().copy(), L.energy_history().copy()))
        return out
    finally:
        os.environ.pop("BL_EXACT_ENGINE", None)


def _noalloc_runs(core, g, xy, runs):
    """The same runs through bl_layout_run_noalloc on caller-owned device buffers."""
    import torch
    lib = core.load()
    fn = _noalloc_fn(lib)
    dev = torch.device("cuda")
    rp = torch.from_numpy(g.rowptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(g.colids.astype(np.int32) if g.nnz else np.zeros(1, np.int32)).to(dev)
    d_xy = torch.from_numpy(xy.copy()).to(dev)
    stream = torch.cuda.current_stream()
    out, t = [], 0
    for it in runs:
        d_e = torch.zeros(it, dtype=torch.float64, device=dev)
        st = fn(g.n, rp.data_ptr(), ci.data_ptr(), d_xy.data_ptr(), it, 256, None, t, d_e.data_ptr(),
                ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.bl_last_error()
        out.append((d_xy.cpu().numpy().copy(), d_e.cpu().numpy().copy()))
        t += it
    return out


@pytest.mark.parametrize("name,maker", [
    ("er4000", lambda: synth.erdos_renyi(4000, 6.0, 21)),
    ("grid32", lambda: synth.grid_32x32()),   # small: bl_layout_run would default to the cluster engine
])
def test_noalloc_matches_layout_run_twice(core, name, maker):
    """Two calls in a row (3 then 2 iterations, the second continuing the step
    schedule) equal bl_layout_run on the same engine bit for bit."""
    g = maker()
    xy = synth.uniform_positions(g.n, 21)
    ref = _whole_gpu_reference(core, g, xy, (3, 2))
    got = _noalloc_runs(core, g, xy, (3, 2))
    for k, ((x_r, e_r), (x_g, e_g)) in enumerate(zip(ref, got)):
        assert np.array_equal(x_g, x_r), (name, k, float(np.abs(x_g - x_r).max()))
        assert np.array_equal(e_g, e_r), (name, k, e_g, e_r)


def test_noalloc_small_graph_matches_oracle(core):
    """The 32x32 grid, one iteration of minibatch 256, against the FP64 oracle."""
    g = synth.grid_32x32()
    xy = synth.uniform_positions(g.n, 5)
    (x_g, e_g), = _noalloc_runs(core, g, xy, (1,))
    xr, sens = oracle_sensitivity(g, xy, 1, 256, nthreads=NCPU)
    assert_positions("noalloc grid32", x_g, xr, TOL_POS_EXACT, sens)
    _, er = oracle.run(g, xy, iters=1, batch=256, nthreads=NCPU)
    assert e_g[0] == pytest.approx(er[0], rel=1e-4)


def test_noalloc_allocates_no_device_memory(core):
    """With allocator hooks that refuse every request installed, two calls still
    succeed, the hooks are never called, and neither torch's allocator nor the
    device's free memory changes."""
    import torch
    lib = core.load()
    g = synth.erdos_renyi(4000, 6.0, 22)
    xy = synth.uniform_positions(g.n, 22)
    _noalloc_runs(core, g, xy, (3, 2))        # first calls: the array's address, every copy path
    torch.cuda.synchronize()
    calls = []
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    fail_alloc = ALLOC(lambda nbytes, ctx: calls.append(("alloc", nbytes)) or None)
    no_free = FREE(lambda p, ctx: calls.append(("free", p)))
    dev = torch.device("cuda")
    rp = torch.from_numpy(g.rowptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(g.colids.astype(np.int32)).to(dev)
    d_xy = torch.from_numpy(xy.copy()).to(dev)
    d_e = torch.zeros(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    fn = _noalloc_fn(lib)
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    free_before = torch.cuda.mem_get_info()[0]
    try:
        lib.bl_set_allocator(ctypes.cast(fail_alloc, ctypes.c_void_p), ctypes.cast(no_free, ctypes.c_void_p), None)
        for t0, it in ((0, 3), (3, 2)):
            st = fn(g.n, rp.data_ptr(), ci.data_ptr(), d_xy.data_ptr(), it, 256, None, t0, d_e.data_ptr(),
                    ctypes.c_void_p(stream.cuda_stream))
            assert st == 0, lib.bl_last_error()
    finally:
        lib.bl_set_allocator(ctypes.cast(core._hooks["alloc"], ctypes.c_void_p),
                             ctypes.cast(core._hooks["free"], ctypes.c_void_p), None)
    torch.cuda.synchronize()
    assert calls == []
    assert torch.cuda.memory_allocated() == torch_before
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_sizes_beyond_its_limit(core):
    lib = core.load()
    fn = _noalloc_fn(lib)
    dummy = ctypes.c_void_p(16)   # never dereferenced: the argument checks come first
    st = fn(131073, dummy, dummy, dummy, 1, 256, None, 0, None, None)
    assert st == 1
    assert b"131072" in lib.bl_last_error()
    from paper_2002_08233_gb300.core import ForceParams
    for K, R in ((float("inf"), 1.0), (1.0, float("inf")), (float("nan"), 1.0), (0.0, 1.0)):
        prm = ForceParams(K, R, 0, -1, 0)
        st = fn(1000, dummy, dummy, dummy, 1, 256, ctypes.byref(prm), 0, None, None)
        assert st == 1, (K, R)
        assert b"finite" in lib.bl_last_error()
