"""bl_layout_run_noalloc: the exact-mode run for callers that cannot call
cudaMalloc (their device memory comes from a pool they own, or an allocation's
implicit synchronisation is not acceptable where they run). It keeps its working
memory in a fixed device array inside the library; this test checks, through the
C ABI, that two calls in a row give what bl_layout_run gives on the same inputs.

Collected last on purpose (file name): a failure here leaves every other test
already run."""
import ctypes

import numpy as np
import pytest

from paper_2002_08233_gb300 import synth
from helpers import TOL_POS_EXACT, position_error

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_layout_run_twice(core):
    import torch
    lib = core.load()
    fn = _noalloc_fn(lib)
    g = synth.erdos_renyi(4000, 6.0, 21)   # above the cluster engine's size: both calls run the whole-GPU engine
    xy = synth.uniform_positions(g.n, 21)
    # existing entry point
    G = core.Graph(g)
    L = core.Layout(G, xy=xy)
    L.run(3, 256, "exact")
    ref1 = L.positions().copy()
    e1 = L.energy_history().copy()
    L.run(2, 256, "exact")
    ref2 = L.positions().copy()
    e2 = L.energy_history().copy()
    # caller-owned device buffers
    dev = torch.device("cuda")
    rp = torch.from_numpy(g.rowptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(g.colids.astype(np.int32)).to(dev)
    d_xy = torch.from_numpy(xy.copy()).to(dev)
    d_e = torch.zeros(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    st = fn(g.n, rp.data_ptr(), ci.data_ptr(), d_xy.data_ptr(), 3, 256, None, 0, d_e.data_ptr(),
            ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.bl_last_error()
    out1 = d_xy.cpu().numpy()
    assert position_error(out1, ref1.astype(np.float64)) <= TOL_POS_EXACT
    assert np.allclose(d_e.cpu().numpy(), e1, rtol=1e-9)
    d_e2 = torch.zeros(2, dtype=torch.float64, device=dev)
    st = fn(g.n, rp.data_ptr(), ci.data_ptr(), d_xy.data_ptr(), 2, 256, None, 3, d_e2.data_ptr(),
            ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.bl_last_error()
    out2 = d_xy.cpu().numpy()
    assert position_error(out2, ref2.astype(np.float64)) <= TOL_POS_EXACT
    assert np.allclose(d_e2.cpu().numpy(), e2, rtol=1e-9)


def test_noalloc_rejects_sizes_beyond_its_limit(core):
    lib = core.load()
    fn = _noalloc_fn(lib)
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    st = fn(131073, dummy, dummy, dummy, 1, 256, None, 0, None, None)
    assert st == 1
    assert b"131072" in lib.bl_last_error()
