"""Failure detection without faulting the GPU: a bounded device-side wait that
runs out reaches the host as BL_ETIMEOUT, and a request whose allocation fails
(injected on the host through the allocator hook) fails alone while the server
keeps serving."""
import ctypes
import time

import numpy as np
import pytest

from paper_2002_08233_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def test_bounded_barrier_wait_times_out_and_context_survives(core):
    lib = core.load()
    t0 = time.time()
    assert lib.bl_debug_barrier_timeout(50) == core.BL_ETIMEOUT
    assert time.time() - t0 < 10
    assert b"timed out" in lib.bl_last_error()
    # the context is still usable: a normal run succeeds afterwards
    g = synth.erdos_renyi(500, 5.0, 1)
    L = core.Layout(core.Graph(g), seed=1)
    L.run(2, 64, "exact")
    assert np.isfinite(L.positions()).all()
    assert lib.bl_debug_barrier_timeout(0) == core.BL_EINVAL


def test_server_request_fails_alone_on_allocation_error(core):
    lib = core.load()
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    fail_alloc = ALLOC(lambda nbytes, ctx: None)
    no_free = FREE(lambda p, ctx: None)
    g = synth.erdos_renyi(800, 5.0, 2)
    G = core.Graph(g)
    S = core.Server(1 << 30)
    try:
        lib.bl_set_allocator(ctypes.cast(fail_alloc, ctypes.c_void_p), ctypes.cast(no_free, ctypes.c_void_p), None)
        t_bad = S.submit(G, 1, 20, 64, "exact")
        t0 = time.time()
        with pytest.raises(core.BatchLayoutError) as e:
            while S.poll(t_bad, g.n) is None:
                assert time.time() - t0 < 60
                time.sleep(0.001)
        assert e.value.status == core.BL_ENOMEM
    finally:
        lib.bl_set_allocator(ctypes.cast(core._hooks["alloc"], ctypes.c_void_p),
                             ctypes.cast(core._hooks["free"], ctypes.c_void_p), None)
    t_ok = S.submit(G, 1, 20, 64, "exact")
    t0 = time.time()
    while (r := S.poll(t_ok, g.n)) is None:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    st = S.stats()
    S.close()
    assert st["completed"] == 1 and st["bytes"] == 0
    ref = core.layout_batch([G], [1], 20, 64)[0]
    assert np.array_equal(r[0], ref.positions())


def test_bh_rejects_graphs_over_its_vertex_limit(core):
    # one vertex over the quadtree's budget: 17 n + 1 nodes no longer fit int32
    # indices, so both the run and a serving request are refused before any launch
    n = 126_322_568
    G = core.Graph(n=n, rowptr=np.zeros(n + 1, np.int32), colids=np.zeros(0, np.int32))
    L = core.Layout(G, seed=0)
    with pytest.raises(core.BatchLayoutError) as e:
        L.run(1, 256, "bh")
    assert e.value.status == core.BL_EINVAL
    L.run(0, 256, "bh")   # nothing to do is still fine
    S = core.Server(1 << 40)
    try:
        with pytest.raises(core.BatchLayoutError) as e:
            S.submit(G, 0, 1, 256, "bh")
        assert e.value.status == core.BL_EINVAL
    finally:
        S.close()
    L.close()
    G.close()


def test_exact_run_refuses_more_steps_than_int32_counts(core):
    # 536,871 iterations x 4,000 minibatches of one vertex > 2^31 - 1 steps: refused
    # before any launch, and the layout is left as it was
    g = synth.erdos_renyi(4000, 5.0, 3)
    G = core.Graph(g)
    L = core.Layout(G, seed=3)
    with pytest.raises(core.BatchLayoutError) as e:
        L.run(536_871, 1, "exact")
    assert e.value.status == core.BL_EINVAL
    L.run(1, 1, "exact")
    ref = core.Layout(G, seed=3)
    ref.run(1, 1, "exact")
    assert np.array_equal(L.positions(), ref.positions())
