"""Continuous-batching server: results identical alone and in a mix, identical
to the direct API, admission against the memory budget, cancel, latency stats."""
import time

import numpy as np
import pytest

from paper_2002_08233_gb300 import synth

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def _wait(S, ticket, n, timeout=120.0):
    t0 = time.time()
    while True:
        r = S.poll(ticket, n)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(0.001)


def _requests():
    """(graph, seed, iters, batch, mode): batched exact, whole-GPU exact, BH."""
    return [
        (synth.erdos_renyi(300, 6.0, 1), 11, 120, 64, "exact"),
        (synth.grid2d(20, 20), 12, 75, 256, "auto"),
        (synth.erdos_renyi(17000, 4.0, 2), 13, 7, 256, "exact"),
        (synth.tri_mesh(250, 250, 3), 14, 6, 256, "auto"),      # 62,500 vertices: BH
    ]


def _serve(core, reqs, budget=8 * GB, fillers=()):
    S = core.Server(budget)
    Gs, tickets = [], []
    for g, seed, it, bs, mode in list(fillers) + list(reqs):
        G = core.Graph(g)
        Gs.append(G)
        tickets.append((S.submit(G, seed, it, bs, mode), g.n))
    out = [_wait(S, t, n) for t, n in tickets]
    stats = S.stats()
    S.close()
    return out[len(fillers):], stats


def test_same_alone_and_in_mix(core):
    reqs = _requests()
    alone = [_serve(core, [r])[0][0][0] for r in reqs]
    fillers = [(synth.small_graph_mix(1, 50, 3000, seed=100 + k)[0], 200 + k, 60, 64, "exact")
               for k in range(12)]
    mixed, stats = _serve(core, reqs, fillers=fillers)
    for a, (m, lat) in zip(alone, mixed):
        assert np.array_equal(a, m)
        assert lat > 0
    assert stats["completed"] == len(reqs) + len(fillers)


def test_same_as_direct_api(core):
    """Server results equal the direct calls on the same request: bl_layout_batch
    for the batched requests (one launch there, 50-iteration ticks here),
    bl_layout_run for the whole-GPU ones (one call there, chunks here)."""
    reqs = _requests()
    served, _ = _serve(core, reqs)
    for (g, seed, it, bs, mode), (xy, _) in zip(reqs, served):
        G = core.Graph(g)
        if g.n <= 2048:
            ref = core.layout_batch([G], [seed], it, bs)[0]
        else:
            ref = core.Layout(G, seed=seed)
            ref.run(it, bs, "bh" if mode == "auto" and g.n >= 50000 else "exact")
        assert np.array_equal(ref.positions(), xy), (g.n, mode)


def test_budget_rejects_request_that_never_fits(core):
    S = core.Server(10_000)
    G = core.Graph(synth.erdos_renyi(5000, 5.0, 3))
    with pytest.raises(core.BatchLayoutError) as e:
        S.submit(G, 1, 10, 64, "exact")
    assert e.value.status == core.BL_EBUDGET
    S.close()


def test_admission_under_a_tight_budget(core):
    """A budget that holds two small requests at a time: every request still
    completes, memory in use never passes the budget, results unchanged."""
    gs = [synth.erdos_renyi(1000, 5.0, 30 + k) for k in range(8)]
    budget = 2 * (8 * 1000 + 8 * 100 + 4096) + 100
    S = core.Server(budget)
    Gs = [core.Graph(g) for g in gs]
    ts = [S.submit(G, 40 + k, 100, 64, "exact") for k, G in enumerate(Gs)]
    res = [_wait(S, t, 1000) for t in ts]
    st = S.stats()
    S.close()
    assert st["completed"] == 8
    assert st["peak_bytes"] <= budget
    assert st["bytes"] == 0
    alone, _ = _serve(core, [(gs[5], 45, 100, 64, "exact")])
    assert np.array_equal(alone[0][0], res[5][0])


def test_cancel(core):
    """Four whole-GPU requests fill the server's whole-GPU slots, so a fifth one
    queues: it can be canceled, a running one cannot."""
    g = synth.erdos_renyi(3000, 5.0, 5)
    S = core.Server(GB)
    G = core.Graph(g)
    running = [S.submit(G, k, 3000, 64, "exact") for k in range(4)]
    queued = S.submit(G, 9, 3000, 64, "exact")
    t0 = time.time()
    while S.stats()["in_flight"] < 4:
        assert time.time() - t0 < 30
        time.sleep(0.001)
    S.cancel(queued)
    with pytest.raises(core.BatchLayoutError) as e:
        S.cancel(running[0])
    assert e.value.status == core.BL_EBUSY
    with pytest.raises(core.BatchLayoutError) as e:
        S.poll(queued, g.n)
    assert e.value.status == core.BL_ECANCELED
    S.close()   # drops the running requests


def test_zero_iterations_and_poll_errors(core):
    S = core.Server(GB)
    g = synth.path_graph(10)
    G = core.Graph(g)
    t = S.submit(G, 7, 0, 64, "exact")
    xy, lat = _wait(S, t, g.n)
    assert np.array_equal(xy, synth.uniform_positions(g.n, 7))
    with pytest.raises(core.BatchLayoutError):
        S.poll(t, g.n)          # retired
    t = S.submit(G, 7, 5, 64, "exact")
    with pytest.raises(core.BatchLayoutError):
        while S.poll(t, 3) is None:   # short output buffer once done
            time.sleep(0.001)
    xy, _ = _wait(S, t, g.n)        # the ticket survives the short-buffer error
    assert xy.shape == (10, 2)
    S.close()


def test_latency_percentiles(core):
    gs = synth.small_graph_mix(40, 50, 2000, seed=9)
    S = core.Server(4 * GB)
    Gs = [core.Graph(g) for g in gs]
    ts = [S.submit(G, k, 100, 64, "exact") for k, G in enumerate(Gs)]
    lats = [_wait(S, t, g.n)[1] for t, g in zip(ts, gs)]
    st = S.stats()
    S.close()
    assert st["completed"] == 40
    assert 0 < st["p50_s"] <= st["p99_s"] <= max(lats) + 1e-9
    assert st["p99_s"] == pytest.approx(sorted(lats)[int(np.ceil(0.99 * 40)) - 1])
