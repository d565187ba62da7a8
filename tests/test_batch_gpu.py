"""Batched layouts of many small graphs (one persistent launch, Algorithm 2 per
graph) against the FP64 oracle, plus the batching invariants: a graph's result
does not depend on the launch shape, on the other graphs in the launch, or on how
the iterations are chunked."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import TOL_POS_EXACT, oracle_sensitivity, position_error, assert_positions

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


@pytest.fixture
def env():
    saved = {k: os.environ.get(k) for k in ("BL_BATCH_SHAPE", "BL_BATCH_CHUNK")}
    yield os.environ
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def _mix(count, seed, n_lo=20, n_hi=700):
    return synth.small_graph_mix(count=count, n_lo=n_lo, n_hi=n_hi, seed=seed)


def _batch(core, gs, seeds, iters, bs):
    Gs = [core.Graph(g) for g in gs]
    Ls = core.layout_batch(Gs, seeds, iters, bs)
    return Gs, Ls


@pytest.mark.parametrize("bs", [64, 100, 256, 1])
def test_one_iteration_matches_oracle(core, bs):
    """Every graph of a mixed launch (grids, trees, ER; odd and even n, n below
    and above the minibatch) against the oracle from the same seeded start."""
    gs = _mix(24, 40 + bs)
    seeds = np.arange(len(gs), dtype=np.uint64) + 100
    Gs, Ls = _batch(core, gs, seeds, 1, bs)
    for g, L, sd in zip(gs, Ls, seeds):
        xy = synth.uniform_positions(g.n, int(sd))
        xr, sens = oracle_sensitivity(g, xy, 1, bs, nthreads=NCPU)
        _, er = oracle.run(g, xy, iters=1, batch=bs, nthreads=NCPU)
        assert_positions((g.name, g.n), L.positions(), xr, TOL_POS_EXACT, sens)
        assert L.energy_history()[0] == pytest.approx(er[0], rel=1e-4)


def test_three_iterations_match_oracle(core):
    gs = [synth.grid2d(9, 13), synth.binary_tree(201, 3), synth.erdos_renyi(333, 6.0, 4)]
    seeds = np.array([5, 6, 7], dtype=np.uint64)
    Gs, Ls = _batch(core, gs, seeds, 3, 64)
    for g, L, sd in zip(gs, Ls, seeds):
        xy = synth.uniform_positions(g.n, int(sd))
        xr, sens = oracle_sensitivity(g, xy, 3, 64, nthreads=NCPU)
        assert_positions(g.name, L.positions(), xr, TOL_POS_EXACT, sens)
        assert L.stats()["iterations"] == 3


def test_launch_shape_does_not_change_results(core, env):
    gs = _mix(40, 7)
    seeds = np.arange(len(gs), dtype=np.uint64)
    ref = None
    for shape in range(4):
        env["BL_BATCH_SHAPE"] = str(shape)
        _, Ls = _batch(core, gs, seeds, 3, 64)
        pos = [L.positions() for L in Ls]
        en = [L.energy_history() for L in Ls]
        if ref is None:
            ref = (pos, en)
        else:
            for a, b in zip(pos, ref[0]):
                assert np.array_equal(a, b), shape
            for a, b in zip(en, ref[1]):
                assert np.array_equal(a, b), shape


def test_alone_equals_in_mix(core):
    target = synth.erdos_renyi(500, 6.0, 77)
    _, alone = _batch(core, [target], np.array([9], dtype=np.uint64), 4, 64)
    others = _mix(30, 8)
    gs = others[:13] + [target] + others[13:]
    seeds = np.arange(len(gs), dtype=np.uint64) + 1000
    seeds[13] = 9
    _, mixed = _batch(core, gs, seeds, 4, 64)
    assert np.array_equal(alone[0].positions(), mixed[13].positions())
    assert np.array_equal(alone[0].energy_history(), mixed[13].energy_history())


def test_chunked_launches_equal_one_launch(core, env):
    gs = _mix(20, 9)
    seeds = np.arange(len(gs), dtype=np.uint64)
    _, one = _batch(core, gs, seeds, 7, 64)
    env["BL_BATCH_CHUNK"] = "3"
    _, chunked = _batch(core, gs, seeds, 7, 64)
    for a, b in zip(one, chunked):
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.energy_history(), b.energy_history())


def test_continuation_equals_one_run(core):
    gs = _mix(12, 10)
    seeds = np.arange(len(gs), dtype=np.uint64)
    _, full = _batch(core, gs, seeds, 5, 64)
    _, part = _batch(core, gs, seeds, 3, 64)
    core.run_batch(part, 2, 64)
    for a, b in zip(full, part):
        assert np.array_equal(a.positions(), b.positions())
        assert a.stats()["iterations"] == b.stats()["iterations"] == 5


def test_graph_above_fair_share_runs_on_whole_gpu(core):
    """One large graph with a few tiny ones: the large one exceeds an SM's share
    of the work and runs on the whole-GPU engine; both kinds match the oracle."""
    gs = [synth.erdos_renyi(2500, 5.0, 1)] + [synth.path_graph(30 + k) for k in range(4)]
    seeds = np.arange(len(gs), dtype=np.uint64) + 3
    _, Ls = _batch(core, gs, seeds, 1, 256)
    for g, L, sd in zip(gs, Ls, seeds):
        xy = synth.uniform_positions(g.n, int(sd))
        xr, sens = oracle_sensitivity(g, xy, 1, 256, nthreads=NCPU)
        assert_positions(("mixed", g.n), L.positions(), xr, TOL_POS_EXACT, sens)


def test_degenerate_graphs(core):
    gs = [synth.path_graph(1), synth.path_graph(2), synth.from_edge_list(7, []),
          synth.from_edge_list(65, [(0, k) for k in range(1, 65)])]
    seeds = np.array([1, 2, 3, 4], dtype=np.uint64)
    _, Ls = _batch(core, gs, seeds, 2, 64)
    for g, L, sd in zip(gs, Ls, seeds):
        xy = synth.uniform_positions(g.n, int(sd))
        xr, _ = oracle.run(g, xy, iters=2, batch=64)
        assert position_error(L.positions(), xr) <= 1e-4, g.n
    # a lone vertex feels no force and does not move
    assert np.array_equal(Ls[0].positions(), synth.uniform_positions(1, 1))


def test_bh_mode_runs_each_graph_as_bl_layout_run(core):
    gs = [synth.erdos_renyi(400, 5.0, 2), synth.grid2d(20, 20)]
    seeds = np.array([11, 12], dtype=np.uint64)
    Gs = [core.Graph(g) for g in gs]
    Ls = core.layout_batch(Gs, seeds, 2, 64, mode="bh")
    for G, L, sd in zip(Gs, Ls, seeds):
        R = core.Layout(G, seed=int(sd))
        R.run(2, 64, "bh")
        assert np.array_equal(L.positions(), R.positions())


def test_invalid_arguments(core):
    import ctypes
    lib = core.load()
    assert lib.bl_layout_batch(None, 1, None, 1, 64, 0, 1.2, None) == 1
    assert lib.bl_layout_run_batch(None, 1, 1, 64) == 1
    assert lib.bl_layout_run_batch(None, 0, 1, 64) == 0
    G = core.Graph(synth.path_graph(5))
    hs = (ctypes.c_void_p * 1)(G.handle)
    sd = np.zeros(1, dtype=np.uint64)
    outs = (ctypes.c_void_p * 1)()
    assert lib.bl_layout_batch(hs, 1, sd.ctypes.data, 1, 0, 0, 1.2, outs) == 1


def test_full_mix_sampled_parity(core):
    """The bench's batched workload at full size (4,096 graphs, n log-uniform in
    [50, 5,000], minibatch 64) in one launch; an even sample of 12 graphs after
    one iteration against the oracle."""
    gs = synth.small_graph_mix(count=4096, seed=4)
    seeds = np.arange(len(gs), dtype=np.uint64)
    _, Ls = _batch(core, gs, seeds, 1, 64)
    for k in np.linspace(0, len(gs) - 1, 12).astype(int):
        g = gs[k]
        xy = synth.uniform_positions(g.n, int(seeds[k]))
        xr, sens = oracle_sensitivity(g, xy, 1, 64, trials=1, nthreads=NCPU)
        assert_positions(("sample", k, g.n), Ls[k].positions(), xr, TOL_POS_EXACT, sens)
