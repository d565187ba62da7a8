"""Exact mode on one thread-block cluster (small graphs): one iteration against
the oracle for ragged sizes and minibatches, CSR in shared or global memory, and
the same invariance to how iterations are split into runs."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import TOL_POS_EXACT, oracle_sensitivity, assert_positions

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


@pytest.fixture
def cluster_engine():
    os.environ["BL_EXACT_ENGINE"] = "cluster"
    yield
    os.environ.pop("BL_EXACT_ENGINE", None)


CASES = [
    ("grid32", lambda: synth.grid_32x32(), 128),
    ("er777", lambda: synth.erdos_renyi(777, 6.0, 5), 64),
    ("tree300_bs1", lambda: synth.binary_tree(300, 2), 1),
    ("er200_onebatch", lambda: synth.erdos_renyi(200, 5.0, 8), 512),
    ("ba3000", lambda: synth.barabasi_albert(3000, 4, seed=9), 256),
    ("dense_er4000", lambda: synth.erdos_renyi(4000, 60.0, 3), 256),   # CSR too big for shared memory
]


@pytest.mark.parametrize("name,maker,bs", CASES)
def test_one_iteration_matches_oracle(core, cluster_engine, name, maker, bs):
    g = maker()
    xy = synth.uniform_positions(g.n, 11)
    L = core.Layout(core.Graph(g), xy=xy)
    L.run(1, bs, "exact")
    xr, sens = oracle_sensitivity(g, xy, 1, bs, nthreads=NCPU)
    _, er = oracle.run(g, xy, iters=1, batch=bs, nthreads=NCPU)
    assert_positions(name, L.positions(), xr, TOL_POS_EXACT, sens)
    assert L.energy_history()[0] == pytest.approx(er[0], rel=1e-4)


def test_three_iterations_with_models(core, cluster_engine):
    g = synth.grid2d(24, 20)
    xy = synth.uniform_positions(g.n, 2)
    for model, a in (("fr", 2), ("linlog", 0)):
        L = core.Layout(core.Graph(g), xy=xy, model=model, K=0.9, R=1.2)
        L.run(3, 64, "exact")
        xr, sens = oracle_sensitivity(g, xy, 3, 64, a=a, K=0.9, R=1.2, nthreads=NCPU)
        assert_positions(model, L.positions(), xr, TOL_POS_EXACT, sens)


def test_split_runs_equal_one_run(core, cluster_engine):
    g = synth.erdos_renyi(1500, 6.0, 4)
    G = core.Graph(g)
    A = core.Layout(G, seed=3)
    A.run(7, 128, "exact")
    B = core.Layout(G, seed=3)
    B.run(3, 128, "exact")
    B.run(4, 128, "exact")
    assert np.array_equal(A.positions(), B.positions())


def test_cluster_and_grid_engines_agree(core):
    """Both engines run the same iteration (different summation orders)."""
    g = synth.grid_32x32()
    xy = synth.uniform_positions(g.n, 0)
    out = {}
    for eng in ("cluster", "grid"):
        os.environ["BL_EXACT_ENGINE"] = eng
        try:
            L = core.Layout(core.Graph(g), xy=xy)
            L.run(2, 128, "exact")
            out[eng] = L.positions()
        finally:
            os.environ.pop("BL_EXACT_ENGINE", None)
    _, sens = oracle_sensitivity(g, xy, 2, 128, nthreads=NCPU)
    assert_positions("cluster vs grid engine", out["cluster"], out["grid"].astype(np.float64), TOL_POS_EXACT,
                     sens, scale=2.0)
