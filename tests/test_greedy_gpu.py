"""Greedy initialisation (Algorithm 3) in the library against the oracle's, and
its closed-form property: on a tree every edge from a vertex to the neighbour it
placed has length 1."""
import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def _oracle_greedy(g, seed, v0):
    xy = synth.uniform_positions(g.n, seed).astype(np.float64)
    return oracle.greedy_init(g, xy, v0).astype(np.float32)


@pytest.mark.parametrize("maker,v0", [
    (lambda: synth.binary_tree(300, 2), 0),
    (lambda: synth.grid2d(17, 23), 100),
    (lambda: synth.erdos_renyi(500, 6.0, 3), 7),
    (lambda: synth.barabasi_albert(2000, 4, seed=5), 1999),
])
def test_greedy_matches_oracle(core, maker, v0):
    g = maker()
    L = core.greedy_layout(core.Graph(g), v0=v0, seed=11)
    assert np.array_equal(L.positions(), _oracle_greedy(g, 11, v0))


def test_tree_edges_have_unit_length(core):
    g = synth.binary_tree(511, 4)
    xy = core.greedy_layout(core.Graph(g), v0=0, seed=1).positions().astype(np.float64)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    lens = np.linalg.norm(xy[g.colids] - xy[rows], axis=1)
    # a tree's DFS from any root places every vertex on its parent's unit circle
    assert np.allclose(lens, 1.0, atol=1e-5)


def test_unreached_vertices_keep_seeded_positions(core):
    edges = [(i, i + 1) for i in range(9)] + [(20 + i, 21 + i) for i in range(5)]
    g = synth.from_edge_list(30, edges)
    xy = core.greedy_layout(core.Graph(g), v0=3, seed=8).positions()
    seeded = synth.uniform_positions(g.n, 8)
    assert np.array_equal(xy[10:], seeded[10:])            # other component and isolated vertices
    assert np.array_equal(xy[3], np.zeros(2, np.float32))  # the start vertex sits at the origin
    assert np.array_equal(xy, _oracle_greedy(g, 8, 3))


def test_seeded_start_vertex(core):
    g = synth.erdos_renyi(400, 5.0, 9)
    v0 = int(synth.splitmix64(21, 1)[0] % np.uint64(g.n))
    L = core.greedy_layout(core.Graph(g), v0=-1, seed=21)
    assert np.array_equal(L.positions(), _oracle_greedy(g, 21, v0))


def test_bad_start_vertex(core):
    g = synth.path_graph(5)
    with pytest.raises(core.BatchLayoutError):
        core.greedy_layout(core.Graph(g), v0=5)
