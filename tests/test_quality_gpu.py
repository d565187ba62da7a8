"""Quality metrics (Section 3.7) on the GPU against the FP64 oracle: stress at
the optimal scale, 1-hop neighbourhood preservation and edge uniformity, on the
same positions and the same seeded source/query samples."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth

pytestmark = pytest.mark.gpu

QUERY_SALT = 0x5bd1e995


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def _quality(core, g, xy, nsources=0, nqueries=0, seed=0):
    G = core.Graph(g)
    L = core.Layout(G, xy=xy)
    return L.quality(nsources, nqueries, seed), L.positions()


def _oracle(g, xy, nsources=0, nqueries=0, seed=0):
    src = None if nsources <= 0 or nsources >= g.n else synth.seeded_sample(g.n, nsources, seed)
    qs = None if nqueries <= 0 or nqueries >= g.n else synth.seeded_sample(g.n, nqueries, seed ^ QUERY_SALT)
    st, s_star, pairs = oracle.stress(g, xy, src)
    np_val, used, inter = oracle.neighborhood_preservation(g, xy, qs)
    eu = oracle.edge_uniformity(g, xy)
    return dict(stress=st, scale=s_star, stress_pairs=pairs, np=np_val, np_queries=used,
                np_intersections=inter, edge_uniformity=eu)


def _close(a, b, rel):
    if math.isnan(b):
        return math.isnan(a)
    return abs(a - b) <= rel * max(abs(b), 1e-300)


def _check(q, ref, rel=1e-10):
    assert q["stress_pairs"] == ref["stress_pairs"]
    # stress = pairs - a^2/b cancels: its rounding error scales with the O(1)
    # terms summed (about `pairs` of them), not with the result
    tol = rel * max(abs(ref["stress"]), ref["stress_pairs"])
    assert abs(q["stress"] - ref["stress"]) <= tol, (q["stress"], ref["stress"], tol)
    assert _close(q["scale"], ref["scale"], rel), (q["scale"], ref["scale"])
    # 1-hop neighbourhoods: the same keys in the same precision, so the counts match exactly
    assert q["np_queries"] == ref["np_queries"]
    assert q["np_intersections"] == ref["np_intersections"]
    assert _close(q["np"], ref["np"], 1e-15), (q["np"], ref["np"])
    assert _close(q["edge_uniformity"], ref["edge_uniformity"], rel), (q["edge_uniformity"],
                                                                       ref["edge_uniformity"])


def _grid_xy(rows, cols):
    return np.array([(c, r) for r in range(rows) for c in range(cols)], dtype=np.float32)


def test_grid_at_grid_coordinates_full(core):
    """32x32 grid drawn at its integer coordinates: many equal distances, so NP
    exercises the tie rule; all-pairs stress over 523,776 pairs."""
    g = synth.grid_32x32()
    xy = _grid_xy(32, 32)
    q, _ = _quality(core, g, xy)
    ref = _oracle(g, xy)
    assert ref["stress_pairs"] == g.n * (g.n - 1) / 2
    _check(q, ref)


def test_random_layout_er_full(core):
    g = synth.erdos_renyi(777, 6.0, 5)
    xy = synth.uniform_positions(g.n, 5)
    q, _ = _quality(core, g, xy)
    _check(q, _oracle(g, xy))


def test_evolved_layout_sampled(core):
    """Sampled sources and queries: the C side draws the same seeded sample."""
    g = synth.erdos_renyi(3000, 6.0, 21)
    G = core.Graph(g)
    L = core.Layout(G, seed=21)
    L.run(5, 256, "exact")
    xy = L.positions()
    q = L.quality(200, 300, 7)
    _check(q, _oracle(g, xy, 200, 300, 7))


def test_disconnected_with_isolated_vertices(core):
    """Path + cycle + isolated vertices: unreachable pairs skipped, deg-0
    vertices are not NP queries."""
    edges = [(i, i + 1) for i in range(20)] + [(30 + i, 30 + (i + 1) % 15) for i in range(15)]
    g = synth.from_edge_list(50, edges)
    xy = synth.uniform_positions(g.n, 3)
    q, _ = _quality(core, g, xy)
    ref = _oracle(g, xy)
    _check(q, ref)
    assert ref["np_queries"] == 36   # 21 path vertices + 15 cycle vertices


def test_coincident_positions(core):
    """All vertices at one point: every distance ties, so L_i is the deg(i)
    smallest ids; x = 0 gives stress = number of pairs; EU is 0/0."""
    g = synth.erdos_renyi(200, 5.0, 8)
    xy = np.zeros((g.n, 2), dtype=np.float32)
    q, _ = _quality(core, g, xy)
    ref = _oracle(g, xy)
    _check(q, ref)
    assert q["stress"] == q["stress_pairs"]


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_graphs(core, n):
    g = synth.path_graph(n)
    xy = synth.uniform_positions(n, 1)
    q, _ = _quality(core, g, xy)
    _check(q, _oracle(g, xy))


def test_ba65536_sampled(core):
    """The Barabasi-Albert workload (n = 65,536) at a random layout, 256 BFS
    sources and 512 NP queries."""
    g = synth.ba_65536()
    xy = synth.uniform_positions(g.n, 0)
    q, _ = _quality(core, g, xy, 256, 512, 11)
    _check(q, _oracle(g, xy, 256, 512, 11))


def test_quality_is_scale_invariant(core):
    """Stress at s* and NP do not change when the layout is scaled by 2
    (exactly representable), Section 3.7."""
    g = synth.erdos_renyi(500, 6.0, 9)
    xy = synth.uniform_positions(g.n, 9)
    q1, _ = _quality(core, g, xy)
    q2, _ = _quality(core, g, xy * np.float32(2.0))
    assert abs(q2["stress"] - q1["stress"]) <= 1e-10 * q1["stress_pairs"]
    assert q2["np_intersections"] == q1["np_intersections"]
    assert _close(q2["scale"] * 2.0, q1["scale"], 1e-12)
