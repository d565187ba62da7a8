"""Barnes-Hut parity (Section 3.5, Algorithms S3-S5): Morton codes, sort and
quadtree bit-exact against the oracle built by the same rules; tree-walk forces
and one-iteration positions within the BH tolerance; acceptance decisions equal
(the walk's interaction counts)."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import TOL_FORCE_BH, TOL_POS_BH, oracle_sensitivity, assert_positions, assert_forces

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def _layout(core, g, xy, **kw):
    G = core.Graph(g)
    return G, core.Layout(G, xy=xy, **kw)


def _assert_tree_equal(gpu, ref):
    assert np.array_equal(gpu["codes"], ref["codes"])
    assert np.array_equal(gpu["perm"], ref["perm"])
    assert gpu["nnodes"] == ref["nnodes"]
    for key in ("first", "count", "level", "skip"):
        assert np.array_equal(gpu[key], ref[key]), key
    assert np.array_equal(gpu["sumx"], ref["sumx"])
    assert np.array_equal(gpu["sumy"], ref["sumy"])


def _fig4_positions():
    kx, ky = np.meshgrid(np.arange(4), np.arange(4))
    ids = (4 * ky + kx).ravel()
    xy = np.zeros((16, 2), dtype=np.float32)
    xy[ids, 0] = (kx.ravel() + 0.5) / 4.0
    xy[ids, 1] = (ky.ravel() + 0.5) / 4.0
    return xy


TREE_CASES = {
    "fig4": lambda: _fig4_positions(),
    "one": lambda: np.array([[0.3, -0.2]], np.float32),
    "two": lambda: np.array([[0.0, 0.0], [1.0, 1.0]], np.float32),
    "coincident": lambda: np.full((9, 2), 0.25, np.float32),
    "random3000": lambda: synth.uniform_positions(3000, 5),
    "clusters": lambda: np.concatenate([
        np.repeat(synth.uniform_positions(1, 9), 50, axis=0),
        synth.uniform_positions(2000, 10) * np.float32(1e-4),
        synth.uniform_positions(1000, 11)]).astype(np.float32),
    "ragged70001": lambda: synth.uniform_positions(70001, 12),
}


@pytest.mark.parametrize("name", list(TREE_CASES))
def test_tree_bit_exact(core, name):
    xy = TREE_CASES[name]()
    g = synth.from_edge_list(xy.shape[0], [])
    _, L = _layout(core, g, xy)
    gpu = L.debug_bh_tree()
    ref = oracle.bh_tree(xy)
    codes, box = oracle.morton(xy)
    assert gpu["box"] == box
    _assert_tree_equal(gpu, ref)


BH_CASES = [
    ("er2000", lambda: synth.erdos_renyi(2000, 6.0, 3), 3),
    ("ba5000", lambda: synth.barabasi_albert(5000, 4, seed=2), 2),
    ("rmat12", lambda: synth.rmat(12, 8, seed=7), 7),
]


@pytest.mark.parametrize("name,maker,seed", BH_CASES)
@pytest.mark.parametrize("theta", [0.0, 0.6, 1.2])
@pytest.mark.parametrize("rn", [False, True])
def test_bh_forces_match_oracle(core, name, maker, seed, theta, rn):
    g = maker()
    xy = synth.uniform_positions(g.n, seed)
    _, L = _layout(core, g, xy, repulse_neighbors=rn)
    f = L.debug_forces("bh", theta)
    ref, mag = oracle.forces(g, xy.astype(np.float64), mode=oracle.BH, theta=theta,
                             repulse_neighbors=rn, nthreads=NCPU)
    assert_forces((name, theta, rn), f, ref, mag, TOL_FORCE_BH)
    # identical acceptance decisions, query by query: accepted nodes and leaf vertices met
    far, near = oracle.bh_query_counts(xy, theta)
    gfar, gnear = L.debug_bh_counts(theta)
    bad = np.flatnonzero((gfar != far) | (gnear != near))
    assert bad.size == 0, (name, theta, bad[:10], gfar[bad[:10]], far[bad[:10]])
    st = L.stats()
    assert st["bh_far_nodes"] == far.sum() and st["bh_near_pairs"] == near.sum()


def test_bh_theta_zero_equals_exact_engine(core):
    g = synth.erdos_renyi(1500, 5.0, 4)
    xy = synth.uniform_positions(g.n, 4)
    _, L = _layout(core, g, xy)
    fb = L.debug_forces("bh", 0.0).astype(np.float64)
    fe = L.debug_forces("exact").astype(np.float64)
    _, mag = oracle.forces(g, xy.astype(np.float64))
    assert_forces("bh theta 0 vs exact engine", fb, fe, mag, 2 * TOL_FORCE_BH)


@pytest.mark.parametrize("name,maker,bs,seed", [
    ("er2000_bs256", lambda: synth.erdos_renyi(2000, 6.0, 3), 256, 3),
    ("ba5000_bs100", lambda: synth.barabasi_albert(5000, 4, seed=2), 100, 2),
    ("tree3000_bs64", lambda: synth.binary_tree(3000, 5), 64, 5),
])
def test_bh_one_iteration_positions(core, name, maker, bs, seed):
    g = maker()
    xy = synth.uniform_positions(g.n, seed)
    _, L = _layout(core, g, xy)
    L.run(1, bs, "bh", 1.2)
    xr, sens = oracle_sensitivity(g, xy, 1, bs, mode=oracle.BH, theta=1.2, nthreads=NCPU)
    assert_positions(name, L.positions(), xr, TOL_POS_BH, sens)
    _, er = oracle.run(g, xy, 1, bs, mode=oracle.BH, theta=1.2, nthreads=NCPU)
    assert L.energy_history()[0] == pytest.approx(er[0], rel=1e-3)


def _hubs_graph(n=40000, seed=21):
    """ER background plus three hubs: vertex n-1 adjacent to every other vertex
    (its earlier-minibatch columns fill the sweep's maximum of 257 segments, each
    longer than one 128-column round), vertex n-300 to 5,000 random vertices (40
    segments: partial sums read after the gather) and vertex 30,000 to 2,000 (16
    segments: partial sums polled with the gather)."""
    bg = synth.erdos_renyi(n, 4.0, seed)
    rows = np.repeat(np.arange(n), np.diff(bg.rowptr.astype(np.int64)))
    u, v = [rows], [bg.colids.astype(np.int64)]
    rng = np.random.default_rng(seed)
    u.append(np.full(n - 1, n - 1)); v.append(np.arange(n - 1))
    u.append(np.full(5000, n - 300)); v.append(rng.choice(n - 300, 5000, replace=False))
    u.append(np.full(2000, 30000)); v.append(rng.choice(30000, 2000, replace=False))
    return synth.csr_from_edges(n, np.concatenate(u), np.concatenate(v), name="hubs40000")


def test_bh_long_rows_positions(core):
    """Rows of many sweep segments (the long-row paths of the sweep) against the
    oracle's Algorithm S5 iteration."""
    g = _hubs_graph()
    xy = synth.uniform_positions(g.n, 4)
    _, L = _layout(core, g, xy)
    L.run(1, 256, "bh", 1.2)
    xr, sens = oracle_sensitivity(g, xy, 1, 256, mode=oracle.BH, theta=1.2, nthreads=NCPU)
    assert_positions("hubs40000", L.positions(), xr, TOL_POS_BH, sens)


def test_bh_multi_iteration_continues(core):
    g = synth.erdos_renyi(3000, 5.0, 6)
    xy = synth.uniform_positions(g.n, 6)
    _, L = _layout(core, g, xy, start_iter=5)
    L.run(2, 256, "bh", 1.2)
    L.run(1, 256, "bh", 1.2)
    st = L.stats()
    assert st["iterations"] == 8
    xr, sens = oracle_sensitivity(g, xy, 3, 256, mode=oracle.BH, theta=1.2, start_iter=5,
                                  nthreads=NCPU)
    assert_positions("bh continues", L.positions(), xr, TOL_POS_BH, sens)


def test_bh_every_vertex_moves_by_step(core):
    g = synth.rmat(12, 8, seed=8)
    xy = synth.uniform_positions(g.n, 8)
    _, L = _layout(core, g, xy, start_iter=20)
    L.run(1, 256, "bh", 1.2)
    moved = np.linalg.norm(L.positions().astype(np.float64) - xy, axis=1)
    assert np.allclose(moved, 0.999 ** 20, rtol=2e-6)


# ---- full-size workload: R-MAT scale 20, minibatch 256, theta 1.2 -------------------

@pytest.fixture(scope="module")
def rmat20():
    return synth.rmat_scale20()


def test_rmat20_tree_bit_exact(core, rmat20):
    g = rmat20
    xy = synth.uniform_positions(g.n, 0)
    _, L = _layout(core, g, xy)
    gpu = L.debug_bh_tree()
    ref = oracle.bh_tree(xy)
    _assert_tree_equal(gpu, ref)


def test_rmat20_sampled_forces(core, rmat20):
    g = rmat20
    xy = synth.uniform_positions(g.n, 0)
    _, L = _layout(core, g, xy)
    f = L.debug_forces("bh", 1.2)
    rng = np.random.default_rng(1)
    for b in rng.choice(g.n // 256, size=4, replace=False):
        lo, hi = int(b) * 256, int(b) * 256 + 256
        ref, mag = oracle.forces(g, xy.astype(np.float64), mode=oracle.BH, theta=1.2, lo=lo, hi=hi,
                                 nthreads=NCPU)
        assert_forces(("rmat20", lo), f[lo:hi], ref, mag, TOL_FORCE_BH)
    # the hub rows of the first minibatch
    ref, mag = oracle.forces(g, xy.astype(np.float64), mode=oracle.BH, theta=1.2, lo=0, hi=256,
                             nthreads=NCPU)
    assert_forces(("rmat20", 0), f[:256], ref, mag, TOL_FORCE_BH)


def test_rmat20_one_iteration_positions(core, rmat20):
    """The bench's R-MAT scale-20 workload, one whole iteration (tree, walk,
    edge pass, dataflow sweep) against the oracle's Algorithm S5 iteration."""
    g = rmat20
    xy = synth.uniform_positions(g.n, 0)
    _, L = _layout(core, g, xy)
    L.run(1, 256, "bh", 1.2)
    xr, sens = oracle_sensitivity(g, xy, 1, 256, trials=1, mode=oracle.BH, theta=1.2, nthreads=NCPU)
    assert_positions("rmat20 one iteration", L.positions(), xr, TOL_POS_BH, sens)
