"""Pins for the FP64 oracle: closed forms, invariants, special cases and brute
force on tiny inputs. None of these re-calls the oracle to check itself; each
expected value comes from the mathematics of the model (Section 2.2), the
schedule of Algorithms 1/2, the tree rules of Section 3.5 / Algorithm S3, or a
hand-written fixture under tests/golden/.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def two_vertex(d, edge=True):
    g = synth.from_edge_list(2, [(0, 1)] if edge else [])
    xy = np.array([[0.0, 0.0], [d, 0.0]])
    return g, xy


# ---------------------------------------------------------------------------
# force law (Section 2.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("K", [0.5, 1.0, 2.0])
def test_two_vertex_equilibrium_at_K(K):
    """Attraction d^2/K balances repulsion K^2/d exactly at d = K."""
    g, xy = two_vertex(K)
    f, _ = oracle.forces(g, xy, K=K, repulse_neighbors=True)
    assert np.max(np.abs(f)) < 1e-12
    # closer than K: net repulsion (vertex 0 pushed to -x); farther: attraction
    g, xy = two_vertex(0.5 * K)
    f, _ = oracle.forces(g, xy, K=K, repulse_neighbors=True)
    assert f[0, 0] < 0 and f[1, 0] > 0
    g, xy = two_vertex(2.0 * K)
    f, _ = oracle.forces(g, xy, K=K, repulse_neighbors=True)
    assert f[0, 0] > 0 and f[1, 0] < 0


def test_two_vertex_closed_form_values():
    # K=1, d=2, edge and repulsion: 4 - 1/2 = 3.5 towards the other vertex
    g, xy = two_vertex(2.0)
    f, mag = oracle.forces(g, xy, K=1.0, repulse_neighbors=True)
    assert f[0] == pytest.approx([3.5, 0.0], abs=1e-14)
    assert f[1] == pytest.approx([-3.5, 0.0], abs=1e-14)
    assert mag[0] == pytest.approx(4.5, abs=1e-14)
    # default repulsion set excludes neighbours: attraction d^2/K only = 4
    f, _ = oracle.forces(g, xy, K=1.0)
    assert f[0] == pytest.approx([4.0, 0.0], abs=1e-14)
    # no edge, K=2, R=3, d=4: repulsion R K^2 / d = 3 away from the other vertex
    g, xy = two_vertex(4.0, edge=False)
    f, _ = oracle.forces(g, xy, K=2.0, R=3.0)
    assert f[0] == pytest.approx([-3.0, 0.0], abs=1e-14)
    assert f[1] == pytest.approx([3.0, 0.0], abs=1e-14)
    # along a diagonal: d = 5 from a 3-4-5 triangle, K=1: attraction 25 along (3,4)/5
    g = synth.from_edge_list(2, [(0, 1)])
    f, _ = oracle.forces(g, np.array([[1.0, 1.0], [4.0, 5.0]]), K=1.0)
    assert f[0] == pytest.approx([15.0, 20.0], abs=1e-12)


def test_coincident_pair_contributes_zero():
    g = synth.from_edge_list(3, [(0, 1)])
    xy = np.array([[0.5, 0.5], [0.5, 0.5], [0.5, 0.5]])
    f, _ = oracle.forces(g, xy, repulse_neighbors=True)
    assert np.all(f == 0.0)


def _random_case(n, deg, seed):
    g = synth.erdos_renyi(n, deg, seed)
    xy = synth.uniform_positions(n, seed).astype(np.float64)
    return g, xy


@pytest.mark.parametrize("rn", [False, True])
def test_zero_net_force_one_snapshot(rn):
    """Every pair term is antisymmetric (Newton's third law), so the forces of
    one snapshot sum to zero: attraction, repulsion and the neighbour exclusion
    are all symmetric in (i, j)."""
    g, xy = _random_case(60, 5.0, 11)
    f, mag = oracle.forces(g, xy, repulse_neighbors=rn)
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * mag.sum()


def test_translation_invariance_bitwise():
    g, xy = _random_case(50, 4.0, 12)
    f0, _ = oracle.forces(g, xy)
    for shift in (8.0, -4.0, 0.5):
        f1, _ = oracle.forces(g, xy + shift)   # 24-bit inputs: shifts are exact in FP64
        assert np.array_equal(f0, f1)


def test_rotation_by_90_degrees_is_exact():
    g, xy = _random_case(50, 4.0, 13)
    f0, _ = oracle.forces(g, xy)
    rot = np.stack([-xy[:, 1], xy[:, 0]], axis=1)
    f1, _ = oracle.forces(g, rot)
    assert np.array_equal(f1, np.stack([-f0[:, 1], f0[:, 0]], axis=1))


def _dense_forces(A, xy, K, R, rn):
    """Brute force over the dense adjacency matrix (no CSR, no merge)."""
    n = xy.shape[0]
    diff = xy[None, :, :] - xy[:, None, :]          # c_j - c_i
    d = np.sqrt((diff ** 2).sum(-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        att = np.where(d > 0, d / K, 0.0)                 # (d^2/K)/d
        rep = np.where(d > 0, -R * K * K / d ** 2, 0.0)   # (-R K^2/d)/d
    eye = np.eye(n, dtype=bool)
    wrep = ~eye if rn else (~eye & (A == 0))
    coef = A * att + wrep * rep
    return (coef[:, :, None] * diff).sum(axis=1)


@pytest.mark.parametrize("n,rn", [(2, False), (5, True), (9, False), (16, False), (16, True)])
def test_forces_brute_force_tiny(n, rn):
    rng = np.random.default_rng(n)
    A = (rng.random((n, n)) < 0.35).astype(np.int64)
    A = np.triu(A, 1)
    A = A + A.T
    iu, ju = np.nonzero(np.triu(A, 1))
    g = synth.csr_from_edges(n, iu, ju)
    xy = rng.uniform(-1, 1, size=(n, 2))
    f, _ = oracle.forces(g, xy, K=0.7, R=1.3, repulse_neighbors=rn)
    ref = _dense_forces(A, xy, 0.7, 1.3, rn)
    assert np.allclose(f, ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# minibatch semantics and step schedule (Algorithms 1 and 2)
# ---------------------------------------------------------------------------

def _dense_run(A, xy, iters, BS, K, R, rn, step0=1.0):
    """Brute-force minibatch loop over the dense matrices: forces of a batch
    from one snapshot, then the normalised update, Step *= 0.999."""
    xy = xy.copy()
    n = xy.shape[0]
    step = step0
    energies = []
    for _ in range(iters):
        E = 0.0
        for lo in range(0, n, BS):
            hi = min(n, lo + BS)
            F = _dense_forces(A, xy, K, R, rn)[lo:hi]
            for k, i in enumerate(range(lo, hi)):
                nf = math.hypot(F[k, 0], F[k, 1])
                if nf > 0:
                    xy[i] += step * F[k] / nf
                E += nf * nf
        energies.append(E)
        step *= 0.999
    return xy, np.array(energies)


@pytest.mark.parametrize("BS", [1, 3, 7, 12])
def test_run_matches_dense_minibatch_loop(BS):
    n = 12
    rng = np.random.default_rng(100 + BS)
    A = np.triu((rng.random((n, n)) < 0.3).astype(np.int64), 1)
    A = A + A.T
    iu, ju = np.nonzero(np.triu(A, 1))
    g = synth.csr_from_edges(n, iu, ju)
    xy = rng.uniform(-1, 1, size=(n, 2))
    x1, e1 = oracle.run(g, xy, iters=4, batch=BS, K=1.0)
    x2, e2 = _dense_run(A, xy, 4, BS, 1.0, 1.0, False)
    assert np.allclose(x1, x2, rtol=1e-10, atol=1e-10)
    assert np.allclose(e1, e2, rtol=1e-10)


@pytest.mark.parametrize("start", [0, 1, 250])
@pytest.mark.parametrize("BS", [1, 8, 64])
def test_every_vertex_moves_exactly_step(start, BS):
    """c_i += Step * ct_i/|ct_i|: each vertex moves once per iteration by
    exactly Step_t = 0.999^t (t counted from Step=1.0)."""
    g, xy = _random_case(64, 4.0, 21)
    x1, _ = oracle.run(g, xy, iters=1, batch=BS, start_iter=start)
    moved = np.linalg.norm(x1 - xy, axis=1)
    assert np.allclose(moved, 0.999 ** start, rtol=1e-12)


def _pair_distance_jacobi(d0, steps, K):
    d, s, out = d0, 1.0, []
    for _ in range(steps):
        if d > K:
            d = abs(d - 2 * s)
        elif d < K:
            d = d + 2 * s
        out.append(d)
        s *= 0.999
    return out


def _pair_distance_gauss_seidel(d0, steps, K):
    d, s, out = d0, 1.0, []
    for _ in range(steps):
        for _v in range(2):          # vertex 0 moves, then vertex 1 re-evaluates
            if d > K:
                d = abs(d - s)
            elif d < K:
                d = d + s
        out.append(d)
        s *= 0.999
    return out


@pytest.mark.parametrize("d0", [3.5, 0.3, 2.2])
def test_two_vertex_trajectories_closed_form(d0):
    """Two connected vertices with repulsion between them (equilibrium at
    d = K = 1) move along their common line by Step each: minibatch 2 updates
    both from the same snapshot (Jacobi), minibatch 1 is Algorithm 1."""
    g, xy = two_vertex(d0)
    for BS, ref in ((2, _pair_distance_jacobi), (1, _pair_distance_gauss_seidel)):
        expect = ref(d0, 6, 1.0)
        x = xy.copy()
        got = []
        for t in range(6):
            x, e = oracle.run(g, x, iters=1, batch=BS, repulse_neighbors=True, start_iter=t)
            got.append(float(np.linalg.norm(x[1] - x[0])))
        assert np.allclose(got, expect, rtol=1e-12, atol=1e-12), (BS, got, expect)
        assert np.allclose(x[:, 1], 0.0)


def test_energy_is_sum_of_squared_forces_two_vertices():
    d = 3.0
    g, xy = two_vertex(d)
    _, e = oracle.run(g, xy, iters=1, batch=2, repulse_neighbors=True)
    assert e[0] == pytest.approx(2 * (d * d - 1.0 / d) ** 2, rel=1e-14)


def test_batch_one_equals_algorithm_1_by_hand():
    """Three collinear vertices, path 0-1-2, K=1, no repulsion between
    neighbours: Algorithm 1 moves each vertex in turn by Step=1."""
    g = synth.path_graph(3)
    xy = np.array([[0.0, 0.0], [3.0, 0.0], [10.0, 0.0]])
    x, _ = oracle.run(g, xy, iters=1, batch=1)
    # v0: attraction to v1 (+x, 3^2=9), repulsion from v2 (-x, 1/10): 0 -> 1
    # v1 (v0 now at 1): attraction to v0 (-x, 2^2=4) and v2 (+x, 7^2=49): 3 -> 4
    # v2 (v1 now at 4): attraction to v1 (-x, 6^2=36), repulsion from v0 (+x, 1/9): 10 -> 9
    assert x[:, 0] == pytest.approx([1.0, 4.0, 9.0], abs=1e-14)


# ---------------------------------------------------------------------------
# Barnes-Hut (Section 3.5, Algorithms S3-S5)
# ---------------------------------------------------------------------------

def _load_morton_golden():
    rows = []
    with open(os.path.join(GOLDEN, "morton_4x4.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, vid, bits = line.split()
            rows.append((int(k), int(vid), int(bits, 2)))
    return rows


def test_morton_order_fig4_pattern():
    kx, ky = np.meshgrid(np.arange(4), np.arange(4))
    ids = (4 * ky + kx).ravel()
    xy = np.zeros((16, 2), dtype=np.float32)
    xy[ids, 0] = (kx.ravel() + 0.5) / 4.0
    xy[ids, 1] = (ky.ravel() + 0.5) / 4.0
    codes, box = oracle.morton(xy)
    assert box == (0.125, 0.125, 0.75)
    tree = oracle.bh_tree(xy)
    golden = _load_morton_golden()
    assert list(tree["perm"]) == [vid for _, vid, _ in golden]
    assert [int(c >> 28) for c in tree["codes"]] == [bits for _, _, bits in golden]
    # 1 root + 4 level-1 cells + 16 single-vertex leaves at level 2
    assert tree["nnodes"] == 21
    assert list(tree["level"][:6]) == [0, 1, 2, 2, 2, 2]


def test_morton_degenerate_box():
    codes, box = oracle.morton(np.full((5, 2), 0.25, dtype=np.float32))
    assert box[2] == 0.0 and np.all(codes == 0)
    tree = oracle.bh_tree(np.full((5, 2), 0.25, dtype=np.float32))
    # a chain of cells down to the level-16 bucket holding all five vertices
    assert tree["nnodes"] == 17
    assert tree["level"][-1] == 16 and tree["count"][-1] == 5


def _check_tree_invariants(xy, tree):
    n = xy.shape[0]
    m = tree["nnodes"]
    codes = tree["codes"]
    assert np.all(np.diff(codes.astype(np.int64)) >= 0)
    perm = tree["perm"]
    assert sorted(perm.tolist()) == list(range(n))
    # ties broken by vertex id (stable sort)
    same = codes[1:] == codes[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])
    first, count, level, skip = tree["first"], tree["count"], tree["level"], tree["skip"]
    assert first[0] == 0 and count[0] == n and level[0] == 0 and skip[0] == m
    for v in range(m):
        leaf = count[v] == 1 or level[v] == 16
        if leaf:
            assert skip[v] == v + 1
            continue
        # children: v+1, then follow skip links inside [v+1, skip[v])
        c = v + 1
        total = 0
        pos = first[v]
        while c < skip[v]:
            assert level[c] == level[v] + 1
            assert first[c] == pos
            total += count[c]
            pos += count[c]
            c = skip[c]
        assert c == skip[v]
        assert total == count[v]
        # every vertex of the node shares the node's prefix and no vertex outside does
        sh = 32 - 2 * level[v]
        pref = (codes[first[v]:first[v] + count[v]].astype(np.int64) >> sh) if sh < 32 else None
        if pref is not None:
            assert np.all(pref == pref[0])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tree_invariants_random(seed):
    n = 3000
    xy = synth.uniform_positions(n, seed)
    if seed == 2:   # duplicates and a tight cluster exercise level-16 buckets
        xy[:100] = xy[0]
        xy[100:200] = xy[100] + np.float32(1e-6) * np.arange(100, dtype=np.float32)[:, None]
    tree = oracle.bh_tree(xy)
    _check_tree_invariants(xy, tree)
    # node sums: FP32 sums of the node's vertices, within FP32 rounding of FP64
    sx = tree["sumx"].astype(np.float64)
    for v in range(0, tree["nnodes"], 97):
        idx = tree["perm"][tree["first"][v]:tree["first"][v] + tree["count"][v]]
        exact = xy[idx, 0].astype(np.float64).sum()
        assert abs(sx[v] - exact) <= 1e-6 * (np.abs(xy[idx, 0]).sum() + 1e-30) * 4


def test_tree_brute_force_cells_tiny():
    """Nodes = non-empty cells whose parent cell holds >= 2 vertices, from the
    geometry of the 2^l x 2^l grid over the root square (Section 3.5)."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(1, 17))
        xy = rng.uniform(-1, 1, size=(n, 2)).astype(np.float32)
        tree = oracle.bh_tree(xy)
        xmin, ymin = xy[:, 0].min(), xy[:, 1].min()
        D = max(xy[:, 0].max() - xmin, xy[:, 1].max() - ymin)
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.float32(65536.0) / np.float32(D)
            qx = np.nan_to_num(np.minimum(np.floor((xy[:, 0] - xmin) * s), 65535)).astype(np.int64)
            qy = np.nan_to_num(np.minimum(np.floor((xy[:, 1] - ymin) * s), 65535)).astype(np.int64)
        expected = set()
        frontier = [(0, tuple(range(n)))]
        while frontier:
            lev, members = frontier.pop()
            expected.add((lev, members))
            if len(members) == 1 or lev == 16:
                continue
            sh = 16 - (lev + 1)
            cells = {}
            for v in members:
                cells.setdefault((qx[v] >> sh, qy[v] >> sh), []).append(v)
            for mem in cells.values():
                frontier.append((lev + 1, tuple(sorted(mem))))
        got = set()
        for v in range(tree["nnodes"]):
            mem = tree["perm"][tree["first"][v]:tree["first"][v] + tree["count"][v]]
            got.add((int(tree["level"][v]), tuple(sorted(int(u) for u in mem))))
        assert got == expected, trial


@pytest.mark.parametrize("rn", [False, True])
def test_bh_theta_zero_equals_exact(rn):
    """No node passes the MAC at theta = 0, so every vertex is summed directly
    at a leaf: Barnes-Hut reduces to the exact all-pairs repulsion."""
    g, xy = _random_case(300, 5.0, 31)
    xy = xy.astype(np.float32).astype(np.float64)
    fe, me = oracle.forces(g, xy, repulse_neighbors=rn, mode=oracle.EXACT)
    fb, mb = oracle.forces(g, xy, repulse_neighbors=rn, mode=oracle.BH, theta=0.0)
    assert np.max(np.linalg.norm(fe - fb, axis=1) / me) < 1e-13


def test_bh_root_only_at_huge_theta():
    """With theta -> infinity the root passes the MAC for every vertex not at the
    centroid: the repulsion is n * f_r towards the centroid of all vertices."""
    xy = np.array([[0, 0], [1, 0], [0, 1], [3, 2], [-2, 1], [1.5, -1], [2, 2], [-1, -1]],
                  dtype=np.float64) / 4.0
    n = xy.shape[0]
    g = synth.from_edge_list(n, [])
    f, _ = oracle.forces(g, xy, repulse_neighbors=True, mode=oracle.BH, theta=1e18, K=1.0, R=1.0)
    gc = xy.sum(axis=0) / n            # dyadic inputs: the FP32 centroid is exact
    diff = gc[None, :] - xy
    expect = -n * diff / (diff ** 2).sum(axis=1)[:, None]
    assert np.allclose(f, expect, rtol=1e-12, atol=1e-12)


def test_bh_error_shrinks_with_theta():
    g, xy = _random_case(2000, 4.0, 41)
    xy = xy.astype(np.float32).astype(np.float64)
    fe, me = oracle.forces(g, xy, mode=oracle.EXACT)
    errs = []
    for th in (2.0, 1.2, 0.6, 0.3):
        fb, _ = oracle.forces(g, xy, mode=oracle.BH, theta=th)
        errs.append(float(np.mean(np.linalg.norm(fb - fe, axis=1) / me)))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[1] < 0.05


def _dense_bh_theta0_run(A, xy, iters, BS, K, R, rn, start_iter=0):
    """Algorithm S5 by brute force over the dense adjacency matrix at theta = 0,
    where no node passes the MAC and the tree repulsion is the plain sum over every
    other vertex. Per iteration the repulsion is taken once, at the snapshot S of
    the positions at iteration start as the quadtree stores them (FP32, reading
    R7), and without the neighbours unless rn; the attraction of each minibatch is
    taken at the live positions (earlier minibatches already moved)."""
    xy = xy.copy()
    n = xy.shape[0]
    step = 1.0
    for _ in range(start_iter):
        step *= 0.999
    eye = np.eye(n, dtype=bool)
    wrep = ~eye if rn else (~eye & (A == 0))
    energies = []
    for _ in range(iters):
        S = xy.astype(np.float32).astype(np.float64)
        dS = S[None, :, :] - S[:, None, :]
        d2S = (dS ** 2).sum(-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            rep = np.where(wrep & (d2S > 0), -R * K * K / d2S, 0.0)
        Frep = (rep[:, :, None] * dS).sum(axis=1)
        E = 0.0
        for lo in range(0, n, BS):
            hi = min(n, lo + BS)
            diff = xy[None, :, :] - xy[lo:hi, None, :]
            d = np.sqrt((diff ** 2).sum(-1))
            att = A[lo:hi] * np.where(d > 0, d / K, 0.0)       # (d^2/K)/d
            F = (att[:, :, None] * diff).sum(axis=1) + Frep[lo:hi]
            for k, i in enumerate(range(lo, hi)):
                nf = math.hypot(F[k, 0], F[k, 1])
                if nf > 0:
                    xy[i] += step * F[k] / nf
                E += nf * nf
        energies.append(E)
        step *= 0.999
    return xy, np.array(energies)


@pytest.mark.parametrize("BS", [1, 3, 12])
@pytest.mark.parametrize("rn", [False, True])
def test_bh_run_matches_dense_snapshot_loop(BS, rn):
    """The oracle's Barnes-Hut iteration (Algorithm S5) at theta = 0 against the
    dense brute force above: the tree is built once per iteration from the
    snapshot, the attraction follows the live positions. Rebuilding the tree per
    minibatch, or taking the attraction at the snapshot, fails this."""
    n = 13
    rng = np.random.default_rng(200 + BS + 7 * rn)
    A = np.triu((rng.random((n, n)) < 0.3).astype(np.int64), 1)
    A = A + A.T
    iu, ju = np.nonzero(np.triu(A, 1))
    g = synth.csr_from_edges(n, iu, ju)
    xy = rng.uniform(-1, 1, size=(n, 2))
    x1, e1 = oracle.run(g, xy, iters=3, batch=BS, mode=oracle.BH, theta=0.0, repulse_neighbors=rn,
                        start_iter=4)
    x2, e2 = _dense_bh_theta0_run(A, xy, 3, BS, 1.0, 1.0, rn, start_iter=4)
    assert np.allclose(x1, x2, rtol=1e-10, atol=1e-10)
    assert np.allclose(e1, e2, rtol=1e-10)


def _pair_bh_gauss_seidel(x0, x1, iters, K, start_iter):
    """Two vertices joined by an edge on the x axis, minibatch 1, repulsion
    between them (repulse_neighbors): vertex 0 moves, then vertex 1. The
    attraction follows the live positions, the repulsion the iteration's snapshot
    (FP32, as the tree stores it), and each vertex moves by Step towards the sign
    of its net force."""
    step = 1.0
    for _ in range(start_iter):
        step *= 0.999
    out = []
    for _ in range(iters):
        s0, s1 = float(np.float32(x0)), float(np.float32(x1))
        dS = abs(s1 - s0)
        f0 = math.copysign((x1 - x0) ** 2 / K, x1 - x0) + math.copysign(K * K / dS, s0 - s1)
        x0 += math.copysign(step, f0)
        f1 = math.copysign((x0 - x1) ** 2 / K, x0 - x1) + math.copysign(K * K / dS, s1 - s0)
        x1 += math.copysign(step, f1)
        out.append((x0, x1, f0 * f0 + f1 * f1))
        step *= 0.999
    return out


def test_bh_two_vertex_trajectory_closed_form():
    """At d = 1.4 and Step ~ 0.5 vertex 0 is pulled to d = 0.9; vertex 1 then
    feels the live attraction 0.81 against the snapshot repulsion 1/1.4 and is
    pulled too, where the exact mode (repulsion 1/0.9) would push it away."""
    g = synth.from_edge_list(2, [(0, 1)])
    x0, x1, start = 0.0, 1.4, 693
    expect = _pair_bh_gauss_seidel(x0, x1, 6, 1.0, start)
    x = np.array([[x0, 0.0], [x1, 0.0]])
    for t in range(6):
        x, e = oracle.run(g, x, iters=1, batch=1, mode=oracle.BH, theta=1.2, repulse_neighbors=True,
                          start_iter=start + t)
        assert x[0, 0] == pytest.approx(expect[t][0], abs=1e-12), t
        assert x[1, 0] == pytest.approx(expect[t][1], abs=1e-12), t
        assert e[0] == pytest.approx(expect[t][2], rel=1e-12), t
        assert np.all(x[:, 1] == 0.0)
    assert expect[0][1] < 1.0        # pulled in the first iteration
    xe, _ = oracle.run(g, np.array([[x0, 0.0], [x1, 0.0]]), iters=1, batch=1, repulse_neighbors=True,
                       start_iter=start)
    assert xe[1, 0] > 1.8            # the exact mode pushes vertex 1 away instead


def _fig4_grid():
    """16 vertices at the centres of a 4 x 4 grid of cells in [0,1]^2 (Fig. 4):
    root side D = 0.75, four quadrant nodes, sixteen one-vertex leaves."""
    c = (np.arange(4) + 0.5) / 4.0
    X, Y = np.meshgrid(c, c)
    return np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float32)


def test_bh_mac_counts_fig4_grid_by_hand():
    """MAC decisions counted by hand on the Fig. 4 grid. The root (D^2 = 0.5625)
    never passes for theta <= 1.2 (every vertex is within d^2 = 0.28125 of the
    centre). A quadrant node (D^2 = 0.140625) passes at theta = 1.2 when
    d^2 > 0.0977 (every other quadrant: 3 far nodes, 4 leaves per vertex) and at
    theta = 0.6 when d^2 > 0.390625: a corner vertex accepts the 3 other quadrants
    (4 leaves), a vertex with one coordinate on the rim accepts 2 (8 leaves), an
    inner vertex none (16 leaves)."""
    xy = _fig4_grid()
    assert oracle.bh_interactions(xy, 1.2) == (48, 64)
    assert oracle.bh_interactions(xy, 0.6) == (4 * 7, 4 * 36)
    assert oracle.bh_interactions(xy, 0.0) == (0, 256)       # every leaf, no far node
    assert oracle.bh_interactions(xy, 1e18) == (16, 0)       # the root, for all 16
    far, near = oracle.bh_query_counts(xy, 0.6)
    rim = ((xy == np.float32(0.125)) | (xy == np.float32(0.875))).sum(axis=1)
    expect_far = np.choose(rim, [0, 2, 3])
    expect_near = np.choose(rim, [16, 8, 4])
    assert np.array_equal(far, expect_far) and np.array_equal(near, expect_near)
    far, near = oracle.bh_query_counts(xy, 1.2)
    assert np.all(far == 3) and np.all(near == 4)


def test_bh_mac_counts_limits_random():
    """theta = 0: no node is accepted and every query meets all n vertices at the
    leaves (distinct codes); a huge theta accepts the root once per vertex that
    is not at the centroid."""
    xy = synth.uniform_positions(500, 17)
    far, near = oracle.bh_query_counts(xy, 0.0)
    assert np.all(far == 0) and np.all(near == 500)
    far, near = oracle.bh_query_counts(xy, 1e18)
    assert np.all(far == 1) and np.all(near == 0)
    assert oracle.bh_interactions(xy, 0.7) == (int(oracle.bh_query_counts(xy, 0.7)[0].sum()),
                                              int(oracle.bh_query_counts(xy, 0.7)[1].sum()))


# ---------------------------------------------------------------------------
# quality metrics (Section 3.7)
# ---------------------------------------------------------------------------

def test_stress_zero_for_path_at_hop_distances():
    g = synth.path_graph(7)
    xy = np.stack([np.arange(7.0) * 3.0, np.zeros(7)], axis=1)   # any scale
    st, s, pairs = oracle.stress(g, xy)
    assert st == pytest.approx(0.0, abs=1e-12)
    assert s == pytest.approx(1.0 / 3.0, rel=1e-12)
    assert pairs == 21


def test_stress_unit_square_closed_form():
    g = synth.cycle_graph(4)
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
    st, s, _ = oracle.stress(g, xy)
    r2 = math.sqrt(2.0)
    assert s == pytest.approx((4 + r2) / 5, rel=1e-12)
    assert st == pytest.approx((12 - 8 * r2) / 5, rel=1e-12)
    st2, _, _ = oracle.stress(g, xy * 7.5)
    assert st2 == pytest.approx(st, rel=1e-12)


def test_stress_every_source_sampled_equals_all_pairs():
    """With every vertex as a sampled source each unordered pair is met twice:
    the ordered sums double and the n / (2 n) rescale restores the all-pairs
    stress; the optimal scale is unchanged and the pair count doubles."""
    g = synth.erdos_renyi(40, 4.0, 7)
    xy = synth.uniform_positions(40, 7)
    st, s, p = oracle.stress(g, xy)
    st2, s2, p2 = oracle.stress(g, xy, sources=np.arange(40))
    assert p2 == 2 * p
    assert st2 == pytest.approx(st, rel=1e-12)
    assert s2 == pytest.approx(s, rel=1e-12)


def test_stress_sampled_sources_by_hand():
    """Path 0-1-2-3 drawn at x = 0, 1, 3, 6 plus an isolated vertex 4.
    Source 0: hop distances 1, 2, 3, layout distances 1, 3, 6, so x/d = 1, 1.5, 2:
    a = 9/2, b = 29/4, stress = 3 - a^2/b = 6/29, scaled by n/(2 ns) = 5/2.
    Sources {0, 3}: source 3 adds x/d = 2, 2.5, 3: a = 12, b = 53/2,
    stress = 6 - 288/53 = 30/53, scaled by 5/4. Vertex 4 is unreachable."""
    g = synth.from_edge_list(5, [(0, 1), (1, 2), (2, 3)])
    xy = np.array([[0, 0], [1, 0], [3, 0], [6, 0], [100, 0]], dtype=np.float64)
    st, s, p = oracle.stress(g, xy, sources=[0])
    assert (st, s, p) == (pytest.approx(2.5 * 6 / 29, rel=1e-13), pytest.approx(18 / 29, rel=1e-13), 3)
    st, s, p = oracle.stress(g, xy, sources=[0, 3])
    assert (st, s, p) == (pytest.approx(1.25 * 30 / 53, rel=1e-13), pytest.approx(24 / 53, rel=1e-13), 6)


def test_neighborhood_preservation_closed_forms():
    n = 9
    ang = 2 * np.pi * np.arange(n) / n
    poly = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    npv, used, _ = oracle.neighborhood_preservation(synth.cycle_graph(n), poly)
    assert npv == pytest.approx(1.0) and used == n
    # star with k leaves on the unit circle: hub J=1; for k >= 7 each leaf's
    # nearest point is a leaf (2 sin(pi/k) < 1), J=0; for k=4 the hub, J=1
    for k, expect in ((8, 1.0 / 9.0), (4, 1.0)):
        ang = 2 * np.pi * np.arange(k) / k
        xy = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], axis=1)])
        g = synth.from_edge_list(k + 1, [(0, i) for i in range(1, k + 1)])
        npv, _, _ = oracle.neighborhood_preservation(g, xy)
        assert npv == pytest.approx(expect, rel=1e-12)


def test_edge_uniformity_closed_forms():
    n = 6
    ang = 2 * np.pi * np.arange(n) / n
    poly = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    assert oracle.edge_uniformity(synth.cycle_graph(n), poly) == pytest.approx(0.0, abs=1e-7)
    # path with edge lengths 1 and 3: mean 2, sqrt((1+1)/(2*4)) = 0.5
    xy = np.array([[0, 0], [1, 0], [4, 0]], dtype=np.float64)
    assert oracle.edge_uniformity(synth.path_graph(3), xy) == pytest.approx(0.5, rel=1e-12)


def test_greedy_init_tree_edges_have_unit_length():
    """Algorithm 3 places each newly reached vertex on the unit circle around the
    vertex that reached it: in a tree every edge has length 1."""
    g = synth.binary_tree(200, 3)
    x = oracle.greedy_init(g, np.zeros((200, 2)))
    lens = []
    for i in range(g.n):
        for k in range(g.rowptr[i], g.rowptr[i + 1]):
            lens.append(np.linalg.norm(x[g.colids[k]] - x[i]))
    assert np.allclose(lens, 1.0, atol=1e-12)


# ---- (a,r)-energy models (Section 2.2): attraction d^a / K, repulsion R K^2 / d ----

@pytest.mark.parametrize("a", [0, 1, 2, 3])
@pytest.mark.parametrize("K,R", [(1.0, 1.0), (0.5, 2.0), (2.0, 0.5)])
def test_model_two_vertex_equilibrium(a, K, R):
    """d^a / K = R K^2 / d at d* = (R K^3)^(1/(a+1)): zero net force there,
    repulsion inside, attraction outside."""
    dstar = (R * K ** 3) ** (1.0 / (a + 1))
    g, xy = two_vertex(dstar)
    f, mag = oracle.forces(g, xy, K=K, R=R, a=a, repulse_neighbors=True)
    assert np.max(np.abs(f)) <= 1e-12 * mag.max()
    g, xy = two_vertex(0.5 * dstar)
    f, _ = oracle.forces(g, xy, K=K, R=R, a=a, repulse_neighbors=True)
    assert f[0, 0] < 0 and f[1, 0] > 0
    g, xy = two_vertex(2.0 * dstar)
    f, _ = oracle.forces(g, xy, K=K, R=R, a=a, repulse_neighbors=True)
    assert f[0, 0] > 0 and f[1, 0] < 0


@pytest.mark.parametrize("a,expect", [(0, 0.5), (1, 1.5), (2, 4.5), (3, 13.5)])
def test_model_attraction_closed_form(a, expect):
    """One edge of length d = 3, K = 2: |f| = 3^a / 2 towards the other end
    (neighbours do not repel by default)."""
    g, xy = two_vertex(3.0)
    f, _ = oracle.forces(g, xy, K=2.0, a=a)
    assert f[0] == pytest.approx([expect, 0.0], abs=1e-13)
    assert f[1] == pytest.approx([-expect, 0.0], abs=1e-13)


def test_model_default_is_fruchterman_reingold():
    g = synth.erdos_renyi(60, 5.0, 1)
    xy = synth.uniform_positions(60, 1)
    f2, m2 = oracle.forces(g, xy, a=2)
    fd, md = oracle.forces(g, xy)
    assert np.array_equal(f2, fd) and np.array_equal(m2, md)


def test_model_out_of_range_is_rejected():
    g, xy = two_vertex(1.0)
    with pytest.raises(Exception):
        oracle.forces(g, xy, a=4)
