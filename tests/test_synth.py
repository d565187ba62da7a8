"""Seeded input generators: shapes, determinism, CSR hygiene."""
import numpy as np
import pytest

from paper_2002_08233_gb300 import synth


def _check_csr(g):
    rp, ci = g.rowptr, g.colids
    assert rp.dtype == np.int32 and ci.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    for i in range(g.n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)      # sorted, no duplicates
        assert not np.any(row == i)          # no self-loops
    # symmetric
    a = np.repeat(np.arange(g.n), np.diff(rp))
    fwd = set(zip(a.tolist(), ci.tolist()))
    assert all((j, i) in fwd for (i, j) in fwd)


def test_grid_32x32_shape():
    g = synth.grid_32x32()
    assert g.n == 1024 and g.n_edges == 1984 and g.nnz == 3968
    _check_csr(g)


def test_ba_shape_small():
    g = synth.barabasi_albert(2000, 4, seed=1)
    assert g.n_edges == 10 + (2000 - 5) * 4
    _check_csr(g)
    assert synth.barabasi_albert(2000, 4, seed=1).colids.tobytes() == g.colids.tobytes()


def test_rmat_small():
    g = synth.rmat(10, 8, seed=3)
    assert g.n == 1024
    _check_csr(g)
    deg = g.degrees()
    assert deg[:64].mean() > deg[-512:].mean()   # low ids are the hubs for a=0.57


@pytest.mark.parametrize("maker", [
    lambda: synth.binary_tree(300, 1),
    lambda: synth.erdos_renyi(300, 6.0, 2),
    lambda: synth.tri_mesh(10, 13, 3),
    lambda: synth.cycle_graph(7),
])
def test_small_families(maker):
    _check_csr(maker())


def test_binary_tree_degrees():
    g = synth.binary_tree(500, 7)
    assert g.n_edges == 499
    assert g.degrees().max() <= 3


def test_uniform_positions_splitmix64_reference_values():
    # SplitMix64 from state 0: first outputs published with the generator
    z = synth.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    xy = synth.uniform_positions(1000, 0)
    assert xy.dtype == np.float32 and xy.shape == (1000, 2)
    assert xy.min() >= -1.0 and xy.max() < 1.0
    # 24-bit grid: exact multiples of 2^-23
    assert np.all((xy.astype(np.float64) * (1 << 23)) % 1 == 0)
    assert not np.array_equal(xy, synth.uniform_positions(1000, 1))


def test_small_graph_mix_sizes():
    gs = synth.small_graph_mix(count=60, seed=4)
    ns = np.array([g.n for g in gs])
    assert ns.min() >= 40 and ns.max() <= 5100


def test_seeded_sample_is_distinct_and_seeded():
    s = synth.seeded_sample(1000, 100, 7)
    assert s.dtype == np.int32 and len(s) == 100
    assert len(set(s.tolist())) == 100 and s.min() >= 0 and s.max() < 1000
    assert np.array_equal(s, synth.seeded_sample(1000, 100, 7))
    assert not np.array_equal(s, synth.seeded_sample(1000, 100, 8))
    # step 0 swaps entry 0 with entry z_0 mod n
    z0 = int(synth.splitmix64(7, 1)[0])
    assert s[0] == z0 % 1000
    # m = n gives a permutation
    p = synth.seeded_sample(50, 50, 3)
    assert sorted(p.tolist()) == list(range(50))
