"""bl_force_params.kahan on every engine: compensated (1) and plain (0) FP32
repulsion sums both stay within the parity tolerance of the FP64 oracle, and the
flag changes the bits of the result on every engine; the default (-1) is plain
below 1,000,000 vertices; other values are refused."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import (TOL_FORCE_BH, TOL_FORCE_EXACT, TOL_POS_EXACT, assert_forces, assert_positions,
                     oracle_sensitivity)

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


@pytest.mark.parametrize("mode,tol", [("exact", TOL_FORCE_EXACT), ("bh", TOL_FORCE_BH)])
def test_snapshot_forces_both_ways(core, mode, tol):
    """The whole-GPU exact engine (12 column tiles per row) and the Barnes-Hut walk."""
    g = synth.erdos_renyi(12000, 6.0, 31)
    xy = synth.uniform_positions(g.n, 31)
    G = core.Graph(g)
    om = oracle.EXACT if mode == "exact" else oracle.BH
    ref, mag = oracle.forces(g, xy.astype(np.float64), mode=om, theta=1.2, nthreads=NCPU)
    f = {}
    for k in (0, 1, -1):
        L = core.Layout(G, xy=xy, kahan=k)
        f[k] = L.debug_forces(mode, 1.2)
        assert_forces((mode, "kahan", k), f[k], ref, mag, tol)
    assert not np.array_equal(f[0], f[1])
    assert np.array_equal(f[-1], f[0])      # n < 1,000,000: plain by default


@pytest.mark.parametrize("engine", ["grid", "cluster", "batched"])
def test_one_iteration_both_ways(core, engine):
    g = synth.erdos_renyi(3000, 6.0, 32)
    xy = synth.uniform_positions(g.n, 32)
    G = core.Graph(g)
    bs = 64 if engine == "batched" else 256
    xr, sens = oracle_sensitivity(g, xy, 1, bs, nthreads=NCPU)
    out = {}
    for k in (0, 1):
        L = core.Layout(G, xy=xy, kahan=k)
        if engine == "batched":
            core.run_batch([L], 1, bs)
        else:
            os.environ["BL_EXACT_ENGINE"] = engine
            try:
                L.run(1, bs, "exact")
            finally:
                os.environ.pop("BL_EXACT_ENGINE", None)
        out[k] = L.positions()
        assert_positions((engine, "kahan", k), out[k], xr, TOL_POS_EXACT, sens)
    assert not np.array_equal(out[0], out[1]), engine


def test_bad_kahan_value_is_refused(core):
    G = core.Graph(synth.path_graph(4))
    with pytest.raises(core.BatchLayoutError) as e:
        core.Layout(G, seed=0, kahan=2)
    assert e.value.status == core.BL_EINVAL
