"""(a,r)-energy models (Section 2.2): attraction |d|^a / K with a in {0,1,2,3},
repulsion R K^2 / |d|, on every engine against the FP64 oracle with the same
exponent."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import (TOL_FORCE_BH, TOL_FORCE_EXACT, TOL_POS_BH, TOL_POS_EXACT, force_error,
                     oracle_sensitivity, assert_positions, assert_forces)

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1
MODELS = [("fr", 2), ("fa", 1), ("linlog", 0), ("a3", 3)]


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


@pytest.mark.parametrize("model,a", MODELS)
@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_snapshot_forces(core, model, a, mode):
    g = synth.erdos_renyi(1500, 6.0, 3)
    xy = synth.uniform_positions(g.n, 3) * np.float32(2.0)
    L = core.Layout(core.Graph(g), xy=xy, K=0.8, R=1.5, model=model)
    f = L.debug_forces(mode, theta=0.6)
    ref, mag = oracle.forces(g, xy.astype(np.float64), K=0.8, R=1.5, a=a,
                             mode=oracle.EXACT if mode == "exact" else oracle.BH, theta=0.6,
                             nthreads=NCPU)
    tol = TOL_FORCE_EXACT if mode == "exact" else TOL_FORCE_BH
    assert_forces((model, mode), f, ref, mag, tol)


@pytest.mark.parametrize("model,a", MODELS)
@pytest.mark.parametrize("engine", ["exact", "exact_grid", "bh", "batched"])
def test_one_iteration(core, model, a, engine):
    """exact: the default engine at this size (one thread-block cluster);
    exact_grid: the whole-GPU engine forced."""
    g = synth.grid2d(20, 25)
    xy = synth.uniform_positions(g.n, 7)
    L = core.Layout(core.Graph(g), xy=xy, model=model)
    if engine == "batched":
        core.run_batch([L], 1, 64)
    elif engine == "exact_grid":
        os.environ["BL_EXACT_ENGINE"] = "grid"
        try:
            L.run(1, 64, "exact")
        finally:
            os.environ.pop("BL_EXACT_ENGINE", None)
    else:
        L.run(1, 64, engine, 1.2)
    mode = oracle.BH if engine == "bh" else oracle.EXACT
    xr, sens = oracle_sensitivity(g, xy, 1, 64, mode=mode, theta=1.2, a=a, nthreads=NCPU)
    base = TOL_POS_BH if engine == "bh" else TOL_POS_EXACT
    assert_positions((model, engine), L.positions(), xr, base, sens)


@pytest.mark.parametrize("model,a", MODELS)
def test_two_vertex_equilibrium(core, model, a):
    """Two connected vertices that also repel balance at d* = (R K^3)^(1/(a+1))."""
    K, R = 1.3, 0.7
    dstar = (R * K ** 3) ** (1.0 / (a + 1))
    g = synth.from_edge_list(2, [(0, 1)])
    xy = np.array([[0.0, 0.0], [dstar, 0.0]], dtype=np.float32)
    L = core.Layout(core.Graph(g), xy=xy, K=K, R=R, repulse_neighbors=True, model=model)
    f = L.debug_forces("exact").astype(np.float64)
    ref, mag = oracle.forces(g, xy.astype(np.float64), K=K, R=R, a=a, repulse_neighbors=True)
    assert force_error(f, ref, mag).max() <= TOL_FORCE_EXACT
    assert np.abs(f).max() <= 1e-5 * mag.max()


def test_invalid_model_is_rejected(core):
    import ctypes
    lib = core.load()
    G = core.Graph(synth.path_graph(4))
    prm = core.ForceParams(1.0, 1.0, 0, -1, 4)
    h = ctypes.c_void_p()
    assert lib.bl_layout_init(G.handle, None, 0, 0, ctypes.byref(prm), ctypes.byref(h)) == core.BL_EINVAL
