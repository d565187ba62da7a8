"""Convergence mode (Section 4.5: run until the energy difference between
successive iterations is small, read relatively): bl_layout_run_until stops at
the same iteration, with the same positions and energies, as running one
iteration at a time and applying the rule by hand."""
import numpy as np
import pytest

from paper_2002_08233_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def _by_hand(core, G, seed, max_iters, bs, mode, tol):
    L = core.Layout(G, seed=seed)
    hist = []
    prev = None
    for it in range(max_iters):
        L.run(1, bs, mode)
        e = float(L.energy_history()[0])
        hist.append(e)
        if prev is not None and abs(e - prev) <= tol * max(prev, 1.0):
            return L, hist, True
        prev = e
    return L, hist, False


@pytest.mark.parametrize("mode,maker,tol", [
    ("exact", lambda: synth.erdos_renyi(300, 5.0, 2), 3e-3),
    ("exact", lambda: synth.grid2d(12, 12), 1e-3),
    ("bh", lambda: synth.erdos_renyi(2000, 5.0, 4), 3e-3),
])
def test_stops_where_the_rule_first_holds(core, mode, maker, tol):
    g = maker()
    G = core.Graph(g)
    ref, hist, conv = _by_hand(core, G, 5, 400, 64, mode, tol)
    L = core.Layout(G, seed=5)
    it, cv = L.run_until(400, 64, mode, tol=tol)
    assert cv == conv and it == len(hist)
    assert conv, "the tolerance should be reached within 400 iterations"
    assert np.array_equal(L.positions(), ref.positions())
    assert np.array_equal(L.energy_history(), np.array(hist))
    assert L.stats()["iterations"] == it


def test_hits_max_iters_without_converging(core):
    G = core.Graph(synth.erdos_renyi(300, 5.0, 2))
    L = core.Layout(G, seed=1)
    it, cv = L.run_until(40, 64, "exact", tol=0.0)
    assert (it, cv) == (40, False)
    assert len(L.energy_history()) == 40


def test_continues_from_the_previous_run(core):
    """The first iteration of the call compares with the last of the previous run."""
    G = core.Graph(synth.erdos_renyi(300, 5.0, 2))
    L = core.Layout(G, seed=1)
    L.run(10, 64, "exact")
    it, cv = L.run_until(100, 64, "exact", tol=1e9)
    assert (it, cv) == (1, True)
