"""Convergence mode (Section 4.5: run until the energy difference between
successive iterations is small, read relatively): bl_layout_run_until stops at
the same iteration, with the same positions and energies, as running one
iteration at a time and applying the rule by hand, and at the iteration where
the rule first holds on the FP64 oracle's own energy sequence."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import log_parity

NCPU = os.cpu_count() or 1

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


def _rule_stop(e, tol):
    """The stop rule on an energy sequence: the first iteration t (1-based) whose
    energy differs from the previous one by at most tol * max(E_prev, 1)."""
    for k in range(1, len(e)):
        if abs(e[k] - e[k - 1]) <= tol * max(e[k - 1], 1.0):
            return k + 1
    return None


def _grid_at_coordinates():
    """A 16x16 grid drawn at its grid coordinates, spacing 1.3: no close pairs, so
    the energy sequence is well-conditioned (a one-ulp change of the start moves
    the oracle's energies by ~1e-4 over the first 40 iterations, where a random
    start moves them by ~10% within 10)."""
    g = synth.grid2d(16, 16)
    r, c = np.divmod(np.arange(g.n), 16)
    return g, np.stack([c * 1.3, r * 1.3], axis=1).astype(np.float32)


@pytest.mark.parametrize("mode", ["exact", "bh"])
def test_stop_iteration_matches_oracle(core, mode):
    """The GPU stops inside the window of iterations where the rule first holds
    on the oracle's energies from the same start and from starts moved by one ulp
    (on this input all of them stop at the same iteration); the energies up to
    there agree within max(1e-4, 2x the oracle's own one-ulp spread)."""
    g, xy = _grid_at_coordinates()
    om = oracle.EXACT if mode == "exact" else oracle.BH
    tol, bs, cap = 2e-3, 64, 120
    _, e = oracle.run(g, xy, iters=cap, batch=bs, mode=om, theta=1.2, nthreads=NCPU)
    stops, others = [_rule_stop(e, tol)], []
    rng = np.random.default_rng(7)
    for _ in range(3):
        dirs = np.where(rng.random(xy.shape) < 0.5, -np.inf, np.inf).astype(np.float32)
        _, ep = oracle.run(g, np.nextafter(xy, dirs), iters=cap, batch=bs, mode=om, theta=1.2,
                           nthreads=NCPU)
        stops.append(_rule_stop(ep, tol))
        others.append(ep)
    assert None not in stops, stops
    L = core.Layout(core.Graph(g), xy=xy)
    it, cv = L.run_until(cap, bs, mode, tol=tol)
    eg = L.energy_history()
    spread = max(float(np.abs(ep[:it] / e[:it] - 1).max()) for ep in others)
    tol_e = max(1e-4, 2 * spread)
    err_e = float(np.abs(eg / e[:it] - 1).max())
    info = dict(mode=mode, gpu_stop=it, oracle_stops=stops, energy_err=err_e, energy_spread=spread,
                energy_tol=tol_e)
    log_parity("convergence", **info)
    assert cv and min(stops) <= it <= max(stops), info
    assert len(eg) == it and err_e <= tol_e, info
