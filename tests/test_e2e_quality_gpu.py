"""End-to-end layouts: the whole seeded run on the GPU against the FP64 oracle's
run from the same start, compared by what the paper measures (Section 3.7):
stress and neighbourhood preservation.

The iteration is chaotic on some families: moving the FP32 start positions by one
ulp changes the oracle's own final stress by up to ~15% on grids and trees
(different local minima), while on random graphs it stays within ~0.2%. Each run
is therefore held to max(2%, 2x the oracle's own one-ulp spread on that input),
which is the strict 2% wherever the run is well-conditioned; on the chaotic
families the ensemble over 16 seeds must show no systematic shift."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def core():
    from paper_2002_08233_gb300 import core as c
    c.load()
    c.use_torch()
    return c


def _q(g, xy):
    return oracle.stress(g, xy)[0], oracle.neighborhood_preservation(g, xy)[0]


def _oracle_with_spread(g, xy0, iters, bs, trials=3):
    """The oracle's layout and quality, and how far its quality moves when every
    start coordinate moves by one ulp."""
    xr, _ = oracle.run(g, xy0, iters=iters, batch=bs, nthreads=NCPU)
    s0, n0 = _q(g, xr)
    rng = np.random.default_rng(12345)
    ds = dn = 0.0
    for _ in range(trials):
        dirs = np.where(rng.random(xy0.shape) < 0.5, -np.inf, np.inf).astype(np.float32)
        xp, _ = oracle.run(g, np.nextafter(xy0, dirs), iters=iters, batch=bs, nthreads=NCPU)
        s, n_ = _q(g, xp)
        ds = max(ds, abs(s / s0 - 1))
        dn = max(dn, abs(n_ / n0 - 1) if n0 > 0 else 0.0)
    return xr, s0, n0, ds, dn


def _gpu_run(core, G, xy0, iters, bs, engine):
    L = core.Layout(G, xy=xy0)
    if engine == "whole_gpu":
        L.run(iters, bs, "exact")
    else:
        core.run_batch([L], iters, bs)
    return L


CASES = [
    # the 32x32 grid at its full schedule: 600 iterations, minibatch 128
    ("grid32", lambda: synth.grid_32x32(), 600, 128),
    ("er1500", lambda: synth.erdos_renyi(1500, 6.0, 3), 300, 256),
    ("tree1023", lambda: synth.binary_tree(1023, 5), 300, 64),
]


@pytest.mark.parametrize("name,maker,iters,bs", CASES)
@pytest.mark.parametrize("seed", [0, 1])
def test_whole_run_quality_matches_oracle(core, name, maker, iters, bs, seed):
    g = maker()
    xy0 = synth.uniform_positions(g.n, seed)
    xr, s_r, np_r, ds, dn = _oracle_with_spread(g, xy0, iters, bs)
    tol_s = max(0.02, 2 * ds)
    tol_np = max(0.02, 2 * dn)
    G = core.Graph(g)
    for engine in ("whole_gpu", "batched"):
        L = _gpu_run(core, G, xy0, iters, bs, engine)
        s_g, np_g = _q(g, L.positions())
        assert abs(s_g / s_r - 1) <= tol_s, (name, engine, s_g, s_r, ds)
        assert abs(np_g / np_r - 1) <= tol_np, (name, engine, np_g, np_r, dn)
        # the GPU's own quality kernels agree with the oracle's on the GPU layout
        q = L.quality()
        assert abs(q["stress"] - s_g) <= 1e-10 * q["stress_pairs"]
        assert q["np"] == pytest.approx(np_g, rel=1e-12)


@pytest.mark.parametrize("name,maker,iters,bs", [CASES[0], CASES[2]])
def test_chaotic_families_show_no_systematic_shift(core, name, maker, iters, bs):
    """Over 16 seeds the GPU's stress relative to the oracle's averages out:
    |mean| <= max(2%, 3 standard errors)."""
    g = maker()
    G = core.Graph(g)
    d = []
    for seed in range(16):
        xy0 = synth.uniform_positions(g.n, 100 + seed)
        xr, _ = oracle.run(g, xy0, iters=iters, batch=bs, nthreads=NCPU)
        L = _gpu_run(core, G, xy0, iters, bs, "whole_gpu")
        d.append(_q(g, L.positions())[0] / _q(g, xr)[0] - 1)
    d = np.array(d)
    se = d.std(ddof=1) / np.sqrt(len(d))
    assert abs(d.mean()) <= max(0.02, 3 * se), (name, d.mean(), se, d)
