"""End-to-end layouts: the whole seeded run on the GPU against the FP64 oracle's
run from the same start, compared by what the paper measures (Section 3.7):
stress and neighbourhood preservation.

Every exact-mode engine is run on the inputs it serves: the one-cluster engine
(the default up to 3,072 vertices), the whole-GPU engine (`exact_grid_kernel`,
the default above that and forced below it with BL_EXACT_ENGINE=grid) and the
batched kernel; Barnes-Hut runs (Algorithm S5, theta = 1.2) are checked against
the oracle's Barnes-Hut run.

The iteration is chaotic on some families: moving the FP32 start positions by one
ulp changes the oracle's own final stress by up to ~15% on grids and trees
(different local minima), while on random graphs it stays within ~0.2%. Each run
is therefore held to max(2%, 2x the oracle's own one-ulp spread on that input),
which is the strict 2% wherever the run is well-conditioned; on the chaotic
families the ensemble over 16 seeds must show no systematic shift. NP is a mean of
Jaccard ratios of small neighbour counts: on random graphs (NP ~ 0.002) the
whole layout has under a hundred hits, so NP also gets the floor of two standard
errors of that count, 2/sqrt(hits). Every assert
message carries the error, the spread and the tolerance applied; with
BL_PARITY_LOG set they are also appended to that file as JSON lines."""
import os

import numpy as np
import pytest

import oracle
from paper_2002_08233_gb300 import synth
from helpers import log_parity

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


def _oracle_with_spread(g, xy0, iters, bs, mode=oracle.EXACT, trials=5):
    """The oracle's layout and quality, how far its quality moves when every start
    coordinate moves by one ulp, and its NP hit count (intersections summed over
    the queries)."""
    kw = dict(iters=iters, batch=bs, mode=mode, theta=1.2, nthreads=NCPU)
    xr, _ = oracle.run(g, xy0, **kw)
    s0 = oracle.stress(g, xr)[0]
    n0, _, hits = oracle.neighborhood_preservation(g, xr)
    rng = np.random.default_rng(12345)
    ds = dn = 0.0
    for _ in range(trials):
        dirs = np.where(rng.random(xy0.shape) < 0.5, -np.inf, np.inf).astype(np.float32)
        xp, _ = oracle.run(g, np.nextafter(xy0, dirs), **kw)
        s, n_ = _q(g, xp)
        ds = max(ds, abs(s / s0 - 1))
        dn = max(dn, abs(n_ / n0 - 1) if n0 > 0 else 0.0)
    return xr, s0, n0, ds, dn, hits


def _gpu_run(core, G, xy0, iters, bs, engine):
    """engine: "cluster" / "grid" force that exact engine, "default" lets the
    library choose, "batched" runs the persistent batched kernel, "bh" runs
    Barnes-Hut at theta 1.2."""
    L = core.Layout(G, xy=xy0)
    if engine == "batched":
        core.run_batch([L], iters, bs)
    elif engine == "bh":
        L.run(iters, bs, "bh", 1.2)
    elif engine in ("cluster", "grid"):
        os.environ["BL_EXACT_ENGINE"] = engine
        try:
            L.run(iters, bs, "exact")
        finally:
            os.environ.pop("BL_EXACT_ENGINE", None)
    else:
        L.run(iters, bs, "exact")
    return L


# (name, graph, iterations, minibatch, engines, seeds)
CASES = [
    # the 32x32 grid at its full schedule: 600 iterations, minibatch 128
    ("grid32", lambda: synth.grid_32x32(), 600, 128, ("cluster", "grid", "batched"), (0, 1)),
    ("er1500", lambda: synth.erdos_renyi(1500, 6.0, 3), 300, 256, ("cluster", "grid", "batched"), (0, 1)),
    ("tree1023", lambda: synth.binary_tree(1023, 5), 300, 64, ("cluster", "grid", "batched"), (0, 1)),
    # above the cluster engine's default size: the whole-GPU engine is the default
    ("er5000", lambda: synth.erdos_renyi(5000, 6.0, 3), 300, 256, ("default", "cluster"), (0,)),
    # Barnes-Hut (Algorithm S5) against the oracle's Barnes-Hut run
    ("er5000_bh", lambda: synth.erdos_renyi(5000, 6.0, 3), 300, 256, ("bh",), (0,)),
    ("rmat13_bh", lambda: synth.rmat(13, 8, seed=13), 250, 256, ("bh",), (0,)),
]


def _params():
    for name, maker, iters, bs, engines, seeds in CASES:
        for seed in seeds:
            yield pytest.param(name, maker, iters, bs, engines, seed, id=f"{name}-seed{seed}")


@pytest.mark.parametrize("name,maker,iters,bs,engines,seed", list(_params()))
def test_whole_run_quality_matches_oracle(core, name, maker, iters, bs, engines, seed):
    g = maker()
    xy0 = synth.uniform_positions(g.n, seed)
    mode = oracle.BH if engines == ("bh",) else oracle.EXACT
    xr, s_r, np_r, ds, dn, hits = _oracle_with_spread(g, xy0, iters, bs, mode)
    tol_s = max(0.02, 2 * ds)
    tol_np = max(0.02, 2 * dn, 2 / np.sqrt(max(hits, 1)))
    G = core.Graph(g)
    for engine in engines:
        L = _gpu_run(core, G, xy0, iters, bs, engine)
        s_g, np_g = _q(g, L.positions())
        es, en = abs(s_g / s_r - 1), abs(np_g / np_r - 1)
        info = dict(case=name, seed=seed, engine=engine, n=g.n, iters=iters, batch=bs,
                    stress_gpu=s_g, stress_oracle=s_r, stress_err=es, stress_spread=ds,
                    stress_tol=tol_s, np_gpu=np_g, np_oracle=np_r, np_err=en, np_spread=dn,
                    np_hits=hits, np_tol=tol_np)
        log_parity("e2e_quality", **info)
        assert es <= tol_s, info
        assert en <= tol_np, info
        # the GPU's own quality kernels agree with the oracle's on the GPU layout
        q = L.quality()
        assert abs(q["stress"] - s_g) <= 1e-10 * q["stress_pairs"], (name, engine, q["stress"], s_g)
        assert q["np"] == pytest.approx(np_g, rel=1e-12)


@pytest.mark.parametrize("name,maker,iters,bs", [(c[0], c[1], c[2], c[3]) for c in (CASES[0], CASES[2])])
@pytest.mark.parametrize("engine", ["grid", "cluster"])
def test_chaotic_families_show_no_systematic_shift(core, name, maker, iters, bs, engine):
    """Over 16 seeds the GPU's stress relative to the oracle's averages out:
    |mean| <= max(2%, 3 standard errors)."""
    g = maker()
    G = core.Graph(g)
    d = []
    for seed in range(16):
        xy0 = synth.uniform_positions(g.n, 100 + seed)
        xr, _ = oracle.run(g, xy0, iters=iters, batch=bs, nthreads=NCPU)
        L = _gpu_run(core, G, xy0, iters, bs, engine)
        d.append(_q(g, L.positions())[0] / _q(g, xr)[0] - 1)
    d = np.array(d)
    se = d.std(ddof=1) / np.sqrt(len(d))
    info = dict(case=name, engine=engine, mean=float(d.mean()), std_err=float(se),
                tol=max(0.02, 3 * se), per_seed=[float(v) for v in d])
    log_parity("e2e_ensemble", **info)
    assert abs(d.mean()) <= max(0.02, 3 * se), info
