"""Shared helpers for the tests: tolerances and error measures (Section 2.2 forces).

Force error of vertex i: |f_gpu - f_oracle| / sum_j |t_ij|, the oracle's sum of
the magnitudes of the terms that make up f(i,c). Repulsion sums cancel, so this
measures the FP32 error against the size of what was summed.
"""
import numpy as np

TOL_FORCE_EXACT = 1e-5
TOL_FORCE_BH = 1e-4
TOL_POS_EXACT = 1e-5
TOL_POS_BH = 1e-4


def force_error(f_gpu, f_ref, mag):
    d = np.linalg.norm(np.asarray(f_gpu, np.float64) - f_ref, axis=1)
    return d / np.maximum(mag, 1e-300)


def position_error(x_gpu, x_ref):
    x_gpu = np.asarray(x_gpu, np.float64)
    scale = np.maximum(1.0, np.abs(x_ref))
    return np.max(np.abs(x_gpu - x_ref) / scale)


def oracle_sensitivity(g, xy, iters, batch, trials=3, seed=1, **kw):
    """How far the FP64 oracle's own result moves when every FP32 start
    coordinate moves by one ulp (random direction): the conditioning floor of a
    positions comparison. The normalised update c += Step*ct/|ct| amplifies
    force errors by |sum of terms|/|ct|, and close pairs make the sweep
    sensitive, so a path that stores positions in FP32 cannot be held below it."""
    import oracle
    xy = np.asarray(xy, np.float32)
    ref, _ = oracle.run(g, xy, iters, batch, **kw)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(trials):
        dirs = np.where(rng.random(xy.shape) < 0.5, -np.inf, np.inf).astype(np.float32)
        xp = np.nextafter(xy, dirs)
        out, _ = oracle.run(g, xp, iters, batch, **kw)
        worst = max(worst, position_error(out, ref))
    return ref, worst


def position_tolerance(base_tol, sensitivity, factor=4.0):
    return max(base_tol, factor * sensitivity)
