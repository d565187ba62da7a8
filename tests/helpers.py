"""Shared helpers for the tests: tolerances and error measures (Section 2.2 forces).

Force error of vertex i: |f_gpu - f_oracle| / sum_j |t_ij|, the oracle's sum of
the magnitudes of the terms that make up f(i,c). Repulsion sums cancel, so this
measures the FP32 error against the size of what was summed.
"""
import json
import os

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


def log_parity(kind, **fields):
    """Appends one JSON line {kind, fields...} to the file named by BL_PARITY_LOG
    (nothing when it is unset): the errors, spreads and tolerances a parity test
    applied, so a reader can see how close a passing gate was."""
    path = os.environ.get("BL_PARITY_LOG")
    if not path:
        return
    rec = {"kind": kind}
    for k, v in fields.items():
        rec[k] = v.item() if hasattr(v, "item") and np.ndim(v) == 0 else v
    with open(path, "a") as fh:
        fh.write(json.dumps(rec, default=float) + "\n")


def assert_positions(label, x_gpu, x_ref, base_tol, sensitivity, factor=4.0, scale=1.0):
    """Positions parity with the tolerance of the one-ulp reading: error <=
    scale * max(base_tol, factor * S). The message and the parity log carry the
    error, S and the tolerance that was applied."""
    err = float(position_error(x_gpu, x_ref))
    tol = scale * position_tolerance(base_tol, sensitivity, factor)
    log_parity("positions", label=str(label), err=err, sensitivity=float(sensitivity),
               base_tol=base_tol, tol=tol)
    assert err <= tol, (f"{label}: position error {err:.3e} > tolerance {tol:.3e} (base {base_tol:.0e}, "
                        f"oracle one-ulp sensitivity S = {float(sensitivity):.3e})")
    return err


def assert_forces(label, f_gpu, f_ref, mag, tol):
    """Condition-aware force parity: max_i |f_gpu - f_oracle| / sum_j |t_ij| <= tol."""
    err = float(force_error(f_gpu, f_ref, mag).max()) if len(mag) else 0.0
    log_parity("forces", label=str(label), err=err, tol=tol)
    assert err <= tol, f"{label}: force error {err:.3e} > tolerance {tol:.0e}"
    return err
