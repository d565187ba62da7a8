"""The exact engine's FMA-pipe reciprocal (Newton-Raphson from the 48/17 - 32/17 D
estimate, three steps) against 1/x in FP64: within 2 ulp of FP32 over the range
the engine feeds it (squared distances from 1e-30 to 1e37), and 0 from 2^126 on."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rcp_nr_error_bound():
    from paper_2002_08233_gb300 import core
    lib = core.load()
    core.use_torch()
    rng = np.random.default_rng(3)
    x = np.concatenate([
        10.0 ** rng.uniform(-30, 37, 200000),
        rng.uniform(0.5, 1.0, 20000), rng.uniform(1.0, 2.0, 20000),
        2.0 ** np.arange(-99, 126), np.nextafter(2.0 ** np.arange(-99, 126), 0),
        [1e-30, 1.0, 3.0, 17.0, 0.75]]).astype(np.float32)
    y = np.empty_like(x)
    st = lib.bl_debug_rcp(ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data), x.size)
    assert st == 0, lib.bl_last_error()
    exact = 1.0 / x.astype(np.float64)
    rel = np.abs(y.astype(np.float64) - exact) / exact
    assert rel.max() <= 2 * 2.0 ** -24, (float(rel.max()), float(x[np.argmax(rel)]))
    big = np.array([2.0 ** 126, 3e38], dtype=np.float32)
    yb = np.empty_like(big)
    assert lib.bl_debug_rcp(ctypes.c_void_p(big.ctypes.data), ctypes.c_void_p(yb.ctypes.data), 2) == 0
    assert np.all(yb == 0.0)
