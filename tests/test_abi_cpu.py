"""Host-side checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point that include/batchlayout.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "batchlayout.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(bl_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2002_08233_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("bl_graph_load_csr", "bl_layout_init", "bl_layout_run", "bl_positions",
                     "bl_layout_batch", "bl_serve_submit", "bl_serve_poll"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_calls_need_no_gpu(lib):
    lib.bl_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.bl_version()
    lib.bl_last_error.restype = ctypes.c_char_p
    # argument validation happens before any CUDA call
    lib.bl_graph_load_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
    out = ctypes.c_void_p()
    rp = (ctypes.c_int32 * 3)(0, 1, 1)
    ci = (ctypes.c_int32 * 1)(5)          # column id out of range
    assert lib.bl_graph_load_csr(2, 1, rp, ci, 0, ctypes.byref(out)) == 1
    assert b"out of range" in lib.bl_last_error()
    rp2 = (ctypes.c_int32 * 3)(0, 1, 1)
    ci2 = (ctypes.c_int32 * 1)(1)         # 0->1 without 1->0: not symmetric
    assert lib.bl_graph_load_csr(2, 1, rp2, ci2, 0, ctypes.byref(out)) == 1
    assert b"symmetric" in lib.bl_last_error()
    assert lib.bl_graph_load_csr(0, 0, rp2, ci2, 0, ctypes.byref(out)) == 1


def test_binding_refuses_to_run_without_gpu():
    import torch
    from paper_2002_08233_gb300 import core
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(RuntimeError):
        core.load(require_gpu=True)
