"""The C ABI library loads without a GPU and exports every entry point include/qfs.h declares (no compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qfs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const\s+char\s*\*|void)\s*\*?\s*(qfs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libqfs():
    from paper_2502_12428_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("qfs_heights", "qfs_heights_multi", "qfs_plan_prepare", "qfs_strerror", "qfs_debug_stages"):
        assert must in names


def test_library_exports_every_declared_symbol(libqfs):
    missing = [n for n in declared_functions() if not hasattr(libqfs, n)]
    assert not missing, missing


def test_strerror_without_gpu(libqfs):
    libqfs.qfs_strerror.restype = ctypes.c_char_p
    libqfs.qfs_strerror.argtypes = [ctypes.c_int]
    assert libqfs.qfs_strerror(0) == b"ok"
    assert b"p must be" in libqfs.qfs_strerror(1)


def test_host_side_argument_checks_without_gpu(libqfs):
    # errors that the host can see are returned before any CUDA call, so they work on a machine without a GPU
    f = libqfs.qfs_heights
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(4, 10, 1, 10, 1, None) == 1          # invalid p
    assert f(5, 10, 1, 11, 1, None) == 2          # invalid max_h
    assert f(5, 10, 1, 0, 1, None) == 2
    assert f(5, -1, 1, 10, 1, None) == 3          # invalid n
    assert f(5, 10, None, 10, 1, None) == 4       # null coefficient pointer
    assert f(5, 0, None, 10, None, None) == 0     # n = 0 is a no-op


def test_binding_fails_loudly_without_cuda():
    import torch
    import paper_2502_12428_gb300.qfs as qfs
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(TypeError):
        qfs.heights(5, torch.zeros(3, 35, dtype=torch.uint8))
