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


def test_poly_power_plan_without_gpu():
    # host-only plan of the powering: the prime count follows the exact bound (sum of coefficients)^n against the
    # product of the primes q = c 2^24 + 1 (largest first), the transform length is the power of two >= (d n + 1)^3,
    # and the byte count is the pass structure: per prime the tables, the cleared and filled input, 2k + 1 passes
    # reading and writing the buffer (k outer passes of at most 8 stages), the gather; then the remaindering
    import numpy as np
    import paper_2502_12428_gb300.qfs as qfs
    primes = [2130706433, 2113929217, 2013265921, 1811939329, 1711276033, 1224736769, 1107296257]
    rng = np.random.default_rng(16)
    f = rng.integers(0, 5, 969).astype(np.uint32)
    for n in (5, 10, 15):
        info = qfs.poly_power_info(16, f, n)
        bound, prod, need = int(f.sum()) ** n, 1, 0
        while prod <= bound:
            prod *= primes[need]
            need += 1
        assert info["nprimes"] == need
        B = 16 * n + 1
        N = 1 << (B ** 3 - 1).bit_length()
        assert info["transform_len"] == N
        logN = N.bit_length() - 1
        inner = min(8, logN)
        k = -(-(logN - inner) // 8)
        n_in, n_out = 969, (16 * n + 3) * (16 * n + 2) * (16 * n + 1) // 6
        R = min(256, N)
        tables = 2 * 4 * (min(N, 4096) + max(1, N >> 12) + R)
        # the input sits below index 16 B^2 + 1, so the first forward pass (columns of stride N >> kp0, kp0 =
        # min(8, logN - inner)) clears and reads only the rows that can hold it
        kp0 = min(8, logN - inner)
        stride = N >> kp0
        cleared = -(-(16 * B * B + 1) // stride) * stride
        passes = 4 * cleared + 4 * N + 2 * k * 8 * N
        per_prime = tables + 4 * cleared + 8 * n_in + passes + 8 * n_out
        assert info["hbm_bytes"] == need * per_prime + n_out * (4 * need + 32)
    with pytest.raises(RuntimeError):
        qfs.poly_power_info(16, f, 16)          # degree 256
    with pytest.raises(RuntimeError):
        qfs.poly_power_info(1, [2 ** 31] * 4, 8)  # (sum)^n beyond 256 bits


def test_sweep_tuning_argument_checks_without_gpu(libqfs):
    # the swept-chain shape is host state: set, read back and validated without any CUDA call
    st, gt = libqfs.qfs_sweep_tune_set, libqfs.qfs_sweep_tune_get
    st.argtypes = [ctypes.c_int] * 4
    gt.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    st.restype = gt.restype = ctypes.c_int
    dm, c = ctypes.c_int(-1), ctypes.c_int(-1)
    # the state is process-wide (the binding may have applied a tuned table already): save, reset, restore
    assert gt(1, 7, ctypes.byref(dm), ctypes.byref(c)) == 0
    saved = [(f, ) + tuple(v.value for v in (dm, c)) for f in (1,)]
    d0, c0 = ctypes.c_int(-1), ctypes.c_int(-1)
    assert gt(0, 7, ctypes.byref(d0), ctypes.byref(c0)) == 0
    saved.append((0, d0.value, c0.value))
    assert st(1, 7, 0, 0) == 0 and st(0, 7, 0, 0) == 0
    assert gt(1, 7, ctypes.byref(dm), ctypes.byref(c)) == 0 and (dm.value, c.value) == (12, 0)
    assert st(1, 7, 9, 1) == 0
    assert gt(1, 7, ctypes.byref(dm), ctypes.byref(c)) == 0 and (dm.value, c.value) == (9, 1)
    assert gt(0, 7, ctypes.byref(dm), ctypes.byref(c)) == 0 and (dm.value, c.value) == (12, 0)   # per form
    assert st(1, 7, 0, 0) == 0
    assert gt(1, 7, ctypes.byref(dm), ctypes.byref(c)) == 0 and (dm.value, c.value) == (12, 0)
    assert st(1, 4, 9, 1) == 1          # invalid p
    assert st(2, 7, 9, 1) == 7          # the tensor form has no swept chain
    assert st(1, 7, 17, 1) == 7 and st(1, 7, 9, 33) == 7
    for f, d, n in saved:
        assert st(f, 7, d, n) == 0

