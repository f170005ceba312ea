"""ctypes front end of the plain C oracle (test infrastructure only).

The C sources beside this file implement the paper's Algorithms 1-3 literally (``route_a.c``) and an
independently derived reduced form of the same iteration (``route_r.c``).  ``build()`` compiles them with
gcc into ``oracle/_build/liboracle.so``; nothing here touches a GPU.

Array conventions: every polynomial array is a coefficient list in descending lexicographic order of the
exponent tuple (x1 exponent descending, then x2, then x3), the order in which the paper prints quartics.
"""
import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["hpoly.c", "route_a.c", "route_r.c", "batch.c"]
_lib = None

__all__ = ["build", "lib", "load", "Oracle", "monomial_count", "height_a", "height_r", "heights", "delta1", "split_u",
           "stage_arrays_a", "stage_arrays_r", "stage_arrays_fchain", "theta_matrix", "matmul_mod", "poly_power",
           "form_monomials", "ROUTE_A", "ROUTE_R"]

ROUTE_A = 0
ROUTE_R = 1


def build(force=False, defines=(), path=None):
    """Compile the oracle with gcc (portable C11, no architecture flags) and return the library path.

    `defines` (e.g. ["QFS_MUTATE=3"]) and `path` build a variant elsewhere; tests use that to plant mistakes."""
    os.makedirs(_BUILD, exist_ok=True)
    out = path or _LIB_PATH
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "hpoly.h")])
    if force or defines or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".tmp{os.getpid()}"
        cmd = (["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared", "-o", tmp] + [f"-D{d}" for d in defines]
               + srcs + ["-lpthread"])
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path):
    """ctypes handle of an oracle library build (argument types set)."""
    if True:
        L = ctypes.CDLL(path)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        L.qfs_oracle_height_a.argtypes = [ctypes.c_int, u8p, ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p]
        L.qfs_oracle_height_a.restype = ctypes.c_int
        L.qfs_oracle_height_r.argtypes = [ctypes.c_int, u8p, ctypes.c_int, i32p, i32p]
        L.qfs_oracle_height_r.restype = ctypes.c_int
        L.qfs_oracle_heights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, u8p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
        L.qfs_oracle_heights.restype = ctypes.c_int
        L.qfs_oracle_delta1.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, i32p, i32p]
        L.qfs_oracle_delta1.restype = ctypes.c_int
        L.qfs_oracle_split_u.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p]
        L.qfs_oracle_split_u.restype = ctypes.c_int
        L.qfs_oracle_stages_fchain.argtypes = [ctypes.c_int, u8p, i32p, i32p, i32p]
        L.qfs_oracle_stages_fchain.restype = ctypes.c_int
    return L


class Oracle:
    """The oracle's Python API bound to one library build (the module functions use the default build)."""

    def __init__(self, L):
        self._L = L

    def __getattr__(self, name):
        fn = globals()[name]

        def bound(*a, **k):
            global _lib
            saved = _lib
            _lib = self._L
            try:
                return fn(*a, **k)
            finally:
                _lib = saved
        return bound


def monomial_count(d):
    """Number of degree-d monomials in four variables, C(d+3, 3)."""
    return comb(d + 3, 3) if d >= 0 else 0


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _quartic(f):
    f = np.ascontiguousarray(np.asarray(f, dtype=np.uint8).reshape(35))
    return f


def height_a(p, f, max_h=10, lift_signed=False):
    """Route A (literal Algorithms 1-3) height of one quartic given as 35 coefficients."""
    f = _quartic(f)
    return lib().qfs_oracle_height_a(p, _ptr(f, ctypes.c_uint8), max_h, int(lift_signed), None, None, None, None)


def height_r(p, f, max_h=10):
    """Route R (reduced derivation) height of one quartic."""
    f = _quartic(f)
    return lib().qfs_oracle_height_r(p, _ptr(f, ctypes.c_uint8), max_h, None, None)


def stage_arrays_a(p, f, max_h=10, lift_signed=False):
    """Route A with every intermediate array: returns dict(h, g, D, delta, iters).

    g = f^(p-1) mod p; D = lift(g)^p mod p^2; delta = Delta_1(g) mod p; iters[h-2] = g_h.
    D and delta are None when the height-1 test succeeds; iters holds the rows that were computed.
    """
    f = _quartic(f)
    ld = monomial_count(4 * (p - 1))
    lD = monomial_count(4 * p * (p - 1))
    g = np.zeros(ld, np.int32)
    D = np.zeros(lD, np.int32)
    delta = np.zeros(lD, np.int32)
    iters = np.zeros((max(max_h - 1, 1), ld), np.int32)
    h = lib().qfs_oracle_height_a(p, _ptr(f, ctypes.c_uint8), max_h, int(lift_signed), _ptr(g, ctypes.c_int32),
                                  _ptr(D, ctypes.c_int32), _ptr(delta, ctypes.c_int32), _ptr(iters, ctypes.c_int32))
    out = dict(h=h, g=g, D=None, delta=None, iters=iters[:0])
    if h != 1 and h >= 0:
        out["D"], out["delta"] = D, delta
        n_rows = (h - 1) if h >= 2 else _rows_until_zero_or_end(iters, p, max_h)
        out["iters"] = iters[:n_rows]
    return out


def stage_arrays_fchain(p, f):
    """g = f^(p-1) mod p and, past the height-1 test, D = lift(f)^(p(p-1)) mod p^2 (the same array as route A's
    lift(g)^p, formed by products with f's 35 terms) and Delta_1(g) by Algorithm 1's subtraction and division.
    Returns dict(h1, g, D, delta): h1 = True if the height is 1 (then D and delta are None)."""
    f = _quartic(f)
    ld = monomial_count(4 * (p - 1))
    lD = monomial_count(4 * p * (p - 1))
    g = np.zeros(ld, np.int32)
    D = np.zeros(lD, np.int32)
    delta = np.zeros(lD, np.int32)
    rc = lib().qfs_oracle_stages_fchain(p, _ptr(f, ctypes.c_uint8), _ptr(g, ctypes.c_int32), _ptr(D, ctypes.c_int32),
                                        _ptr(delta, ctypes.c_int32))
    if rc == -2:
        raise ArithmeticError("division by p in Algorithm 1 is not exact")
    if rc < 0:
        raise ValueError(f"oracle failure {rc}")
    return dict(h1=rc == 1, g=g, D=None if rc == 1 else D, delta=None if rc == 1 else delta)


def stage_arrays_r(p, f, max_h=10):
    """Route R with Delta_1(f) and the iterates: returns dict(h, d1f, iters)."""
    f = _quartic(f)
    ld = monomial_count(4 * (p - 1))
    l4p = monomial_count(4 * p)
    d1f = np.zeros(l4p, np.int32)
    iters = np.zeros((max(max_h - 1, 1), ld), np.int32)
    h = lib().qfs_oracle_height_r(p, _ptr(f, ctypes.c_uint8), max_h, _ptr(d1f, ctypes.c_int32),
                                  _ptr(iters, ctypes.c_int32))
    out = dict(h=h, d1f=None, iters=iters[:0])
    if h != 1 and h >= 0:
        out["d1f"] = d1f
        n_rows = (h - 1) if h >= 2 else _rows_until_zero_or_end(iters, p, max_h)
        out["iters"] = iters[:n_rows]
    return out


def _rows_until_zero_or_end(iters, p, max_h):
    # height 0: the loop ran until an iterate vanished or until max_h
    for r in range(max_h - 1):
        if not iters[r].any():
            return r + 1
    return max_h - 1


def heights(p, coeffs, max_h=10, route=ROUTE_R, threads=None):
    """Heights of n quartics (uint8 array n x 35) on a pthread pool; returns int8 array of codes."""
    coeffs = np.ascontiguousarray(np.asarray(coeffs, dtype=np.uint8).reshape(-1, 35))
    n = coeffs.shape[0]
    out = np.zeros(n, np.int8)
    if threads is None:
        threads = os.cpu_count() or 1
    lib().qfs_oracle_heights(route, p, n, _ptr(coeffs, ctypes.c_uint8), max_h, _ptr(out, ctypes.c_int8), threads)
    return out


def delta1(p, g, deg, lift_signed=False):
    """Algorithm 1 on an arbitrary form g of degree deg (coefficients mod p, descending lex).

    Returns (D, delta): D = lift(g)^p mod p^2 and Delta_1(g) mod p, both of degree p*deg.
    Raises ArithmeticError if the division by p is not exact.
    """
    g = np.ascontiguousarray(np.asarray(g, dtype=np.int32).reshape(monomial_count(deg)))
    n = monomial_count(p * deg)
    D = np.zeros(n, np.int32)
    delta = np.zeros(n, np.int32)
    rc = lib().qfs_oracle_delta1(p, deg, _ptr(g, ctypes.c_int32), int(lift_signed), _ptr(D, ctypes.c_int32),
                                 _ptr(delta, ctypes.c_int32))
    if rc == -2:
        raise ArithmeticError("division by p in Algorithm 1 is not exact")
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return D, delta


def split_u(p, P, deg):
    """Algorithm 2 on a form P of degree deg.  Returns (out_degree, coefficients) or (None, None)."""
    rem = deg - 4 * (p - 1)
    if rem < 0 or rem % p:
        return None, None
    P = np.ascontiguousarray(np.asarray(P, dtype=np.int32).reshape(monomial_count(deg)))
    out = np.zeros(monomial_count(rem // p), np.int32)
    d = lib().qfs_oracle_split_u(p, deg, _ptr(P, ctypes.c_int32), _ptr(out, ctypes.c_int32))
    return d, out


def theta_matrix(p, f):
    """The theta matrix of quartic f (Sec. 3.4, the matrix form of Algorithm 3's step), by its definition:
    M[r][c] = Delta[p r + (p-1)1 - c] for r, c in B_d (descending lex), Delta = Delta_1(g) mod p with g = f^(p-1)
    mod p (Algorithm 1 via delta1), and 0 where the exponent leaves the degree-4p(p-1) monomials.  Returns a uint8
    array (ld, ld).  theta(g) = M g mod p; the pins check that against route A's iterates."""
    f = _quartic(f)
    d, D = 4 * (p - 1), 4 * p * (p - 1)
    ld = monomial_count(d)
    g = np.zeros(ld, np.int32)
    D_ = np.zeros(monomial_count(D), np.int32)
    delta = np.zeros(monomial_count(D), np.int32)
    iters = np.zeros((1, ld), np.int32)
    lib().qfs_oracle_height_a(p, _ptr(f, ctypes.c_uint8), 1, 0, _ptr(g, ctypes.c_int32), _ptr(D_, ctypes.c_int32),
                              _ptr(delta, ctypes.c_int32), _ptr(iters, ctypes.c_int32))
    _, delta = delta1(p, g, d)
    # exponent vectors (x1..x4) of B_d and of the degree-D monomials, descending lex
    def monomials(deg):
        out = []
        for a in range(deg, -1, -1):
            for b in range(deg - a, -1, -1):
                for c in range(deg - a - b, -1, -1):
                    out.append((a, b, c, deg - a - b - c))
        return np.array(out, dtype=np.int64)
    B = monomials(d)
    index = {tuple(e): i for i, e in enumerate(monomials(D))}
    M = np.zeros((ld, ld), np.uint8)
    for r in range(ld):
        e = p * B[r][None, :] + (p - 1) - B       # exponent of Delta paired with each column c
        for c in np.nonzero((e >= 0).all(axis=1))[0]:
            M[r, c] = delta[index[tuple(e[c])]]
    return M


def matmul_mod(p, A, B):
    """C = A B mod p (Sec. 5): the integer matrix product (numpy, int64, exact for these sizes) reduced mod p."""
    A = np.asarray(A, dtype=np.int64)
    B = np.asarray(B, dtype=np.int64)
    return (A @ B % p).astype(np.uint8)


def form_monomials(deg):
    """Exponent tuples (x1, x2, x3, x4) of the degree-deg monomials in descending lex order."""
    return [(a, b, c, deg - a - b - c) for a in range(deg, -1, -1) for b in range(deg - a, -1, -1)
            for c in range(deg - a - b, -1, -1)]


def poly_power(d, coeffs, n):
    """f^n over the integers (Sec. 4's powering workload) by repeated multiplication with Python integers: the
    plain definition, for small cases.  coeffs in descending lex order; returns the coefficients of f^n likewise."""
    f = {e: int(c) for e, c in zip(form_monomials(d), coeffs) if int(c)}
    acc = {(0, 0, 0, 0): 1}
    for _ in range(n):
        nxt = {}
        for ea, ca in acc.items():
            for eb, cb in f.items():
                k = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2], ea[3] + eb[3])
                nxt[k] = nxt.get(k, 0) + ca * cb
        acc = nxt
    return [acc.get(e, 0) for e in form_monomials(d * n)]
