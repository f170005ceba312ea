"""Seeded synthetic quartics: the inputs every test and benchmark feeds to both the CUDA path and the oracle.

This module holds no arithmetic of the height method.  It only draws coefficients and changes variables.

A quartic is 35 coefficients in F_p, stored as uint8 in descending lexicographic order of the exponent tuple
(x1^4, x1^3 x2, x1^3 x3, x1^3 x4, x1^2 x2^2, ..., x4^4), the order in which the paper prints its examples
(Figures 4-7).  The paper's own workload is random quartics with coefficients uniform in F_p^35 (Sec. 7.1),
so these generators are that workload and not a stand-in for a dataset.

Randomness is counter based: value (row, slot) = splitmix64(seed XOR (64*row + slot)), with splitmix64 the
published mixer of Steele, Lea and Flood (2014): add 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds
(shifts 30, 27; multipliers 0xBF58476D1CE4E5B9, 0x94D049BB133111EB) and a final xor-shift by 31.
"""
import numpy as np

__all__ = ["splitmix64", "MONOMIALS", "monomial_index", "dense", "sparse", "fermat", "pgl4_matrices",
           "substitute", "config_seed", "CONFIG_SIZES"]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: exponent tuples of the 35 quartic monomials in descending lexicographic order
MONOMIALS = [(e1, e2, e3, 4 - e1 - e2 - e3)
             for e1 in range(4, -1, -1) for e2 in range(4 - e1, -1, -1) for e3 in range(4 - e1 - e2, -1, -1)]
monomial_index = {m: i for i, m in enumerate(MONOMIALS)}

#: workloads: (p, rows, kind) per group; seed of workload c is 0x5EED0000 + c
CONFIG_SIZES = {
    1: [(3, 64, "dense+fermat")],
    2: [(5, 65536, "dense")],
    3: [(5, 1048576, "sparse")],
    4: [(7, 262144, "dense")],
    5: [(5, 131072, "dense+pgl4"), (7, 131072, "dense+pgl4"), (11, 4096, "dense+pgl4")],
}


def config_seed(c):
    return 0x5EED0000 + c


def splitmix64(x):
    """splitmix64 output for counter value(s) x (numpy uint64, wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _draw(seed, rows, slot):
    ctr = (rows.astype(np.uint64) * np.uint64(64) + np.uint64(slot)) ^ np.uint64(seed)
    return splitmix64(ctr)


def dense(p, n, seed, row0=0):
    """n quartics with every coefficient uniform in F_p."""
    rows = np.arange(row0, row0 + n, dtype=np.uint64)
    out = np.empty((n, 35), np.uint8)
    for j in range(35):
        out[:, j] = (_draw(seed, rows, j) % np.uint64(p)).astype(np.uint8)
    return out


def sparse(p, n, seed, row0=0):
    """n quartics with k uniform in 4..12 nonzero terms; monomials by a partial Fisher-Yates shuffle of the 35
    positions, nonzero values uniform in 1..p-1."""
    rows = np.arange(row0, row0 + n, dtype=np.uint64)
    k = (4 + _draw(seed, rows, 0) % np.uint64(9)).astype(np.int64)
    perm = np.tile(np.arange(35, dtype=np.int64), (n, 1))
    ar = np.arange(n)
    for t in range(12):
        j = t + (_draw(seed, rows, 1 + t) % np.uint64(35 - t)).astype(np.int64)
        a, b = perm[ar, t].copy(), perm[ar, j].copy()
        perm[ar, t], perm[ar, j] = b, a
    out = np.zeros((n, 35), np.uint8)
    for t in range(12):
        val = (1 + _draw(seed, rows, 16 + t) % np.uint64(p - 1)).astype(np.uint8)
        sel = t < k
        out[ar[sel], perm[ar[sel], t]] = val[sel]
    return out


def fermat(extra_xyzw=0):
    """x1^4 + x2^4 + x3^4 + x4^4 (+ c * x1 x2 x3 x4)."""
    f = np.zeros(35, np.uint8)
    for m in [(4, 0, 0, 0), (0, 4, 0, 0), (0, 0, 4, 0), (0, 0, 0, 4)]:
        f[monomial_index[m]] = 1
    f[monomial_index[(1, 1, 1, 1)]] = extra_xyzw
    return f


def _det4_mod(A, p):
    """Determinants of a stack of 4x4 integer matrices, reduced mod p (exact int64 cofactor expansion)."""
    A = A.astype(np.int64)

    def det3(M):
        return (M[:, 0, 0] * (M[:, 1, 1] * M[:, 2, 2] - M[:, 1, 2] * M[:, 2, 1])
                - M[:, 0, 1] * (M[:, 1, 0] * M[:, 2, 2] - M[:, 1, 2] * M[:, 2, 0])
                + M[:, 0, 2] * (M[:, 1, 0] * M[:, 2, 1] - M[:, 1, 1] * M[:, 2, 0]))
    d = np.zeros(A.shape[0], np.int64)
    for c in range(4):
        minor = np.delete(np.delete(A, 0, axis=1), c, axis=2)
        d += (-1) ** c * A[:, 0, c] * det3(minor)
    return d % p


def pgl4_matrices(p, n, seed, row0=0):
    """One invertible 4x4 matrix over F_p per row, drawn entrywise until the determinant is nonzero mod p."""
    seed2 = int(splitmix64(np.uint64(seed ^ 0x504C4734)))
    rows = np.arange(row0, row0 + n, dtype=np.uint64)
    out = np.zeros((n, 4, 4), np.int64)
    todo = np.ones(n, bool)
    for attempt in range(64):
        idx = np.nonzero(todo)[0]
        if idx.size == 0:
            break
        cand = np.empty((idx.size, 4, 4), np.int64)
        for e in range(16):
            ctr = (rows[idx] * np.uint64(1024) + np.uint64(attempt * 16 + e)) ^ np.uint64(seed2)
            cand[:, e // 4, e % 4] = (splitmix64(ctr) % np.uint64(p)).astype(np.int64)
        ok = _det4_mod(cand, p) != 0
        out[idx[ok]] = cand[ok]
        todo[idx[ok]] = False
    if todo.any():
        raise RuntimeError("could not draw an invertible matrix")
    return out


def _forms(deg):
    return [(e1, e2, e3, deg - e1 - e2 - e3)
            for e1 in range(deg, -1, -1) for e2 in range(deg - e1, -1, -1) for e3 in range(deg - e1 - e2, -1, -1)]


def _mul_table(a, b):
    fa, fb, fc = _forms(a), _forms(b), _forms(a + b)
    ic = {m: i for i, m in enumerate(fc)}
    T = np.zeros((len(fa) * len(fb), len(fc)), np.int64)
    for i, x in enumerate(fa):
        for j, y in enumerate(fb):
            T[i * len(fb) + j, ic[tuple(u + v for u, v in zip(x, y))]] = 1
    return T


def _form_mul(X, a, Y, b, p, tables):
    key = (a, b)
    if key not in tables:
        tables[key] = _mul_table(a, b).astype(np.float64)
    n = X.shape[0]
    outer = (X[:, :, None] * Y[:, None, :]).reshape(n, -1).astype(np.float64)
    # entries are below p^2 and a product sums at most 35 of them: float64 (BLAS) is exact here
    return np.rint(outer @ tables[key]).astype(np.int64) % p


def _eval_points(p):
    """35 points of F_p^4 on which the quartic monomials are linearly independent mod p (p >= 5: a quartic has
    every partial degree below p, so it is determined by its values), with the inverse of their evaluation matrix."""
    rng = np.random.default_rng(1000 + p)
    while True:
        pts = rng.integers(0, p, (35, 4))
        V = np.array([[int(np.prod([int(x) ** e for x, e in zip(pt, m)])) % p for m in MONOMIALS] for pt in pts])
        inv = _inv_mod(V, p)
        if inv is not None:
            return pts, inv


def _inv_mod(V, p):
    n = V.shape[0]
    M = np.concatenate([V % p, np.eye(n, dtype=np.int64)], axis=1).astype(np.int64)
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r, c] % p), None)
        if piv is None:
            return None
        M[[c, piv]] = M[[piv, c]]
        M[c] = (M[c] * pow(int(M[c, c]), -1, p)) % p
        for r in range(n):
            if r != c and M[r, c]:
                M[r] = (M[r] - M[r, c] * M[c]) % p
    return M[:, n:]


_POINTS = {}


def substitute(coeffs, A, p):
    """f(A x) for each row: x_j -> sum_k A[j,k] x_k, expanded and reduced mod p.  Returns uint8 (n, 35)."""
    if p >= 5:
        # evaluate f at A x_m for 35 fixed points x_m and interpolate: h = V^-1 (f(A x_m))_m mod p
        if p not in _POINTS:
            _POINTS[p] = _eval_points(p)
        pts, inv = _POINTS[p]
        coeffs = np.asarray(coeffs, dtype=np.float64).reshape(-1, 35)
        A = np.asarray(A, dtype=np.int64)
        E = np.array(MONOMIALS)                                   # (35, 4) exponents
        out = np.empty((coeffs.shape[0], 35), np.uint8)
        for r0 in range(0, coeffs.shape[0], 8192):
            Y = (np.einsum("njk,mk->nmj", A[r0:r0 + 8192], pts) % p).astype(np.float64)   # (c, 35 points, 4)
            Yt = np.moveaxis(Y, -1, 0).reshape(4, -1)                                       # (4, c*35)
            pw = np.stack([np.ones_like(Yt), Yt, Yt ** 2, Yt ** 3, Yt ** 4], axis=1)        # (4, 5, c*35)
            # M[I, c*35] = prod_j Y_j^(I_j): entries below p^4, sums below 35 p^5 -- exact in float64
            M = pw[0, E[:, 0]] * pw[1, E[:, 1]] * pw[2, E[:, 2]] * pw[3, E[:, 3]]
            M = M.reshape(35, Y.shape[0], 35)                                              # (I, c, point)
            vals = np.einsum("icm,ci->cm", M, coeffs[r0:r0 + 8192]) % p
            out[r0:r0 + 8192] = ((vals @ inv.T.astype(np.float64)) % p).astype(np.uint8)
        return out
    return _substitute_expand(coeffs, A, p)


def _substitute_expand(coeffs, A, p):
    """f(A x) by expanding the products of the four linear forms (any p)."""
    coeffs = np.asarray(coeffs, dtype=np.int64).reshape(-1, 35)
    n = coeffs.shape[0]
    tables = {}
    # powers of the four linear forms L_j = sum_k A[j,k] x_k, as forms of degree 0..4
    pw = []
    for j in range(4):
        L = A[:, j, :].astype(np.int64) % p          # degree-1 form, order (x1, x2, x3, x4) = descending lex
        powers = [np.ones((n, 1), np.int64), L]
        for e in range(2, 5):
            powers.append(_form_mul(powers[-1], e - 1, L, 1, p, tables))
        pw.append(powers)
    out = np.zeros((n, 35), np.int64)
    for idx, I in enumerate(MONOMIALS):
        T, deg = np.ones((n, 1), np.int64), 0
        for j in range(4):
            if I[j]:
                T = _form_mul(T, deg, pw[j][I[j]], I[j], p, tables)
                deg += I[j]
        out = (out + coeffs[:, idx:idx + 1] * T) % p
    return out.astype(np.uint8)
