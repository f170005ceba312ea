"""Test helpers: golden fixture readers and small independent utilities (no height arithmetic)."""
import os
import re
from math import comb

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def monomials(deg):
    """Exponent tuples of degree deg in descending lexicographic order."""
    return [(e1, e2, e3, deg - e1 - e2 - e3)
            for e1 in range(deg, -1, -1) for e2 in range(deg - e1, -1, -1) for e3 in range(deg - e1 - e2, -1, -1)]


def mono_index(deg):
    return {m: i for i, m in enumerate(monomials(deg))}


def n_monomials(deg):
    return comb(deg + 3, 3)


def parse_poly(text, p, deg=4):
    """'4 x1^4 + 2 x1^3 x2 + x4^4' -> coefficients mod p in descending lex order."""
    idx = mono_index(deg)
    f = np.zeros(len(idx), np.int64)
    for term in text.split("+"):
        toks = term.split()
        c = 1
        if toks and re.fullmatch(r"\d+", toks[0]):
            c, toks = int(toks[0]), toks[1:]
        e = [0, 0, 0, 0]
        for v in toks:
            m = re.fullmatch(r"x(\d)(?:\^(\d+))?", v)
            assert m, term
            e[int(m.group(1)) - 1] += int(m.group(2) or 1)
        f[idx[tuple(e)]] += c
    return (f % p).astype(np.uint8 if deg == 4 else np.int64)


def example_quartics():
    """Rows of Figures 4-7: list of (p, height, citation, coefficients uint8[35])."""
    rows = []
    with open(os.path.join(GOLDEN, "example_quartics.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p, h, cite, poly = [s.strip() for s in line.split("|")]
            rows.append((int(p), int(h), cite, parse_poly(poly, int(p))))
    return rows


def read_tuples(name):
    out, extra = [], {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            toks = line.split()
            if not re.fullmatch(r"-?\d+", toks[0]):
                extra[toks[0]] = tuple(int(t) for t in toks[1:])
            else:
                out.append(tuple(int(t) for t in toks))
    return out, extra


def affine_zero_count(f, p):
    """#{x in F_p^4 : f(x) = 0} by brute force (f = 35 coefficients, descending lex)."""
    xs = np.array(np.meshgrid(*[np.arange(p)] * 4, indexing="ij")).reshape(4, -1).astype(np.int64)
    val = np.zeros(xs.shape[1], np.int64)
    for c, e in zip(f, monomials(4)):
        if c:
            val = (val + int(c) * xs[0] ** e[0] * xs[1] ** e[1] * xs[2] ** e[2] * xs[3] ** e[3]) % p
    return int((val == 0).sum())
