"""Quick versions of the oracle pins, callable on any oracle build (used to show that planted mistakes are caught).

Each check returns True when the build agrees with what the paper and the mathematics fix.  Run as a script with a
library path, it prints a JSON object {check: bool} (the mutation test runs every planted mistake in a child
process, so a mistake that crashes cannot take the test run down).
"""
import json
import os
import sys
from math import comb

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
from helpers import affine_zero_count, example_quartics, mono_index, monomials, n_monomials, read_tuples  # noqa: E402
from paper_2502_12428_gb300 import inputs  # noqa: E402


def check_fermat(o):
    ok = all(o.height_a(p, inputs.fermat()) == (1 if p % 4 == 1 else 0) for p in (3, 5, 7))
    return ok and all(o.height_r(p, inputs.fermat()) == (1 if p % 4 == 1 else 0) for p in (3, 5, 7, 11))


def check_examples(o):
    rows = example_quartics()
    ok = all(o.height_a(p, f) == h for p, h, c, f in rows if p == 5)
    return ok and all(o.height_r(p, f) == h for p, h, c, f in rows if p in (5, 7))


def check_chevalley_warning(o):
    for p, seed in ((3, 11), (5, 12)):
        idx = mono_index(4 * (p - 1))[(p - 1,) * 4]
        for row in inputs.dense(p, 8, seed):
            g = o.stage_arrays_a(p, row, max_h=1)["g"]
            if g[idx] % p != (-affine_zero_count(row, p)) % p:
                return False
    return True


def check_delta1_binomial(o):
    rng = np.random.default_rng(3)
    mons = monomials(4)
    for p in (3, 5):
        for _ in range(4):
            i, j = rng.choice(35, 2, replace=False)
            a, b = int(rng.integers(1, p)), int(rng.integers(1, p))
            g = np.zeros(35, np.int64)
            g[i], g[j] = a, b
            try:
                _, delta = o.delta1(p, g, 4)
            except ArithmeticError:
                return False
            expect = np.zeros(n_monomials(4 * p), np.int64)
            idx = mono_index(4 * p)
            for k in range(1, p):
                e = tuple(k * x + (p - k) * y for x, y in zip(mons[i], mons[j]))
                expect[idx[e]] += (comb(p, k) // p) * a ** k * b ** (p - k)
            if not np.array_equal(delta, expect % p):
                return False
    return True


def check_routes_agree(o):
    for p, n in ((3, 30), (5, 10)):
        for row in np.concatenate([inputs.dense(p, n, 40 + p), inputs.sparse(p, n, 50 + p)]):
            a, r = o.stage_arrays_a(p, row), o.stage_arrays_r(p, row)
            if a["h"] != r["h"] or not np.array_equal(a["iters"], r["iters"]):
                return False
    return True


def check_split_u_example(o):
    p, d = 5, 16
    tuples, extra = read_tuples("wics_example.txt")
    delta = extra["delta"]
    deg = sum(delta) + d
    idx = mono_index(deg)
    P = np.zeros(n_monomials(deg), np.int64)
    for m in monomials(d):
        P[idx[tuple(x + y for x, y in zip(delta, m))]] = 1
    out_deg, U = o.split_u(p, P, deg)
    expect = np.zeros(U.size, np.int64)
    oidx = mono_index(out_deg)
    for m in tuples:
        expect[oidx[tuple((x + y - (p - 1)) // p for x, y in zip(delta, m))]] = 1
    return bool(np.array_equal(U, expect))


def check_max_h_bound(o):
    p, h, c, f = next(r for r in example_quartics() if r[0] == 5 and r[1] == 10)
    return o.height_a(p, f, max_h=10) == 10 and o.height_a(p, f, max_h=9) == 0


CHECKS = [check_fermat, check_examples, check_chevalley_warning, check_delta1_binomial, check_routes_agree,
          check_split_u_example, check_max_h_bound]


def run_all(o):
    out = {}
    for chk in CHECKS:
        try:
            out[chk.__name__] = bool(chk(o))
        except Exception:  # a planted mistake may also break an invariant loudly
            out[chk.__name__] = False
    return out


if __name__ == "__main__":
    o = oracle.Oracle(oracle.load(sys.argv[1]))
    print(json.dumps(run_all(o)))
