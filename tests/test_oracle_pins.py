"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Every check here is independent of the oracle's own code path: printed examples from the paper, closed forms,
brute-force counts, invariants, and agreement of two independently derived routes.
"""
from math import comb

import numpy as np
import pytest

import oracle
from helpers import (affine_zero_count, example_quartics, mono_index, monomials, n_monomials, read_tuples)
from paper_2502_12428_gb300 import inputs


def fermat():
    return inputs.fermat()


# ---------------------------------------------------------------- sizes
def test_matrix_sizes_sec6():
    # Sec. 6 lists the sizes of the square matrix of "multiply then split" for p = 3, 5, 7, 11, 13
    for p, size in zip([3, 5, 7, 11, 13], [165, 969, 2925, 12341, 20825]):
        assert oracle.monomial_count(4 * (p - 1)) == size == comb(4 * p - 1, 3)


def test_stage_array_lengths():
    # degrees: f^(p-1) has degree 4(p-1), Delta_1(f^(p-1)) has degree 4p(p-1) (Sec. 3.4)
    f = inputs.dense(5, 1, 11)[0]
    for row in range(50):
        f = inputs.dense(5, 1, 11, row0=row)[0]
        st = oracle.stage_arrays_a(5, f)
        if st["h"] != 1:
            break
    assert st["h"] != 1
    assert st["g"].shape == (969,)
    assert st["delta"].shape == (91881,) and st["D"].shape == (91881,)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("p", [3, 5, 7])
def test_fermat_route_a(p):
    # Fermat quartic: height 1 iff p = 1 mod 4, otherwise infinity (Example of Sec. 3.3, Figure 4 row 1)
    assert oracle.height_a(p, fermat()) == (1 if p % 4 == 1 else 0)


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13, 17, 19])
def test_fermat_route_r(p):
    assert oracle.height_r(p, fermat()) == (1 if p % 4 == 1 else 0)


def test_fermat_p3_example():
    # Example of Sec. 3.3: g = f^2 over F_3 as printed, witness coefficient 0, and the first iterate vanishes
    st = oracle.stage_arrays_a(3, fermat())
    terms, _ = read_tuples("fermat_p3_g.txt")
    expect = np.zeros(165, np.int64)
    idx = mono_index(8)
    for c, *e in terms:
        expect[idx[tuple(e)]] = c
    assert np.array_equal(st["g"], expect)
    assert st["g"][idx[(2, 2, 2, 2)]] == 0
    assert st["h"] == 0
    assert st["iters"].shape[0] == 1 and not st["iters"][0].any()


# ---------------------------------------------------------------- printed examples (Figures 4-7)
ROWS = example_quartics()


def test_example_count():
    assert len(ROWS) == 32
    assert sorted({p for p, *_ in ROWS}) == [5, 7, 11, 13]


@pytest.mark.parametrize("row", ROWS, ids=[f"p{p}-{c.split(',')[1].strip()}" for p, h, c, f in ROWS])
def test_paper_examples_route_r(row):
    p, h, cite, f = row
    assert oracle.height_r(p, f) == h, cite


@pytest.mark.parametrize("row", [r for r in ROWS if r[0] == 5], ids=lambda r: r[2])
def test_paper_examples_route_a_p5(row):
    p, h, cite, f = row
    assert oracle.height_a(p, f) == h, cite


@pytest.mark.slow
@pytest.mark.parametrize("h_want", [2, 3])
def test_paper_examples_route_a_p7(h_want):
    p, h, cite, f = next(r for r in ROWS if r[0] == 7 and r[1] == h_want)
    assert oracle.height_a(p, f) == h, cite


def test_max_h_bound():
    # Algorithm 3 returns infinity once the bound b is passed: the height-10 example capped at 9 reads 0
    p, h, cite, f = next(r for r in ROWS if r[0] == 5 and r[1] == 10)
    assert oracle.height_r(p, f, max_h=9) == 0
    assert oracle.height_r(p, f, max_h=10) == 10
    assert oracle.height_a(p, f, max_h=9) == 0


def test_invalid_coefficient():
    f = inputs.dense(5, 1, 3)[0].copy()
    f[7] = 5
    assert oracle.height_a(5, f) == -1 and oracle.height_r(5, f) == -1


# ---------------------------------------------------------------- height-1 test (Fedder) vs brute force
@pytest.mark.parametrize("p,n", [(3, 40), (5, 25), (7, 8)])
def test_chevalley_warning(p, n):
    # Sum over F_p^4 of f^(p-1) is the coefficient of (x1..x4)^(p-1), so that coefficient = -#zeros (mod p)
    f = inputs.dense(p, n, 991 + p)
    idx = mono_index(4 * (p - 1))[(p - 1,) * 4]
    for row in f:
        g = oracle.stage_arrays_a(p, row, max_h=1)["g"]
        assert g[idx] % p == (-affine_zero_count(row, p)) % p


# ---------------------------------------------------------------- Algorithm 1
def _random_form(p, deg, seed, density=0.5):
    rng = np.random.default_rng(seed)
    g = rng.integers(0, p, n_monomials(deg))
    g[rng.random(g.size) > density] = 0
    return g


@pytest.mark.parametrize("p", [3, 5, 7])
def test_delta1_of_monomial_is_zero(p):
    g = np.zeros(n_monomials(4), np.int64)
    g[mono_index(4)[(1, 2, 0, 1)]] = 2
    D, delta = oracle.delta1(p, g, 4)
    assert not delta.any()


@pytest.mark.parametrize("p", [3, 5, 7])
def test_delta1_binomial_closed_form(p):
    # Delta_1(a x^I + b x^J) = sum_{k=1}^{p-1} (C(p,k)/p) a^k b^(p-k) x^(kI + (p-k)J)  (mod p)
    rng = np.random.default_rng(p)
    mons = monomials(4)
    for trial in range(5):
        i, j = rng.choice(35, 2, replace=False)
        a, b = int(rng.integers(1, p)), int(rng.integers(1, p))
        g = np.zeros(35, np.int64)
        g[i], g[j] = a, b
        D, delta = oracle.delta1(p, g, 4)
        expect = np.zeros(n_monomials(4 * p), np.int64)
        idx = mono_index(4 * p)
        I, J = mons[i], mons[j]
        for k in range(1, p):
            e = tuple(k * x + (p - k) * y for x, y in zip(I, J))
            expect[idx[e]] += (comb(p, k) // p) * a ** k * b ** (p - k)
        assert np.array_equal(delta, expect % p)


@pytest.mark.parametrize("p,deg", [(3, 8), (5, 8), (5, 16)])
def test_delta1_lift_independent(p, deg):
    g = _random_form(p, deg, 7 + p + deg)
    D0, d0 = oracle.delta1(p, g, deg, lift_signed=False)
    D1, d1 = oracle.delta1(p, g, deg, lift_signed=True)
    assert np.array_equal(D0, D1) and np.array_equal(d0, d1)


@pytest.mark.parametrize("p", [3, 5])
def test_power_is_frobenius_mod_p(p):
    # lift(g)^p = g(x^p) mod p: D mod p lives on the p-lattice and D[pJ] = c_J
    g = _random_form(p, 4 * (p - 1), 100 + p)
    D, _ = oracle.delta1(p, g, 4 * (p - 1))
    idx_big = mono_index(4 * p * (p - 1))
    expect = np.zeros(D.size, np.int64)
    for c, e in zip(g, monomials(4 * (p - 1))):
        expect[idx_big[tuple(p * x for x in e)]] = c
    assert np.array_equal(D % p, expect)


# ---------------------------------------------------------------- Algorithm 2
def test_split_u_example_sec4():
    # Example of Sec. 4.3: exactly ten monomials of B_16 match delta = x^(21,19,22,18) at p = 5.
    # u is linear and delta*m are distinct monomials, so u(sum_m delta*m) has one nonzero per matching m,
    # at (delta + m - (4,4,4,4)) / 5.
    p, d = 5, 16
    tuples, extra = read_tuples("wics_example.txt")
    delta = extra["delta"]
    deg = sum(delta) + d
    idx = mono_index(deg)
    P = np.zeros(n_monomials(deg), np.int64)
    for m in monomials(d):
        P[idx[tuple(x + y for x, y in zip(delta, m))]] = 1
    out_deg, U = oracle.split_u(p, P, deg)
    assert out_deg == (deg - 4 * (p - 1)) // p
    expect = np.zeros(U.size, np.int64)
    oidx = mono_index(out_deg)
    for m in tuples:
        assert sum(m) == d
        expect[oidx[tuple((x + y - (p - 1)) // p for x, y in zip(delta, m))]] = 1
    assert len(tuples) == 10 and np.array_equal(U, expect)


@pytest.mark.parametrize("p", [3, 5])
def test_split_u_on_monomials(p):
    # u(x^(p a + (p-1))) = x^a and u(x^b) = 0 unless every b_j = p-1 mod p
    rng = np.random.default_rng(p)
    for trial in range(20):
        a = rng.integers(0, 3, 4)
        if rng.random() < 0.5:
            b = p * a + (p - 1)
            want = tuple(int(x) for x in a)
        else:
            b = p * a + (p - 1)
            b[rng.integers(0, 4)] += 1 + rng.integers(0, p - 1)
            want = None
        deg = int(b.sum())
        rem = deg - 4 * (p - 1)
        if rem % p:
            continue
        P = np.zeros(n_monomials(deg), np.int64)
        P[mono_index(deg)[tuple(int(x) for x in b)]] = 1
        out_deg, U = oracle.split_u(p, P, deg)
        if want is None:
            assert not U.any()
        else:
            expect = np.zeros(U.size, np.int64)
            expect[mono_index(out_deg)[want]] = 1
            assert np.array_equal(U, expect)


# ---------------------------------------------------------------- two routes agree (heights and iterates)
@pytest.mark.parametrize("p,n", [(3, 120), (5, 60)])
def test_route_a_equals_route_r(p, n):
    f = np.concatenate([inputs.dense(p, n, 5000 + p), inputs.sparse(p, n, 6000 + p)])
    checked_iters = 0
    for row in f:
        a = oracle.stage_arrays_a(p, row)
        r = oracle.stage_arrays_r(p, row)
        assert a["h"] == r["h"]
        assert np.array_equal(a["iters"], r["iters"])
        checked_iters += a["iters"].shape[0]
    assert checked_iters > 0


@pytest.mark.parametrize("p,n", [(3, 60), (5, 40)])
def test_fchain_stage_arrays_equal_route_a(p, n):
    # D formed as lift(f)^(p(p-1)) by products with f's 35 terms equals route A's lift(g)^p (Sec. 3 reading on the
    # lift: (c + p b)^p = c^p mod p^2), and Algorithm 1's subtraction and division then give route A's Delta
    f = np.concatenate([inputs.dense(p, n, 5100 + p), inputs.sparse(p, n // 2, 5200 + p)])
    checked = 0
    for row in f:
        a = oracle.stage_arrays_a(p, row)
        c = oracle.stage_arrays_fchain(p, row)
        assert np.array_equal(a["g"], c["g"])
        assert c["h1"] == (a["h"] == 1)
        if a["h"] != 1:
            assert np.array_equal(a["D"], c["D"]) and np.array_equal(a["delta"], c["delta"])
            checked += 1
    assert checked > 5


def test_fchain_stage_arrays_equal_route_a_p7():
    row = next(r[3] for r in example_quartics() if r[0] == 7 and r[1] == 2)
    a = oracle.stage_arrays_a(7, row)
    c = oracle.stage_arrays_fchain(7, row)
    assert np.array_equal(a["D"], c["D"]) and np.array_equal(a["delta"], c["delta"])


# ---------------------------------------------------------------- invariance and statistics
@pytest.mark.parametrize("p,n", [(5, 300), (7, 150)])
def test_pgl4_invariance_route_r(p, n):
    f = inputs.dense(p, n, 7100 + p)
    A = inputs.pgl4_matrices(p, n, 7200 + p)
    g = inputs.substitute(f, A, p)
    h1, h2 = oracle.heights(p, f), oracle.heights(p, g)
    assert np.array_equal(h1, h2)
    assert (h1 >= 2).sum() > 0


def test_pgl4_invariance_route_a_p5():
    f = inputs.dense(5, 20, 7300)
    A = inputs.pgl4_matrices(5, 20, 7400)
    g = inputs.substitute(f, A, 5)
    assert np.array_equal(oracle.heights(5, f, route=oracle.ROUTE_A), oracle.heights(5, g, route=oracle.ROUTE_A))


def test_height_statistics_p5():
    # Heuristic of Sec. 7: height >= 2 with probability about 1/p (read as P(h >= k) ~ p^-(k-1)); wide 5-sigma band
    n, p = 3000, 5
    h = oracle.heights(p, inputs.dense(p, n, inputs.config_seed(2)))
    frac = float((h != 1).mean())
    sigma = (0.2 * 0.8 / n) ** 0.5
    assert abs(frac - 1 / p) < 5 * sigma
    assert set(np.unique(h)) <= set(range(0, 11))


# ------------------------------------------------------------------------------------- theta matrix (Sec. 3.4)
@pytest.mark.parametrize("p", [3, 5])
def test_theta_matrix_reproduces_route_a_iterates(p):
    """The matrix built from its definition (M[r][c] = Delta[p r + (p-1)1 - c]) maps each iterate of route A -- the
    full product Delta g followed by Algorithm 2's u -- to the next one."""
    f = inputs.dense(p, 300, 4100 + p)
    h = oracle.heights(p, f, route=oracle.ROUTE_A)
    rows = [i for i in range(len(f)) if h[i] >= 3 or h[i] == 0][:3]
    assert rows
    for i in rows:
        ref = oracle.stage_arrays_a(p, f[i])
        M = oracle.theta_matrix(p, f[i]).astype(np.int64)
        seq = [ref["g"].astype(np.int64)] + [x.astype(np.int64) for x in ref["iters"]]
        for a, b in zip(seq, seq[1:]):
            assert np.array_equal(M @ a % p, b)


def test_theta_matrix_shape_and_sparsity():
    """Entries outside the Delta cone are zero: at p = 3 the nonzero pattern of M covers at most the 60 % of
    entries whose exponent p r + (p-1)1 - c is nonnegative (nnz of M, 16,245 of 165^2)."""
    p = 3
    M = oracle.theta_matrix(p, inputs.dense(p, 1, 4200)[0])
    assert M.shape == (165, 165) and M.max() < p
    B = np.array(monomials(4 * (p - 1)))
    support = sum(int(((p * B[r][None, :] + (p - 1) - B) >= 0).all(axis=1).sum()) for r in range(len(B)))
    assert support == 16245
    assert np.count_nonzero(M) <= support


# ------------------------------------------------------------------------------------- matrix multiplication mod p (Sec. 5)
@pytest.mark.parametrize("p,n,m,k", [(11, 3, 4, 5), (2, 6, 1, 7), (251, 2, 3, 9)])
def test_matmul_mod_brute_force(p, n, m, k):
    rng = np.random.default_rng(p + n + m + k)
    A = rng.integers(0, p, (n, k))
    B = rng.integers(0, p, (k, m))
    want = [[sum(int(A[i][t]) * int(B[t][j]) for t in range(k)) % p for j in range(m)] for i in range(n)]
    assert np.array_equal(oracle.matmul_mod(p, A, B), np.array(want, np.uint8))


def test_matmul_mod_identity_and_associativity():
    p = 11
    rng = np.random.default_rng(5)
    A, B, C = (rng.integers(0, p, (8, 8)) for _ in range(3))
    assert np.array_equal(oracle.matmul_mod(p, A, np.eye(8, dtype=np.int64)), A.astype(np.uint8))
    assert np.array_equal(oracle.matmul_mod(p, oracle.matmul_mod(p, A, B), C),
                          oracle.matmul_mod(p, A, oracle.matmul_mod(p, B, C)))


# ------------------------------------------------------------------------------------- powering over Z (Sec. 4)
def _multinomial(es):
    from math import factorial
    out = factorial(sum(es))
    for e in es:
        out //= factorial(e)
    return out


def test_poly_power_sum_of_variables_is_multinomial():
    """(x1+x2+x3+x4)^2 to the 3rd power is (x1+...+x4)^6: every coefficient is a multinomial coefficient."""
    d, n = 2, 3
    f = [_multinomial(e) for e in oracle.form_monomials(d)]
    got = oracle.poly_power(d, f, n)
    assert got == [_multinomial(e) for e in oracle.form_monomials(d * n)]


def test_poly_power_evaluation_identity():
    """f^n evaluated at integer points equals f(point)^n."""
    rng = np.random.default_rng(4)
    d, n = 4, 3
    f = [int(x) for x in rng.integers(0, 5, len(oracle.form_monomials(d)))]
    P = oracle.poly_power(d, f, n)
    for pt in [(1, 2, 3, 4), (2, -1, 5, 0), (7, 1, 1, -3)]:
        ev = lambda cs, deg: sum(c * pt[0] ** e[0] * pt[1] ** e[1] * pt[2] ** e[2] * pt[3] ** e[3]
                                 for c, e in zip(cs, oracle.form_monomials(deg)))
        assert ev(P, d * n) == ev(f, d) ** n
