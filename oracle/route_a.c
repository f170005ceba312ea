/*
 * CPU oracle, route A: the paper's naive algorithm taken literally -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this code.
 *
 *   Algorithm 1 (calculation of Delta_1):  lift, D <- lift^p, subtract t^p for every term t, divide by p.
 *   Algorithm 2 (splitting u):             keep terms whose exponents are all = p-1 mod p, map e -> (e-(p-1))/p.
 *   Algorithm 3 (naive height):            g <- f^(p-1); test; Delta <- Delta_1(f^(p-1)); loop g <- u(Delta g), test.
 *
 * The membership test "g not in m^[p]" reads one coefficient: for a form of degree 4(p-1) in four variables the
 * only monomial outside m^[p] = (x1^p, .., x4^p) is (x1 x2 x3 x4)^(p-1) (Sec. 3.3, matrix-based algorithm).
 *
 * Readings of the paper that this file takes:
 *  - Delta_1 follows the Proposition of Sec. 3.1: (lift^p - sum of (lifted term)^p) / p reduced mod p.  The W_2
 *    addition polynomial printed in Sec. 2 has the opposite sign; heights do not depend on that sign.
 *  - "terms(f~)" in Algorithm 1 are the terms of the lift of g = f^(p-1) reduced mod p.  Any termwise lift gives
 *    the same result mod p because (c + p b)^p = c^p mod p^2; lift_signed selects the symmetric lift to show it.
 *  - D <- lift^p is only needed mod p^2, since (D - S)/p is then known mod p; the power is formed by repeated
 *    multiplication by the lift.
 *  - The loop of Algorithm 3 runs h = 2 .. max_h inclusive; it returns 0 for "infinity / not found by max_h".
 *    If an iterate is identically zero it returns 0 at once: the map g -> u(Delta g) is linear, so every later
 *    iterate is zero too (the Fermat example of Sec. 3.3 notes that the iterate vanishes).
 */
#include "hpoly.h"
#include <stdlib.h>
#include <string.h>

/* The end of Algorithm 1, given D = lift^p mod p^2 for the lift `lift` of g: subtract t^p for every term t of the
   lift, divide by p and read the result mod p into Delta.  Consumes D and lift.  Returns 0, -2 if a division is not
   exact, or -1 on allocation failure. */
static int alg1_subtract_divide(int p, hpoly *lift, hpoly *D, hpoly *Delta);

/* Algorithm 1 on a homogeneous g of degree deg with coefficients in [0,p).  Fills D (= lift^p mod p^2, before the
   subtraction) and Delta (mod p), both of degree p*deg.  Returns 0, or -2 if some coefficient of D - S is not
   divisible by p (impossible by the Proposition; reported rather than ignored), or -1 on allocation failure. */
static int delta1_alg1(int p, const hpoly *g, int lift_signed, hpoly *D_out, hpoly *Delta) {
  const int64_t p2 = (int64_t)p * p;
  hpoly lift;
  if (hpoly_init(&lift, g->deg)) return -1;
  size_t n = (size_t)g->side * g->side * g->side;
  for (size_t i = 0; i < n; i++) {
    int64_t c = mod_pos(g->c[i], p);
    if (lift_signed && 2 * c > p) c -= p;
    lift.c[i] = c;
  }
  /* D <- lift^p, by p-1 multiplications, reduced mod p^2 after each. */
  hpoly D, next;
  if (hpoly_init(&D, g->deg)) { hpoly_free(&lift); return -1; }
  memcpy(D.c, lift.c, n * sizeof(int64_t));
  hpoly_reduce(&D, p2);
  for (int k = 2; k <= p; k++) {
#if QFS_MUTATE == 4 /* planted mistake: lift^p taken mod p instead of mod p^2 */
    if (hpoly_mul_mod(&next, &D, &lift, p)) { hpoly_free(&D); hpoly_free(&lift); return -1; }
#else
    if (hpoly_mul_mod(&next, &D, &lift, p2)) { hpoly_free(&D); hpoly_free(&lift); return -1; }
#endif
    hpoly_free(&D);
    D = next;
  }
  if (D_out) {
    if (hpoly_init(D_out, D.deg)) { hpoly_free(&D); hpoly_free(&lift); return -1; }
    memcpy(D_out->c, D.c, (size_t)D.side * D.side * D.side * sizeof(int64_t));
  }
  return alg1_subtract_divide(p, &lift, &D, Delta);
}

static int alg1_subtract_divide(int p, hpoly *lift_in, hpoly *D_in, hpoly *Delta) {
  const int64_t p2 = (int64_t)p * p;
  hpoly lift = *lift_in, D = *D_in;
  const hpoly *g = &lift;
  /* D <- D - t^p for every term t = c x^J of the lift: t^p = c^p x^(pJ). */
  for (int e1 = 0; e1 <= g->deg; e1++)
    for (int e2 = 0; e1 + e2 <= g->deg; e2++)
      for (int e3 = 0; e1 + e2 + e3 <= g->deg; e3++) {
        int64_t c = *hpoly_at(&lift, e1, e2, e3);
        if (c == 0) continue;
#if QFS_MUTATE == 14 /* planted mistake: t^p subtracted at a transposed lattice point */
        int64_t *slot = hpoly_at(&D, p * e2, p * e1, p * e3);
#else
        int64_t *slot = hpoly_at(&D, p * e1, p * e2, p * e3);
#endif
#if QFS_MUTATE == 8 /* planted mistake: c^(p-1) subtracted instead of c^p */
        *slot = mod_pos(*slot - ipow_mod(c, p - 1, p2), p2);
#else
        *slot = mod_pos(*slot - ipow_mod(c, p, p2), p2);
#endif
      }
  hpoly_free(&lift);
  /* D <- D / p: exact division, then the result is read mod p. */
  if (hpoly_init(Delta, D.deg)) { hpoly_free(&D); return -1; }
  size_t nd = (size_t)D.side * D.side * D.side;
  int bad = 0;
  for (size_t i = 0; i < nd; i++) {
    if (D.c[i] % p != 0) bad = 1;
#if QFS_MUTATE == 1 /* planted mistake: sign of Delta_1 */
    Delta->c[i] = mod_pos(-(D.c[i] / p), p);
#else
    Delta->c[i] = mod_pos(D.c[i] / p, p);
#endif
  }
  hpoly_free(&D);
  return bad ? -2 : 0;
}

/* Algorithm 2: u(P).  The result has degree (deg P - 4(p-1))/p; returns -1 if that is not a non-negative
   integer (then no term survives and the map is zero, as the paper's convention for d' says). */
static int split_u_alg2(int p, const hpoly *P, hpoly *out) {
  int rem = P->deg - 4 * (p - 1);
  if (rem < 0 || rem % p != 0) return -1;
  if (hpoly_init(out, rem / p)) return -1;
  for (int e1 = 0; e1 <= P->deg; e1++)
    for (int e2 = 0; e1 + e2 <= P->deg; e2++)
      for (int e3 = 0; e1 + e2 + e3 <= P->deg; e3++) {
        int e4 = P->deg - e1 - e2 - e3;
        int64_t c = *hpoly_at(P, e1, e2, e3);
        if (c == 0) continue;
        if (e1 % p == p - 1 && e2 % p == p - 1 && e3 % p == p - 1 && e4 % p == p - 1)
#if QFS_MUTATE == 2 /* planted mistake: transposed output exponents in u */
          *hpoly_at(out, (e2 - (p - 1)) / p, (e1 - (p - 1)) / p, (e3 - (p - 1)) / p) += c;
#else
          *hpoly_at(out, (e1 - (p - 1)) / p, (e2 - (p - 1)) / p, (e3 - (p - 1)) / p) += c;
#endif
      }
  return 0;
}

static int64_t witness_coeff(int p, const hpoly *g) {
#if QFS_MUTATE == 3 /* planted mistake: wrong witness monomial */
  return *hpoly_at(g, p - 1, p - 1, p - 2);
#else
  return *hpoly_at(g, p - 1, p - 1, p - 1);
#endif
}

static int load_quartic(int p, const uint8_t *f35, hpoly *f) {
  int64_t c[35];
  for (int i = 0; i < 35; i++) {
    if (f35[i] >= p) return -1;
    c[i] = f35[i];
  }
  if (hpoly_init(f, 4)) return -3;
  hpoly_from_desc_lex(f, c);
  return 0;
}

int qfs_oracle_delta1(int p, int deg, const int32_t *g_desc, int lift_signed, int32_t *D_out, int32_t *delta_out) {
  int64_t n = monomial_count(deg);
  int64_t *c = (int64_t *)malloc(sizeof(int64_t) * n);
  if (!c) return -1;
  for (int64_t i = 0; i < n; i++) c[i] = mod_pos(g_desc[i], p);
  hpoly g, D, Delta;
  if (hpoly_init(&g, deg)) { free(c); return -1; }
  hpoly_from_desc_lex(&g, c);
  free(c);
  int rc = delta1_alg1(p, &g, lift_signed, D_out ? &D : NULL, &Delta);
  hpoly_free(&g);
  if (rc == -1) return -1;
  if (D_out) { hpoly_to_desc_lex(&D, D_out); hpoly_free(&D); }
  if (delta_out) hpoly_to_desc_lex(&Delta, delta_out);
  hpoly_free(&Delta);
  return rc;
}

int qfs_oracle_split_u(int p, int deg, const int32_t *P_desc, int32_t *out) {
  int64_t n = monomial_count(deg);
  int64_t *c = (int64_t *)malloc(sizeof(int64_t) * n);
  if (!c) return -1;
  for (int64_t i = 0; i < n; i++) c[i] = P_desc[i];
  hpoly P, U;
  if (hpoly_init(&P, deg)) { free(c); return -1; }
  hpoly_from_desc_lex(&P, c);
  free(c);
  int rc = split_u_alg2(p, &P, &U);
  hpoly_free(&P);
  if (rc) return -1;
  hpoly_reduce(&U, p);
  hpoly_to_desc_lex(&U, out);
  int d = U.deg;
  hpoly_free(&U);
  return d;
}

/* Stage arrays of Algorithms 1 and 3 for one quartic with D formed as lift(f)^(p(p-1)) mod p^2, one product by
   the lift of f at a time, instead of lift(g)^p by products of the lift of g = f^(p-1) (route A).  The two are the
   same array: termwise lifts agree mod p, and (c + p b)^p = c^p mod p^2 carries that to the p-th power, so
   lift(g)^p = (lift(f)^(p-1) + p B)^p = lift(f)^(p(p-1)) mod p^2.  Products by the 35 terms of f keep the p = 11 and
   p = 13 arrays within a test's time, where products by the C(4p-1,3) terms of g do not.  Outputs as for
   qfs_oracle_height_a: g_out = f^(p-1) mod p, then (if the witness coefficient is zero) D_out and delta_out.
   Returns 1 if the witness coefficient is nonzero, 0 if D and Delta were written, -1 for a coefficient >= p, -2 if
   a division by p was not exact, -3 on allocation failure. */
int qfs_oracle_stages_fchain(int p, const uint8_t *f35, int32_t *g_out, int32_t *D_out, int32_t *delta_out) {
  const int64_t p2 = (int64_t)p * p;
  hpoly f, g, t;
  int rc = load_quartic(p, f35, &f);
  if (rc) return rc;
  if (hpoly_init(&g, 0)) { hpoly_free(&f); return -3; }
  g.c[0] = 1;
  for (int k = 1; k <= p - 1; k++) {
    if (hpoly_mul_mod(&t, &g, &f, p)) { hpoly_free(&g); hpoly_free(&f); return -3; }
    hpoly_free(&g);
    g = t;
  }
  if (g_out) hpoly_to_desc_lex(&g, g_out);
  if (witness_coeff(p, &g) != 0) { hpoly_free(&g); hpoly_free(&f); return 1; }
  /* D <- lift(f)^(p(p-1)) mod p^2 (f's coefficients are already in [0, p)) */
  hpoly D;
  if (hpoly_init(&D, 0)) { hpoly_free(&g); hpoly_free(&f); return -3; }
  D.c[0] = 1;
  for (int k = 1; k <= p * (p - 1); k++) {
    if (hpoly_mul_mod(&t, &D, &f, p2)) { hpoly_free(&D); hpoly_free(&g); hpoly_free(&f); return -3; }
    hpoly_free(&D);
    D = t;
  }
  hpoly_free(&f);
  if (D_out) hpoly_to_desc_lex(&D, D_out);
  hpoly Delta;
  rc = alg1_subtract_divide(p, &g, &D, &Delta);   /* the lift of g is g itself: coefficients in [0, p) */
  if (rc == -1) return -3;
  if (delta_out) hpoly_to_desc_lex(&Delta, delta_out);
  hpoly_free(&Delta);
  return rc == -2 ? -2 : 0;
}

/* Algorithm 3.  Returns the height 1..max_h, 0 for infinity / not found by max_h, -1 for a coefficient >= p,
   -2 if the exact division of Algorithm 1 failed, -3 on allocation failure.  Optional outputs (descending-lex
   order): g_out = f^(p-1) mod p (C(4p-1,3) values), D_out = lift(g)^p mod p^2 and delta_out = Delta_1(g)
   (C(4p(p-1)+3,3) values each; written only if the height-1 test fails), iters_out = the iterates g_2, g_3, ...
   (row h-2 holds g_h, C(4p-1,3) values per row; rows past the returned height are left untouched). */
int qfs_oracle_height_a(int p, const uint8_t *f35, int max_h, int lift_signed, int32_t *g_out, int32_t *D_out,
                        int32_t *delta_out, int32_t *iters_out) {
  hpoly f, g, t;
  int rc = load_quartic(p, f35, &f);
  if (rc) return rc;
  /* g <- f^(p-1) over F_p */
  if (hpoly_init(&g, 0)) { hpoly_free(&f); return -3; }
  g.c[0] = 1;
#if QFS_MUTATE == 7 /* planted mistake: f^(p-2) instead of f^(p-1) */
  for (int k = 1; k <= p - 2; k++) {
#else
  for (int k = 1; k <= p - 1; k++) {
#endif
    if (hpoly_mul_mod(&t, &g, &f, p)) { hpoly_free(&g); hpoly_free(&f); return -3; }
    hpoly_free(&g);
    g = t;
  }
  hpoly_free(&f);
  if (g_out) hpoly_to_desc_lex(&g, g_out);
  if (witness_coeff(p, &g) != 0) { hpoly_free(&g); return 1; }
  /* Delta <- Delta_1(f^(p-1)) by Algorithm 1 */
  hpoly Delta, D;
  rc = delta1_alg1(p, &g, lift_signed, D_out ? &D : NULL, &Delta);
  if (rc) {
    if (rc == -2) { if (D_out) hpoly_free(&D); hpoly_free(&Delta); }
    hpoly_free(&g);
    return rc == -1 ? -3 : rc;
  }
  if (D_out) { hpoly_to_desc_lex(&D, D_out); hpoly_free(&D); }
  if (delta_out) hpoly_to_desc_lex(&Delta, delta_out);
  const int64_t ld = monomial_count(4 * (p - 1));
  int result = 0;
#if QFS_MUTATE == 12 /* planted mistake: the bound b tested with < instead of <= */
  for (int h = 2; h < max_h; h++) {
#else
  for (int h = 2; h <= max_h; h++) {
#endif
    hpoly prod, next;
    if (hpoly_mul_mod(&prod, &Delta, &g, p)) { result = -3; break; }
    rc = split_u_alg2(p, &prod, &next);
    hpoly_free(&prod);
    if (rc) { result = -3; break; }
    hpoly_reduce(&next, p);
    hpoly_free(&g);
    g = next;
    if (iters_out) hpoly_to_desc_lex(&g, iters_out + (int64_t)(h - 2) * ld);
    if (witness_coeff(p, &g) != 0) { result = h; break; }
#if QFS_MUTATE == 11 /* planted mistake: a zero iterate read as height 1 */
    if (hpoly_is_zero(&g)) { result = 1; break; }
#else
    if (hpoly_is_zero(&g)) { result = 0; break; }
#endif
  }
  hpoly_free(&g);
  hpoly_free(&Delta);
  return result;
}
