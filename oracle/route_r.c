/*
 * CPU oracle, route R: a second, independent derivation of the same heights -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this code.
 *
 * Derivation (from the Proposition of Sec. 3.1 and Algorithm 2; the paper does not state it):
 *   Let f~ lift f and A = sum_I a~_I^p x^(pI).  The Proposition gives f~^p = A + p D~ with D~ = Delta_1(f) mod p.
 *   Then f~^(p(p-1)) = (A + p D~)^(p-1) = A^(p-1) - p A^(p-2) D~ (mod p^2).  Since A^(p-1) and the subtracted terms
 *   of Algorithm 1 both live on the p-lattice and A^(p-2) = f(x^p)^(p-2) (mod p),
 *       Delta_1(f^(p-1)) = E(x^p) - f(x^p)^(p-2) Delta_1(f)   (mod p)   for some form E.
 *   u is semilinear over p-th powers (u(h(x^p) k) = h u(k), read off Algorithm 2), and for F of degree 4(p-1)
 *   u(F) is the single coefficient F[(p-1,..,p-1)].  Hence for such F
 *       u(F Delta_1(f^(p-1))) = E F[(p-1,..,p-1)] - f^(p-2) u(F Delta_1(f)),
 *   and the iteration only applies the map to F whose witness coefficient is zero, so there
 *       theta(F) = - f^(p-2) u(F Delta_1(f))   (mod p),
 *   where u(F Delta_1(f)) is a quartic.  The Delta_1(f^(p-1)) array of degree 4p(p-1) is never formed.
 * Heights, zero-iterate exit and return codes follow route A exactly.
 */
#include "hpoly.h"
#include <stdlib.h>
#include <string.h>

static int load_quartic_r(int p, const uint8_t *f35, hpoly *f) {
  int64_t c[35];
  for (int i = 0; i < 35; i++) {
    if (f35[i] >= p) return -1;
    c[i] = f35[i];
  }
  if (hpoly_init(f, 4)) return -3;
  hpoly_from_desc_lex(f, c);
  return 0;
}

/* P := B^k mod m (k >= 1) by repeated multiplication. */
static int power_mod(hpoly *P, const hpoly *B, int k, int64_t m) {
  hpoly acc, t;
  if (hpoly_init(&acc, B->deg)) return -1;
  memcpy(acc.c, B->c, (size_t)B->side * B->side * B->side * sizeof(int64_t));
  hpoly_reduce(&acc, m);
  for (int i = 2; i <= k; i++) {
    if (hpoly_mul_mod(&t, &acc, B, m)) { hpoly_free(&acc); return -1; }
    hpoly_free(&acc);
    acc = t;
  }
  *P = acc;
  return 0;
}

/* Returns the same codes as qfs_oracle_height_a.  Optional outputs: d1f_out = Delta_1(f) mod p in descending-lex
   order (C(4p+3,3) values, written only when the height-1 test fails) and iters_out as in route A. */
int qfs_oracle_height_r(int p, const uint8_t *f35, int max_h, int32_t *d1f_out, int32_t *iters_out) {
  const int64_t p2 = (int64_t)p * p;
  hpoly f, fpm2, g, fp;
  int rc = load_quartic_r(p, f35, &f);
  if (rc) return rc;
  /* f^(p-2) mod p (the constant 1 when p = 2 is excluded: p >= 3 here) and g = f^(p-1) = f^(p-2) f */
  if (p == 2) { hpoly_free(&f); return -3; }
  if (p == 3) {
    if (hpoly_init(&fpm2, 4)) { hpoly_free(&f); return -3; }
    memcpy(fpm2.c, f.c, (size_t)f.side * f.side * f.side * sizeof(int64_t));
  } else if (power_mod(&fpm2, &f, p - 2, p)) { hpoly_free(&f); return -3; }
  if (hpoly_mul_mod(&g, &fpm2, &f, p)) { hpoly_free(&fpm2); hpoly_free(&f); return -3; }
  if (*hpoly_at(&g, p - 1, p - 1, p - 1) != 0) { hpoly_free(&g); hpoly_free(&fpm2); hpoly_free(&f); return 1; }
  /* Delta_1(f) = (f~^p - sum a~_I^p x^(pI)) / p mod p, with the [0,p) lift */
  if (power_mod(&fp, &f, p, p2)) { hpoly_free(&g); hpoly_free(&fpm2); hpoly_free(&f); return -3; }
  for (int e1 = 0; e1 <= 4; e1++)
    for (int e2 = 0; e1 + e2 <= 4; e2++)
      for (int e3 = 0; e1 + e2 + e3 <= 4; e3++) {
        int64_t a = *hpoly_at(&f, e1, e2, e3);
        if (a == 0) continue;
        int64_t *slot = hpoly_at(&fp, p * e1, p * e2, p * e3);
        *slot = mod_pos(*slot - ipow_mod(a, p, p2), p2);
      }
  hpoly_free(&f);
  size_t nfp = (size_t)fp.side * fp.side * fp.side;
  int bad = 0;
  for (size_t i = 0; i < nfp; i++) {
    if (fp.c[i] % p != 0) bad = 1;
    fp.c[i] = mod_pos(fp.c[i] / p, p);
  }
  if (bad) { hpoly_free(&fp); hpoly_free(&g); hpoly_free(&fpm2); return -2; }
  if (d1f_out) hpoly_to_desc_lex(&fp, d1f_out);
  const int64_t ld = monomial_count(4 * (p - 1));
  int result = 0;
  for (int h = 2; h <= max_h; h++) {
    hpoly prod, q, next;
    /* q = u(g Delta_1(f)), a quartic, by Algorithm 2's rule */
    if (hpoly_mul_mod(&prod, &g, &fp, p)) { result = -3; break; }
    if (hpoly_init(&q, 4)) { hpoly_free(&prod); result = -3; break; }
    for (int e1 = 0; e1 <= prod.deg; e1++)
      for (int e2 = 0; e1 + e2 <= prod.deg; e2++)
        for (int e3 = 0; e1 + e2 + e3 <= prod.deg; e3++) {
          int e4 = prod.deg - e1 - e2 - e3;
          int64_t c = *hpoly_at(&prod, e1, e2, e3);
          if (c == 0) continue;
          if (e1 % p == p - 1 && e2 % p == p - 1 && e3 % p == p - 1 && e4 % p == p - 1)
            *hpoly_at(&q, (e1 - (p - 1)) / p, (e2 - (p - 1)) / p, (e3 - (p - 1)) / p) += c;
        }
    hpoly_free(&prod);
    hpoly_reduce(&q, p);
    /* g <- -f^(p-2) q */
    if (hpoly_mul_mod(&next, &fpm2, &q, p)) { hpoly_free(&q); result = -3; break; }
    hpoly_free(&q);
    size_t nn = (size_t)next.side * next.side * next.side;
#if QFS_MUTATE == 6 /* planted mistake: the minus sign of the reduced step dropped */
    for (size_t i = 0; i < nn; i++) next.c[i] = mod_pos(next.c[i], p);
#else
    for (size_t i = 0; i < nn; i++) next.c[i] = mod_pos(-next.c[i], p);
#endif
    hpoly_free(&g);
    g = next;
    if (iters_out) hpoly_to_desc_lex(&g, iters_out + (int64_t)(h - 2) * ld);
    if (*hpoly_at(&g, p - 1, p - 1, p - 1) != 0) { result = h; break; }
    if (hpoly_is_zero(&g)) { result = 0; break; }
  }
  hpoly_free(&g);
  hpoly_free(&fpm2);
  hpoly_free(&fp);
  return result;
}
