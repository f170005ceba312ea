/* Dense homogeneous polynomial helpers for the CPU oracle (test infrastructure; see hpoly.h). */
#include "hpoly.h"
#include <stdlib.h>
#include <string.h>

int64_t mod_pos(int64_t a, int64_t m) {
  int64_t r = a % m;
  return r < 0 ? r + m : r;
}

int64_t ipow_mod(int64_t a, int e, int64_t m) {
  int64_t r = 1 % m;
  a = mod_pos(a, m);
  for (int i = 0; i < e; i++) r = (r * a) % m;
  return r;
}

int64_t monomial_count(int d) {
  if (d < 0) return 0;
  return (int64_t)(d + 3) * (d + 2) * (d + 1) / 6;
}

int hpoly_init(hpoly *P, int deg) {
  P->deg = deg;
  P->side = deg + 1;
  size_t n = (size_t)P->side * P->side * P->side;
  P->c = (int64_t *)calloc(n, sizeof(int64_t));
  return P->c ? 0 : -1;
}

void hpoly_free(hpoly *P) {
  free(P->c);
  P->c = NULL;
}

int64_t *hpoly_at(const hpoly *P, int e1, int e2, int e3) {
  return &P->c[((size_t)e1 * P->side + e2) * P->side + e3];
}

void hpoly_reduce(hpoly *P, int64_t m) {
  size_t n = (size_t)P->side * P->side * P->side;
  for (size_t i = 0; i < n; i++) P->c[i] = mod_pos(P->c[i], m);
}

int hpoly_is_zero(const hpoly *P) {
  size_t n = (size_t)P->side * P->side * P->side;
  for (size_t i = 0; i < n; i++)
    if (P->c[i] != 0) return 0;
  return 1;
}

int hpoly_mul_mod(hpoly *C, const hpoly *A, const hpoly *B, int64_t m) {
  if (hpoly_init(C, A->deg + B->deg)) return -1;
  /* Term list of B, with each exponent turned into an offset in C's cube. */
  int64_t nb = 0;
  for (int e1 = 0; e1 <= B->deg; e1++)
    for (int e2 = 0; e1 + e2 <= B->deg; e2++)
      for (int e3 = 0; e1 + e2 + e3 <= B->deg; e3++)
        if (*hpoly_at(B, e1, e2, e3) != 0) nb++;
  int64_t *boff = (int64_t *)malloc(sizeof(int64_t) * (nb ? nb : 1));
  int64_t *bval = (int64_t *)malloc(sizeof(int64_t) * (nb ? nb : 1));
  if (!boff || !bval) { free(boff); free(bval); hpoly_free(C); return -1; }
  int64_t k = 0;
  for (int e1 = 0; e1 <= B->deg; e1++)
    for (int e2 = 0; e1 + e2 <= B->deg; e2++)
      for (int e3 = 0; e1 + e2 + e3 <= B->deg; e3++) {
        int64_t v = *hpoly_at(B, e1, e2, e3);
        if (v != 0) {
          boff[k] = ((int64_t)e1 * C->side + e2) * C->side + e3;
          bval[k] = v;
          k++;
        }
      }
  /* Textbook product: every term of A times every term of B, added into the monomial of their product. */
  for (int e1 = 0; e1 <= A->deg; e1++)
    for (int e2 = 0; e1 + e2 <= A->deg; e2++)
      for (int e3 = 0; e1 + e2 + e3 <= A->deg; e3++) {
        int64_t a = *hpoly_at(A, e1, e2, e3);
        if (a == 0) continue;
        int64_t *base = hpoly_at(C, e1, e2, e3);
        for (int64_t j = 0; j < nb; j++) base[boff[j]] += a * bval[j];
      }
  free(boff);
  free(bval);
#if QFS_MUTATE != 9 /* planted mistake 9: products left unreduced */
  hpoly_reduce(C, m);
#endif
  return 0;
}

void hpoly_from_desc_lex(hpoly *P, const int64_t *coeffs) {
  int64_t k = 0;
#if QFS_MUTATE == 10 /* planted mistake: coefficients read in ascending instead of descending lex order */
  for (int e1 = 0; e1 <= P->deg; e1++)
    for (int e2 = 0; e1 + e2 <= P->deg; e2++)
      for (int e3 = 0; e1 + e2 + e3 <= P->deg; e3++) *hpoly_at(P, e1, e2, e3) = coeffs[k++];
  return;
#endif
  for (int e1 = P->deg; e1 >= 0; e1--)
    for (int e2 = P->deg - e1; e2 >= 0; e2--)
      for (int e3 = P->deg - e1 - e2; e3 >= 0; e3--) *hpoly_at(P, e1, e2, e3) = coeffs[k++];
}

void hpoly_to_desc_lex(const hpoly *P, int32_t *out) {
  int64_t k = 0;
  for (int e1 = P->deg; e1 >= 0; e1--)
    for (int e2 = P->deg - e1; e2 >= 0; e2--)
      for (int e3 = P->deg - e1 - e2; e3 >= 0; e3--) out[k++] = (int32_t)*hpoly_at(P, e1, e2, e3);
}
