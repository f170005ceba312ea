/*
 * Plain CPU oracle for quasi-F-split heights of quartic surfaces -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this code.
 * It shares no source with the CUDA path and is deliberately slow and literal.
 *
 * Dense homogeneous polynomials in x1..x4 with integer coefficients.
 * A polynomial of total degree d is a cube of side d+1 indexed by (e1, e2, e3); the exponent of x4 is
 * d - e1 - e2 - e3.  Cube entries with e1 + e2 + e3 > d are unused and stay zero.  This is the plainest
 * representation of "a homogeneous polynomial as a list of its terms" (paper Sec. 4, Def. of exps/coeff):
 * every monomial has its own slot and a product is the textbook double loop over terms.
 */
#ifndef QFS_ORACLE_HPOLY_H
#define QFS_ORACLE_HPOLY_H
/* QFS_MUTATE = k compiles planted mistake k (tests check that the pins catch each one); 0 = the oracle. */
#ifndef QFS_MUTATE
#define QFS_MUTATE 0
#endif
#include <stdint.h>

typedef struct {
  int deg;      /* total degree */
  int side;     /* deg + 1 */
  int64_t *c;   /* side^3 coefficients */
} hpoly;

int hpoly_init(hpoly *P, int deg);                 /* zero polynomial of degree deg; 0 on success */
void hpoly_free(hpoly *P);
int64_t *hpoly_at(const hpoly *P, int e1, int e2, int e3);
/* C := A * B with every coefficient reduced into [0, m).  C must not alias A or B. */
int hpoly_mul_mod(hpoly *C, const hpoly *A, const hpoly *B, int64_t m);
void hpoly_reduce(hpoly *P, int64_t m);           /* coefficients into [0, m) */
int hpoly_is_zero(const hpoly *P);
/* Number of monomials of degree d in 4 variables: C(d+3, 3) (paper Lemma on |wics(k,n)|). */
int64_t monomial_count(int d);
/* Conversion to and from the descending-lex coefficient list: x1 exponent descending, then x2, then x3. */
void hpoly_from_desc_lex(hpoly *P, const int64_t *coeffs);
void hpoly_to_desc_lex(const hpoly *P, int32_t *out);
int64_t mod_pos(int64_t a, int64_t m);
int64_t ipow_mod(int64_t a, int e, int64_t m);
#endif
