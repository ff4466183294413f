/*
 * ORACLE (test infrastructure only).  Plain 320-bit complex matrix products, the definition of the
 * dense products A X, X^H X and X^H (A X) that the refinement step needs (the "recover the precision"
 * stage of Section 2, ZKCM_CUS paragraph).
 */
#include "mp.h"
#include <stdlib.h>

/* C = op(A) * B, A: (op: 0 -> m x k, 1 -> A is k x m and op = conjugate transpose), B: k x n;
 * column-major complex, wa/wb words per real; C: m x n, wc words. */
int oracle_matmul(int m, int n, int k, int opA, const double* A, int wa, const double* B, int wb,
                  double* C, int wc) {
  cmp_t* a = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)m * k);
  cmp_t* b = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)k * n);
  if (!a || !b) return 3;
  int ar = opA ? k : m;                                /* rows of stored A */
  for (size_t e = 0; e < (size_t)m * k; ++e) {
    mp_from_words(&a[e].re, A + (e * 2 + 0) * wa, wa);
    mp_from_words(&a[e].im, A + (e * 2 + 1) * wa, wa);
  }
  for (size_t e = 0; e < (size_t)k * n; ++e) {
    mp_from_words(&b[e].re, B + (e * 2 + 0) * wb, wb);
    mp_from_words(&b[e].im, B + (e * 2 + 1) * wb, wb);
  }
  for (int j = 0; j < n; ++j) for (int i = 0; i < m; ++i) {
    cmp_t s, t; cmp_zero(&s);
    for (int l = 0; l < k; ++l) {
      if (opA) cmp_mul_conj(&t, &a[(size_t)l + (size_t)i * ar], &b[(size_t)l + (size_t)j * k]);
      else cmp_mul(&t, &a[(size_t)i + (size_t)l * ar], &b[(size_t)l + (size_t)j * k]);
      cmp_add(&s, &s, &t);
    }
    size_t e = (size_t)i + (size_t)j * m;
    mp_to_words(&s.re, C + (e * 2 + 0) * wc, wc);
    mp_to_words(&s.im, C + (e * 2 + 1) * wc, wc);
  }
  free(a); free(b);
  return 0;
}

/* elementwise exact-ish conversion helper used by tests: words (count x w) -> words (count x w_out) */
void oracle_rewords(long count, const double* x, int w, double* y, int w_out) {
  for (long i = 0; i < count; ++i) { mp t; mp_from_words(&t, x + i * w, w); mp_to_words(&t, y + i * w_out, w_out); }
}

/* scalar ops for pinning mp itself: op 0 add, 1 sub, 2 mul, 3 div, 4 sqrt(a) */
void oracle_scalar(int op, const double* a, const double* b, int w, double* out, int w_out) {
  mp x, y, r; mp_from_words(&x, a, w); mp_from_words(&y, b, w);
  switch (op) {
    case 0: mp_add(&r, &x, &y); break;
    case 1: mp_sub(&r, &x, &y); break;
    case 2: mp_mul(&r, &x, &y); break;
    case 3: mp_div(&r, &x, &y); break;
    default: mp_sqrt(&r, &x); break;
  }
  mp_to_words(&r, out, w_out);
}
