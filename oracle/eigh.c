/*
 * ORACLE (test infrastructure only; only tests/, the smoke check and the bench's CPU-baseline leg may
 * load it).  Plain cyclic-by-row complex Jacobi eigensolver for a Hermitian matrix, in the 320-bit
 * arithmetic of mp.c.  It computes the plain definition of what the paper's diagonalisation step
 * produces (Section 2, "Hermitian matrix diagonalization", whose cost dominates the MPS simulation,
 * Section 2.1): all eigenvalues and orthonormal eigenvectors of A, to ~2^-300 ||A||.
 *
 * Rotation for the pair (p, q), b = a_pq = |b| e^{i phi}:
 *   tau = (a_qq - a_pp) / (2|b|),  t = sign(tau) / (|tau| + sqrt(1 + tau^2))  (t = 1 if tau = 0),
 *   c = 1/sqrt(1 + t^2),  s = t c,  J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] on rows/cols (p, q).
 * Then (J^H A J)_pq = e^{i phi}(|b|(c^2 - s^2) + cs(a_pp - a_qq)) = 0 because t^2 + 2 tau t - 1 = 0,
 * and the new diagonal is a_pp - t|b|, a_qq + t|b| (trace preserved).  A <- J^H A J, V <- V J.
 * A sweep visits p < q in row order and skips |a_pq| <= 2^-300 ||A||_F; the run stops after a sweep
 * with no rotation.
 *
 * Output conventions: eigenvalues in descending order (ties keep the original index order); each
 * eigenvector scaled by a unit phase so that its first component of largest modulus is real > 0.
 */
#include "mp.h"
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, n) ((size_t)(i) + (size_t)(j) * (size_t)(n))

static void load_c(cmp_t* z, const double* A, size_t e, int w) {
  mp_from_words(&z->re, A + (e * 2 + 0) * w, w);
  mp_from_words(&z->im, A + (e * 2 + 1) * w, w);
}
static void store_c(const cmp_t* z, double* out, size_t e, int w) {
  mp_to_words(&z->re, out + (e * 2 + 0) * w, w);
  mp_to_words(&z->im, out + (e * 2 + 1) * w, w);
}

/* core solver on an mp matrix (full storage, Hermitian); returns sweeps used or -1 if not converged */
int oracle_jacobi_mp(int n, cmp_t* a, cmp_t* v, int max_sweeps) {
  mp fro, t1;
  mp_zero(&fro);
  for (size_t k = 0; k < (size_t)n * n; ++k) { cmp_abs2(&t1, &a[k]); mp_add(&fro, &fro, &t1); }
  mp_sqrt(&fro, &fro);
  mp tol; mp_ldexp(&tol, &fro, -300);
  for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
    cmp_zero(&v[IDX(i, j, n)]);
    if (i == j) mp_from_double(&v[IDX(i, j, n)].re, 1.0);
  }
  if (mp_is_zero(&fro)) return 0;
  mp one; mp_from_double(&one, 1.0);
  for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
    int rotations = 0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        cmp_t b = a[IDX(p, q, n)];
        mp absb; cmp_abs2(&absb, &b); mp_sqrt(&absb, &absb);
        if (mp_cmp(&absb, &tol) <= 0) continue;
        ++rotations;
        cmp_t ephi; mp_div(&ephi.re, &b.re, &absb); mp_div(&ephi.im, &b.im, &absb);
        mp tau, t, c, s, num, den;
        mp_sub(&num, &a[IDX(q, q, n)].re, &a[IDX(p, p, n)].re);
        mp_ldexp(&den, &absb, 1);
        mp_div(&tau, &num, &den);
        if (mp_is_zero(&tau)) {
          t = one;
        } else {
          mp at, r; mp_abs(&at, &tau);
          mp_mul(&r, &tau, &tau); mp_add(&r, &r, &one); mp_sqrt(&r, &r);
          mp_add(&r, &r, &at); mp_div(&t, &one, &r);
          if (mp_sign(&tau) < 0) mp_neg(&t, &t);
        }
        mp_mul(&c, &t, &t); mp_add(&c, &c, &one); mp_sqrt(&c, &c); mp_div(&c, &one, &c);
        mp_mul(&s, &t, &c);
        cmp_t z1, z2;                                 /* z1 = s e^{-i phi}, z2 = s e^{i phi} */
        mp_mul(&z2.re, &s, &ephi.re); mp_mul(&z2.im, &s, &ephi.im);
        z1.re = z2.re; mp_neg(&z1.im, &z2.im);
        for (int i = 0; i < n; ++i) {
          if (i == p || i == q) continue;
          cmp_t x = a[IDX(i, p, n)], y = a[IDX(i, q, n)], u1, u2, np_, nq;
          cmp_scale(&u1, &x, &c); cmp_mul(&u2, &z1, &y); cmp_sub(&np_, &u1, &u2);   /* c x - z1 y */
          cmp_mul(&u1, &z2, &x); cmp_scale(&u2, &y, &c); cmp_add(&nq, &u1, &u2);    /* z2 x + c y */
          a[IDX(i, p, n)] = np_; a[IDX(i, q, n)] = nq;
          cmp_conj(&a[IDX(p, i, n)], &np_); cmp_conj(&a[IDX(q, i, n)], &nq);
        }
        mp tb; mp_mul(&tb, &t, &absb);
        mp_sub(&a[IDX(p, p, n)].re, &a[IDX(p, p, n)].re, &tb);
        mp_add(&a[IDX(q, q, n)].re, &a[IDX(q, q, n)].re, &tb);
        cmp_zero(&a[IDX(p, q, n)]); cmp_zero(&a[IDX(q, p, n)]);
        for (int i = 0; i < n; ++i) {
          cmp_t x = v[IDX(i, p, n)], y = v[IDX(i, q, n)], u1, u2, np_, nq;
          cmp_scale(&u1, &x, &c); cmp_mul(&u2, &z1, &y); cmp_sub(&np_, &u1, &u2);
          cmp_mul(&u1, &z2, &x); cmp_scale(&u2, &y, &c); cmp_add(&nq, &u1, &u2);
          v[IDX(i, p, n)] = np_; v[IDX(i, q, n)] = nq;
        }
      }
    }
    if (rotations == 0) return sweep;
  }
  return -1;
}

/* sort descending (stable), normalise eigenvector phases; lam[i] = a_ii */
void oracle_finish_mp(int n, const cmp_t* a, cmp_t* v, mp* lam, int* order) {
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 1; i < n; ++i) {                        /* insertion sort: stable */
    int k = order[i], j = i - 1;
    while (j >= 0 && mp_cmp(&a[IDX(order[j], order[j], n)].re, &a[IDX(k, k, n)].re) < 0) { order[j + 1] = order[j]; --j; }
    order[j + 1] = k;
  }
  for (int i = 0; i < n; ++i) lam[i] = a[IDX(order[i], order[i], n)].re;
  for (int c = 0; c < n; ++c) {
    cmp_t* col = v + (size_t)n * c;
    int best = 0; mp bm, t; cmp_abs2(&bm, &col[0]);
    for (int i = 1; i < n; ++i) { cmp_abs2(&t, &col[i]); if (mp_cmp(&t, &bm) > 0) { bm = t; best = i; } }
    mp r; mp_sqrt(&r, &bm);
    cmp_t ph; mp_div(&ph.re, &col[best].re, &r); mp_div(&ph.im, &col[best].im, &r);   /* unit phase */
    for (int i = 0; i < n; ++i) { cmp_t u; cmp_mul_conj(&u, &ph, &col[i]); col[i] = u; }
    mp_zero(&col[best].im);
  }
}

/* A: n x n column-major complex, w words per real.  lam_out: n x w_out words (descending).
 * V_out (may be NULL): column c = eigenvector of lam_out[c], w_out words per real.
 * Returns 0 on success, 1 if A is not exactly Hermitian, 2 if not converged, 3 on allocation failure. */
int oracle_eigh(int n, const double* A, int w, int w_out, double* lam_out, double* V_out, int* sweeps_out) {
  cmp_t* a = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)n * n);
  cmp_t* v = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)n * n);
  cmp_t* vs = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)n * n);
  mp* lam = (mp*)malloc(sizeof(mp) * n);
  int* order = (int*)malloc(sizeof(int) * n);
  if (!a || !v || !vs || !lam || !order) return 3;
  for (size_t k = 0; k < (size_t)n * n; ++k) load_c(&a[k], A, k, w);
  for (int i = 0; i < n; ++i) for (int j = 0; j <= i; ++j) {
    cmp_t c; cmp_conj(&c, &a[IDX(j, i, n)]);
    if (mp_cmp(&c.re, &a[IDX(i, j, n)].re) != 0 || mp_cmp(&c.im, &a[IDX(i, j, n)].im) != 0) {
      free(a); free(v); free(vs); free(lam); free(order); return 1;
    }
  }
  int sw = oracle_jacobi_mp(n, a, v, 80);
  if (sweeps_out) *sweeps_out = sw;
  int rc = 0;
  if (sw < 0) rc = 2;
  else {
    oracle_finish_mp(n, a, v, lam, order);
    for (int i = 0; i < n; ++i) mp_to_words(&lam[i], lam_out + (size_t)i * w_out, w_out);
    if (V_out)
      for (int c = 0; c < n; ++c) for (int i = 0; i < n; ++i)
        store_c(&v[IDX(i, order[c], n)], V_out, IDX(i, c, n), w_out);
  }
  free(a); free(v); free(vs); free(lam); free(order);
  return rc;
}

/* max_i ||A v_i - lam_i v_i||_2 and max |(V^H V - I)_ij| for given (lam, V) of any word counts,
 * evaluated at 320 bits.  cols: evaluate only these column indices (ncols of them), or all if NULL. */
int oracle_residual(int n, const double* A, int w, const double* lam, const double* V, int wv,
                    int ncols, const int* cols, double* res_out, double* orth_out) {
  cmp_t* a = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)n * n);
  cmp_t* vv = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)n * n);
  if (!a || !vv) return 3;
  for (size_t k = 0; k < (size_t)n * n; ++k) { load_c(&a[k], A, k, w); load_c(&vv[k], V, k, wv); }
  int nc = cols ? ncols : n;
  for (int ci = 0; ci < nc; ++ci) {
    int c = cols ? cols[ci] : ci;
    mp l; mp_from_words(&l, lam + (size_t)c * wv, wv);
    mp acc; mp_zero(&acc);
    for (int i = 0; i < n; ++i) {
      cmp_t s, t; cmp_zero(&s);
      for (int k = 0; k < n; ++k) { cmp_mul(&t, &a[IDX(i, k, n)], &vv[IDX(k, c, n)]); cmp_add(&s, &s, &t); }
      cmp_scale(&t, &vv[IDX(i, c, n)], &l); cmp_sub(&s, &s, &t);
      mp m2; cmp_abs2(&m2, &s); mp_add(&acc, &acc, &m2);
    }
    mp_sqrt(&acc, &acc);
    res_out[ci] = mp_to_double(&acc);
    if (orth_out) {
      mp worst; mp_zero(&worst);
      for (int d = 0; d < n; ++d) {
        cmp_t s, t; cmp_zero(&s);
        for (int i = 0; i < n; ++i) { cmp_mul_conj(&t, &vv[IDX(i, d, n)], &vv[IDX(i, c, n)]); cmp_add(&s, &s, &t); }
        if (d == c) { mp one; mp_from_double(&one, 1.0); mp_sub(&s.re, &s.re, &one); }
        mp m2; cmp_abs2(&m2, &s); if (mp_cmp(&m2, &worst) > 0) worst = m2;
      }
      mp_sqrt(&worst, &worst);
      orth_out[ci] = mp_to_double(&worst);
    }
  }
  free(a); free(vv);
  return 0;
}
