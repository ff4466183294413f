/*
 * ORACLE (test infrastructure only).  Singular value decomposition of a complex m x n matrix at 320 bits by
 * one-sided (Hestenes) Jacobi: the plain definition of the SVD variant of the gate update, where the
 * Schmidt decomposition of the reshaped two-site tensor M is taken from M directly instead of from the
 * Gram matrix M M^H (which squares its condition number).
 *
 * For each column pair (p, q) with alpha = |a_p|^2, beta = |a_q|^2, g = a_p^H a_q = |g| e^{i phi}: if |g| is
 * above 2^-300 sqrt(alpha beta) and above 2^-620 ||M||_F^2, the rotation that diagonalises the 2 x 2 Gram block [[alpha, g], [conj(g),
 * beta]] is applied to the columns and accumulated in V:
 *   tau = (beta - alpha) / (2|g|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)) (t = 1 if tau = 0),
 *   c = 1 / sqrt(1 + t^2), s = t c, J = [[c, s e^{i phi}], [-s e^{-i phi}, c]],  [a_p a_q] <- [a_p a_q] J.
 * Sweeps visit p < q in row order until one makes no rotation.  Then sigma_j = |a_j|, u_j = a_j / sigma_j
 * (zero when sigma_j <= 2^-300 max sigma), sorted by descending sigma (ties keep the column order).
 */
#include "mp.h"
#include <stdlib.h>

#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* The one-sided Jacobi on an mp matrix: a (m x n, overwritten by A V), v (n x n, out: V), sg (n, out:
 * column norms sigma_j), order (n, out: column indices by descending sigma, ties in column order).
 * Returns 0, or 2 if 80 sweeps did not converge. */
int oracle_svd_mp(int m, int n, cmp_t* a, cmp_t* v, mp* sg, int* order) {
  for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) {
    cmp_zero(&v[IX(i, j, n)]);
    if (i == j) mp_from_double(&v[IX(i, j, n)].re, 1.0);
  }
  mp one; mp_from_double(&one, 1.0);
  /* absolute floor 2^-620 ||M||_F^2 for |g|: columns that rank deficiency reduces to rounding noise
   * (entries ~2^-320 ||M||) are left alone instead of being rotated against each other forever */
  mp floor_g, t0; mp_zero(&floor_g);
  for (size_t e = 0; e < (size_t)m * n; ++e) { cmp_abs2(&t0, &a[e]); mp_add(&floor_g, &floor_g, &t0); }
  mp_ldexp(&floor_g, &floor_g, -620);
  int rc = 2;
  for (int sweep = 0; sweep < 80; ++sweep) {
    int rotations = 0;
    for (int p = 0; p < n - 1; ++p) for (int q = p + 1; q < n; ++q) {
      mp al, be, t1; cmp_t g, t; mp_zero(&al); mp_zero(&be); cmp_zero(&g);
      for (int i = 0; i < m; ++i) {
        cmp_abs2(&t1, &a[IX(i, p, m)]); mp_add(&al, &al, &t1);
        cmp_abs2(&t1, &a[IX(i, q, m)]); mp_add(&be, &be, &t1);
        cmp_mul_conj(&t, &a[IX(i, p, m)], &a[IX(i, q, m)]); cmp_add(&g, &g, &t);
      }
      mp absg, lim; cmp_abs2(&absg, &g); mp_sqrt(&absg, &absg);
      mp_mul(&lim, &al, &be); mp_sqrt(&lim, &lim); mp_ldexp(&lim, &lim, -300);
      if (mp_is_zero(&absg) || mp_cmp(&absg, &lim) <= 0 || mp_cmp(&absg, &floor_g) <= 0) continue;
      ++rotations;
      cmp_t ephi; mp_div(&ephi.re, &g.re, &absg); mp_div(&ephi.im, &g.im, &absg);
      mp tau, tt, c, s, num, den;
      mp_sub(&num, &be, &al); mp_ldexp(&den, &absg, 1); mp_div(&tau, &num, &den);
      if (mp_is_zero(&tau)) tt = one;
      else {
        mp at, r; mp_abs(&at, &tau);
        mp_mul(&r, &tau, &tau); mp_add(&r, &r, &one); mp_sqrt(&r, &r); mp_add(&r, &r, &at); mp_div(&tt, &one, &r);
        if (mp_sign(&tau) < 0) mp_neg(&tt, &tt);
      }
      mp_mul(&c, &tt, &tt); mp_add(&c, &c, &one); mp_sqrt(&c, &c); mp_div(&c, &one, &c);
      mp_mul(&s, &tt, &c);
      cmp_t z1, z2;                                   /* z2 = s e^{i phi}, z1 = s e^{-i phi} */
      mp_mul(&z2.re, &s, &ephi.re); mp_mul(&z2.im, &s, &ephi.im);
      z1.re = z2.re; mp_neg(&z1.im, &z2.im);
      for (int pass = 0; pass < 2; ++pass) {          /* columns of A (m rows), then of V (n rows) */
        cmp_t* x = pass == 0 ? a : v;
        const int rows = pass == 0 ? m : n;
        for (int i = 0; i < rows; ++i) {
          cmp_t xp = x[IX(i, p, rows)], xq = x[IX(i, q, rows)], u1, u2, np_, nq;
          cmp_scale(&u1, &xp, &c); cmp_mul(&u2, &z1, &xq); cmp_sub(&np_, &u1, &u2);   /* c x_p - z1 x_q */
          cmp_mul(&u1, &z2, &xp); cmp_scale(&u2, &xq, &c); cmp_add(&nq, &u1, &u2);    /* z2 x_p + c x_q */
          x[IX(i, p, rows)] = np_; x[IX(i, q, rows)] = nq;
        }
      }
    }
    if (rotations == 0) { rc = 0; break; }
  }
  if (rc == 0) {
    for (int j = 0; j < n; ++j) {
      mp acc, t1; mp_zero(&acc);
      for (int i = 0; i < m; ++i) { cmp_abs2(&t1, &a[IX(i, j, m)]); mp_add(&acc, &acc, &t1); }
      mp_sqrt(&sg[j], &acc);
    }
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 1; i < n; ++i) {                     /* stable insertion sort, descending */
      int k = order[i], j = i - 1;
      while (j >= 0 && mp_cmp(&sg[order[j]], &sg[k]) < 0) { order[j + 1] = order[j]; --j; }
      order[j + 1] = k;
    }
  }
  return rc;
}

/* M: m x n column-major complex, w words per real.  sigma_out: n values (w_out words, descending);
 * U_out (m x n) and V_out (n x n), column-major complex, w_out words.  Returns 0, 1 on bad arguments,
 * 2 if 80 sweeps did not converge. */
int oracle_svd(int m, int n, const double* M, int w, int w_out, double* sigma_out, double* U_out, double* V_out) {
  if (m < 1 || n < 1 || w < 1) return 1;
  cmp_t* a = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)m * n);
  cmp_t* v = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)n * n);
  mp* sg = (mp*)malloc(sizeof(mp) * n);
  int* order = (int*)malloc(sizeof(int) * n);
  for (size_t e = 0; e < (size_t)m * n; ++e) {
    mp_from_words(&a[e].re, M + (e * 2 + 0) * w, w);
    mp_from_words(&a[e].im, M + (e * 2 + 1) * w, w);
  }
  int rc = oracle_svd_mp(m, n, a, v, sg, order);
  if (rc == 0) {
    mp smax = sg[order[0]];
    mp floor_; mp_ldexp(&floor_, &smax, -300);
    for (int c = 0; c < n; ++c) {
      const int j = order[c];
      mp_to_words(&sg[j], sigma_out + (size_t)c * w_out, w_out);
      const int keep = mp_cmp(&sg[j], &floor_) > 0;
      for (int i = 0; i < m; ++i) {
        cmp_t u;
        if (keep) { mp_div(&u.re, &a[IX(i, j, m)].re, &sg[j]); mp_div(&u.im, &a[IX(i, j, m)].im, &sg[j]); }
        else cmp_zero(&u);
        const size_t e = IX(i, c, m);
        mp_to_words(&u.re, U_out + (e * 2 + 0) * w_out, w_out);
        mp_to_words(&u.im, U_out + (e * 2 + 1) * w_out, w_out);
      }
      for (int i = 0; i < n; ++i) {
        const size_t e = IX(i, c, n);
        mp_to_words(&v[IX(i, j, n)].re, V_out + (e * 2 + 0) * w_out, w_out);
        mp_to_words(&v[IX(i, j, n)].im, V_out + (e * 2 + 1) * w_out, w_out);
      }
    }
  }
  free(a); free(v); free(sg); free(order);
  return rc;
}
