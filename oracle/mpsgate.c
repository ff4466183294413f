/*
 * ORACLE (test infrastructure only).  One two-site gate update of a Vidal MPS at 320 bits, the plain
 * definition of the MPS step of the paper (Section 2: a two-qubit gate is applied to the two-site tensor
 * and the result split back by a Schmidt decomposition; Section 1: the MPS stays a nested Schmidt
 * decomposition).  For the gate G on sites (l, l+1), with bond dimensions a = chi[l-1], c = chi[l],
 * d = chi[l+1] (1 at the ends) and weights lamL = lam[l-1], lamC = lam[l], lamR = lam[l+1] (1 at the
 * ends):
 *   theta^{ij}_{alpha gamma} = sum over k, m, beta of G_{(i j),(k m)} lamL_alpha Gamma[l]^k_{alpha beta}
 *                              lamC_beta Gamma[l+1]^m_{beta gamma} lamR_gamma,
 *   M[(i, alpha)][(j, gamma)] = theta^{ij}_{alpha gamma}   (2a x 2d),
 *   M = U diag(sigma) V^H by one-sided Jacobi (svd.c) on M itself, so small sigma keep full relative
 *     accuracy,
 *   keep the sigma_beta with sigma_beta^2 > 2^-tol_log2 sum sigma^2, at most r_max of them (at least one),
 *   lam'_beta = sigma_beta / sqrt(sum of the kept sigma^2),
 *   Gamma'[l]^i_{alpha beta} = U[(i, alpha)][beta] / lamL_alpha,
 *   Gamma'[l+1]^j_{beta gamma} = conj(V[(j, gamma)][beta]) / lamR_gamma.
 * The layout is that of oracle_mps_amplitudes (Gamma (s, alpha, beta) row-major, w words).
 */
#include "mp.h"
#include <stdlib.h>
#include <string.h>

int oracle_svd_mp(int m, int n, cmp_t* a, cmp_t* v, mp* sg, int* order);

static void ld(cmp_t* z, const double* p, size_t e, int w) {
  mp_from_words(&z->re, p + (e * 2 + 0) * w, w);
  mp_from_words(&z->im, p + (e * 2 + 1) * w, w);
}
static void st(const cmp_t* z, double* p, size_t e, int w) {
  mp_to_words(&z->re, p + (e * 2 + 0) * w, w);
  mp_to_words(&z->im, p + (e * 2 + 1) * w, w);
}

/* Returns 0, 1 on bad arguments, 2 if the SVD did not converge.  chi_out, gam_out, lam_out receive the
 * whole updated MPS (the caller sizes them for the bond dimension min(2a, 2d, r_max) at bond l);
 * *discarded receives the dropped sum sigma^2 over the total (rounded to double). */
int oracle_mps_apply2(int n, const int* chi, const double* gam, const double* lam, int w, int site,
                      const double* G, int wg, int tol_log2, int r_max, int* chi_out, double* gam_out,
                      double* lam_out, int w_out, double* discarded) {
  if (n < 2 || site < 0 || site + 1 >= n || w < 1 || wg < 1 || r_max < 1) return 1;
  const int l = site;
  const int a = l == 0 ? 1 : chi[l - 1], c = chi[l], d = l + 1 == n - 1 ? 1 : chi[l + 1];
  /* offsets of the tensors and weights in the packed input */
  size_t go[2] = {0, 0}, gsz = 0;
  {
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
      const int cl = k == 0 ? 1 : chi[k - 1], cr = k == n - 1 ? 1 : chi[k];
      if (k == l) go[0] = off;
      if (k == l + 1) go[1] = off;
      off += (size_t)2 * cl * cr;
    }
    gsz = off;
  }
  size_t lo[3] = {0, 0, 0}, lsz = 0;                  /* lam[l-1], lam[l], lam[l+1] */
  for (int k = 0; k < n - 1; ++k) {
    if (k == l - 1) lo[0] = lsz;
    if (k == l) lo[1] = lsz;
    if (k == l + 1) lo[2] = lsz;
    lsz += chi[k];
  }
  mp* wl = (mp*)malloc(sizeof(mp) * a);
  mp* wc = (mp*)malloc(sizeof(mp) * c);
  mp* wr = (mp*)malloc(sizeof(mp) * d);
  for (int k = 0; k < a; ++k) { if (l == 0) mp_from_double(&wl[k], 1.0); else mp_from_words(&wl[k], lam + (lo[0] + k) * w, w); }
  for (int k = 0; k < c; ++k) mp_from_words(&wc[k], lam + (lo[1] + k) * w, w);
  for (int k = 0; k < d; ++k) { if (l + 1 == n - 1) mp_from_double(&wr[k], 1.0); else mp_from_words(&wr[k], lam + (lo[2] + k) * w, w); }
  cmp_t g[16];
  for (int e = 0; e < 16; ++e) ld(&g[e], G, (size_t)e, wg);
  /* T^{km}_{alpha gamma} = lamL_alpha sum_beta Gamma[l]^k_{alpha beta} lamC_beta Gamma[l+1]^m_{beta gamma} lamR_gamma */
  const int R = 2 * a, C = 2 * d;
  cmp_t* T = (cmp_t*)malloc(sizeof(cmp_t) * 4 * (size_t)a * d);
  for (int k = 0; k < 2; ++k) for (int m = 0; m < 2; ++m) for (int al = 0; al < a; ++al) for (int ga = 0; ga < d; ++ga) {
    cmp_t acc, x, y, u; cmp_zero(&acc);
    for (int be = 0; be < c; ++be) {
      ld(&x, gam, go[0] + ((size_t)k * a + al) * c + be, w);
      ld(&y, gam, go[1] + ((size_t)m * c + be) * d + ga, w);
      cmp_scale(&x, &x, &wc[be]);
      cmp_mul(&u, &x, &y); cmp_add(&acc, &acc, &u);
    }
    mp s; mp_mul(&s, &wl[al], &wr[ga]);
    cmp_scale(&acc, &acc, &s);
    T[(((size_t)k * 2 + m) * a + al) * d + ga] = acc;
  }
  /* M[(i, alpha)][(j, gamma)] = sum over k, m of G_{(i j),(k m)} T^{km}_{alpha gamma}; column-major R x C */
  cmp_t* M = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)R * C);
  for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) for (int al = 0; al < a; ++al) for (int ga = 0; ga < d; ++ga) {
    cmp_t acc, u; cmp_zero(&acc);
    for (int km = 0; km < 4; ++km) {
      cmp_mul(&u, &g[(i * 2 + j) * 4 + km], &T[(((size_t)km) * a + al) * d + ga]);
      cmp_add(&acc, &acc, &u);
    }
    M[(size_t)(i * a + al) + (size_t)(j * d + ga) * R] = acc;
  }
  /* SVD: one-sided Jacobi on the columns of M (R x C): M V = [sigma_j u_j] */
  cmp_t* Vm = (cmp_t*)malloc(sizeof(cmp_t) * (size_t)C * C);
  mp* sg = (mp*)malloc(sizeof(mp) * C);
  int* order = (int*)malloc(sizeof(int) * C);
  int rc = oracle_svd_mp(R, C, M, Vm, sg, order);
  if (rc == 0) {
    mp tot; mp_zero(&tot);
    for (int k = 0; k < C; ++k) { mp t; mp_mul(&t, &sg[k], &sg[k]); mp_add(&tot, &tot, &t); }
    mp thr; mp_ldexp(&thr, &tot, -tol_log2);
    int keep = 0;
    const int cap = R < C ? R : C;
    while (keep < cap && keep < r_max) {
      mp t; mp_mul(&t, &sg[order[keep]], &sg[order[keep]]);
      if (mp_cmp(&t, &thr) <= 0) break;
      ++keep;
    }
    if (keep == 0) keep = 1;
    mp kept; mp_zero(&kept);
    for (int k = 0; k < keep; ++k) { mp t; mp_mul(&t, &sg[order[k]], &sg[order[k]]); mp_add(&kept, &kept, &t); }
    if (discarded) {
      mp dd; mp_sub(&dd, &tot, &kept); mp_div(&dd, &dd, &tot);
      *discarded = mp_to_double(&dd);
    }
    mp nrm; mp_sqrt(&nrm, &kept);
    /* the new MPS: copy every other tensor and weight, replace sites l, l+1 and bond l */
    for (int k = 0; k < n - 1; ++k) chi_out[k] = k == l ? keep : chi[k];
    size_t oo = 0, ol = 0;
    for (int k = 0; k < n; ++k) {
      const int cl = k == 0 ? 1 : chi_out[k - 1], cr = k == n - 1 ? 1 : chi_out[k];
      if (k == l) {
        for (int s = 0; s < 2; ++s) for (int al = 0; al < a; ++al) for (int be = 0; be < keep; ++be) {
          const int j = order[be];
          cmp_t u; mp inv;                               /* U[(s, al)][be] = (M V)[(s,al)][j] / sigma_j */
          mp_mul(&inv, &sg[j], &wl[al]);
          mp_div(&u.re, &M[(size_t)(s * a + al) + (size_t)j * R].re, &inv);
          mp_div(&u.im, &M[(size_t)(s * a + al) + (size_t)j * R].im, &inv);
          st(&u, gam_out, oo + ((size_t)s * a + al) * keep + be, w_out);
        }
      } else if (k == l + 1) {
        for (int s = 0; s < 2; ++s) for (int be = 0; be < keep; ++be) for (int ga = 0; ga < d; ++ga) {
          const int j = order[be];
          cmp_t u; cmp_conj(&u, &Vm[(size_t)(s * d + ga) + (size_t)j * C]);
          mp_div(&u.re, &u.re, &wr[ga]); mp_div(&u.im, &u.im, &wr[ga]);
          st(&u, gam_out, oo + ((size_t)s * keep + be) * d + ga, w_out);
        }
      } else {
        size_t ii = 0;                                   /* the same tensor in the input */
        for (int q = 0; q < k; ++q) { const int ql = q == 0 ? 1 : chi[q - 1], qr = q == n - 1 ? 1 : chi[q]; ii += (size_t)2 * ql * qr; }
        for (size_t e = 0; e < (size_t)2 * cl * cr; ++e) { cmp_t u; ld(&u, gam, ii + e, w); st(&u, gam_out, oo + e, w_out); }
      }
      oo += (size_t)2 * cl * cr;
      if (k < n - 1) {
        if (k == l) {
          for (int be = 0; be < keep; ++be) { mp t; mp_div(&t, &sg[order[be]], &nrm); mp_to_words(&t, lam_out + (ol + be) * w_out, w_out); }
        } else {
          size_t il = 0; for (int q = 0; q < k; ++q) il += chi[q];
          for (int be = 0; be < chi[k]; ++be) { mp t; mp_from_words(&t, lam + (il + be) * w, w); mp_to_words(&t, lam_out + (ol + be) * w_out, w_out); }
        }
        ol += chi_out[k];
      }
    }
  }
  (void)gsz;
  free(wl); free(wc); free(wr); free(T); free(M); free(Vm); free(sg); free(order);
  return rc;
}

/* Sampling a bit string from a Vidal MPS in canonical form, by the chain rule of its Born probabilities:
 * with the left vector l^(k)_beta = (Gamma[0]^{s_0} lam[0] Gamma[1]^{s_1} ... lam[k-1] Gamma[k]^{s_k})_beta, the
 * marginal of the prefix s_0..s_k is p = sum over beta of |l^(k)_beta|^2 lam[k]_beta^2 (lam[n-1] = 1), because the
 * sites to the right are orthonormal in the weights.  Site k takes s_k = 1 when u[k] >= p(prefix, 0) /
 * p(prefix) (inverse CDF with the uniform numbers u passed in), else 0.  bits receives the string, prob the
 * probability of the whole string (w_out words).  Returns 0, or 1 on bad arguments. */
int oracle_mps_sample(int n, const int* chi, const double* gam, const double* lam, int w, const double* u,
                      int* bits, double* prob, int w_out) {
  if (n < 1 || w < 1) return 1;
  int maxc = 1;
  for (int k = 0; k < n - 1; ++k) if (chi[k] > maxc) maxc = chi[k];
  cmp_t* lv = (cmp_t*)malloc(sizeof(cmp_t) * maxc);
  cmp_t* nv[2];
  nv[0] = (cmp_t*)malloc(sizeof(cmp_t) * maxc);
  nv[1] = (cmp_t*)malloc(sizeof(cmp_t) * maxc);
  cmp_zero(&lv[0]); mp_from_double(&lv[0].re, 1.0);      /* the empty prefix */
  mp pprev; mp_from_double(&pprev, 1.0);
  size_t go = 0, lo = 0;
  for (int k = 0; k < n; ++k) {
    const int a = k == 0 ? 1 : chi[k - 1], b = k == n - 1 ? 1 : chi[k];
    mp pk[2];
    for (int s = 0; s < 2; ++s) {
      mp_zero(&pk[s]);
      for (int be = 0; be < b; ++be) {
        cmp_t acc, x, t; cmp_zero(&acc);
        for (int al = 0; al < a; ++al) {
          ld(&x, gam, go + ((size_t)s * a + al) * b + be, w);
          cmp_mul(&t, &lv[al], &x); cmp_add(&acc, &acc, &t);
        }
        nv[s][be] = acc;
        mp m2, wt; cmp_abs2(&m2, &acc);
        if (k < n - 1) { mp_from_words(&wt, lam + (lo + be) * w, w); mp_mul(&wt, &wt, &wt); mp_mul(&m2, &m2, &wt); }
        mp_add(&pk[s], &pk[s], &m2);
      }
    }
    mp thr, uu; mp_div(&thr, &pk[0], &pprev); mp_from_double(&uu, u[k]);
    const int s = mp_cmp(&uu, &thr) >= 0 ? 1 : 0;
    bits[k] = s;
    pprev = pk[s];
    /* carry the chosen branch, weighted by lam[k] for the next site */
    for (int be = 0; be < b; ++be) {
      lv[be] = nv[s][be];
      if (k < n - 1) { mp wt; mp_from_words(&wt, lam + (lo + be) * w, w); cmp_scale(&lv[be], &lv[be], &wt); }
    }
    go += (size_t)2 * a * b;
    if (k < n - 1) lo += chi[k];
  }
  mp_to_words(&pprev, prob, w_out);
  free(lv); free(nv[0]); free(nv[1]);
  return 0;
}
