/*
 * ORACLE (test infrastructure only).  Brute-force statevector simulator in 320-bit arithmetic, the plain
 * definition of what an MPS simulation of a circuit computes (Section 1: the MPS is a nested Schmidt
 * decomposition whose time evolution must equal that of the state vector).
 *
 * Basis index x = sum_l s_l 2^(n-1-l): site 0 is the most significant bit.  A two-qubit gate G on
 * (site, site+1) is a 4x4 matrix, row-major, whose row/column index is 2 i + j with i the bit of `site`
 * and j the bit of `site+1`.
 */
#include "mp.h"
#include <stdlib.h>
#include <string.h>

typedef struct { int n; size_t dim; cmp_t* psi; } sv_t;

void* oracle_sv_new(int n) {
  if (n < 1 || n > 24) return NULL;
  sv_t* h = (sv_t*)malloc(sizeof(sv_t));
  h->n = n; h->dim = (size_t)1 << n;
  h->psi = (cmp_t*)malloc(sizeof(cmp_t) * h->dim);
  for (size_t x = 0; x < h->dim; ++x) cmp_zero(&h->psi[x]);
  mp_from_double(&h->psi[0].re, 1.0);
  return h;
}
void oracle_sv_free(void* hv) { sv_t* h = (sv_t*)hv; if (h) { free(h->psi); free(h); } }

/* set amplitudes from words (dim x 2 x w) */
void oracle_sv_set(void* hv, const double* amps, int w) {
  sv_t* h = (sv_t*)hv;
  for (size_t x = 0; x < h->dim; ++x) {
    mp_from_words(&h->psi[x].re, amps + (x * 2 + 0) * w, w);
    mp_from_words(&h->psi[x].im, amps + (x * 2 + 1) * w, w);
  }
}
void oracle_sv_get(void* hv, double* amps, int w) {
  sv_t* h = (sv_t*)hv;
  for (size_t x = 0; x < h->dim; ++x) {
    mp_to_words(&h->psi[x].re, amps + (x * 2 + 0) * w, w);
    mp_to_words(&h->psi[x].im, amps + (x * 2 + 1) * w, w);
  }
}

static void load_mat(cmp_t* g, const double* G, int dim, int w) {
  for (int k = 0; k < dim * dim; ++k) {
    mp_from_words(&g[k].re, G + ((size_t)k * 2 + 0) * w, w);
    mp_from_words(&g[k].im, G + ((size_t)k * 2 + 1) * w, w);
  }
}

int oracle_sv_apply1(void* hv, int site, const double* U, int w) {
  sv_t* h = (sv_t*)hv;
  if (site < 0 || site >= h->n) return 1;
  cmp_t g[4]; load_mat(g, U, 2, w);
  size_t bit = (size_t)1 << (h->n - 1 - site);
  for (size_t x = 0; x < h->dim; ++x) {
    if (x & bit) continue;
    cmp_t a0 = h->psi[x], a1 = h->psi[x | bit], t, r0, r1;
    cmp_mul(&r0, &g[0], &a0); cmp_mul(&t, &g[1], &a1); cmp_add(&r0, &r0, &t);
    cmp_mul(&r1, &g[2], &a0); cmp_mul(&t, &g[3], &a1); cmp_add(&r1, &r1, &t);
    h->psi[x] = r0; h->psi[x | bit] = r1;
  }
  return 0;
}

int oracle_sv_apply2(void* hv, int site, const double* G, int w) {
  sv_t* h = (sv_t*)hv;
  if (site < 0 || site + 1 >= h->n) return 1;
  cmp_t g[16]; load_mat(g, G, 4, w);
  size_t bi = (size_t)1 << (h->n - 1 - site), bj = (size_t)1 << (h->n - 2 - site);
  for (size_t x = 0; x < h->dim; ++x) {
    if (x & (bi | bj)) continue;
    size_t idx[4] = {x, x | bj, x | bi, x | bi | bj};     /* index 2i + j */
    cmp_t in[4], out[4], t;
    for (int r = 0; r < 4; ++r) in[r] = h->psi[idx[r]];
    for (int r = 0; r < 4; ++r) {
      cmp_zero(&out[r]);
      for (int c = 0; c < 4; ++c) { cmp_mul(&t, &g[r * 4 + c], &in[c]); cmp_add(&out[r], &out[r], &t); }
    }
    for (int r = 0; r < 4; ++r) h->psi[idx[r]] = out[r];
  }
  return 0;
}

/* multi-controlled single-qubit gate: U on `target` when every site l != target has bit ctrl[l]
 * (ctrl[l] = -1: not a control) */
int oracle_sv_apply_mcu(void* hv, int target, const int* ctrl, const double* U, int w) {
  sv_t* h = (sv_t*)hv;
  cmp_t g[4]; load_mat(g, U, 2, w);
  size_t tb = (size_t)1 << (h->n - 1 - target);
  for (size_t x = 0; x < h->dim; ++x) {
    if (x & tb) continue;
    int ok = 1;
    for (int l = 0; l < h->n && ok; ++l) {
      if (l == target || ctrl[l] < 0) continue;
      int bit = (int)((x >> (h->n - 1 - l)) & 1);
      ok = bit == ctrl[l];
    }
    if (!ok) continue;
    cmp_t a0 = h->psi[x], a1 = h->psi[x | tb], t, r0, r1;
    cmp_mul(&r0, &g[0], &a0); cmp_mul(&t, &g[1], &a1); cmp_add(&r0, &r0, &t);
    cmp_mul(&r1, &g[2], &a0); cmp_mul(&t, &g[3], &a1); cmp_add(&r1, &r1, &t);
    h->psi[x] = r0; h->psi[x | tb] = r1;
  }
  return 0;
}

void oracle_sv_norm2(void* hv, double* out, int w) {
  sv_t* h = (sv_t*)hv;
  mp acc, t; mp_zero(&acc);
  for (size_t x = 0; x < h->dim; ++x) { cmp_abs2(&t, &h->psi[x]); mp_add(&acc, &acc, &t); }
  mp_to_words(&acc, out, w);
}

int oracle_jacobi_mp(int n, cmp_t* a, cmp_t* v, int max_sweeps);
void oracle_finish_mp(int n, const cmp_t* a, cmp_t* v, mp* lam, int* order);

/* squared Schmidt coefficients across the cut between sites cut-1 and cut (1 <= cut <= n-1):
 * eigenvalues (descending) of the Gram matrix of the smaller side; writes min(2^cut, 2^(n-cut)) values */
int oracle_sv_schmidt2(void* hv, int cut, double* out, int w) {
  sv_t* h = (sv_t*)hv;
  if (cut < 1 || cut >= h->n) return 1;
  size_t L = (size_t)1 << cut, R = (size_t)1 << (h->n - cut);
  int left_small = L <= R;
  size_t m = left_small ? L : R;
  cmp_t* g = (cmp_t*)malloc(sizeof(cmp_t) * m * m);
  cmp_t* v = (cmp_t*)malloc(sizeof(cmp_t) * m * m);
  mp* lam = (mp*)malloc(sizeof(mp) * m);
  int* order = (int*)malloc(sizeof(int) * m);
  /* psi[x] with x = l * R + r;  left Gram: G_ab = sum_r psi[a,r] conj(psi[b,r]) */
  for (size_t a = 0; a < m; ++a) for (size_t b = 0; b < m; ++b) {
    cmp_t s, t; cmp_zero(&s);
    if (left_small) for (size_t r = 0; r < R; ++r) { cmp_mul_conj(&t, &h->psi[b * R + r], &h->psi[a * R + r]); cmp_add(&s, &s, &t); }
    else for (size_t l = 0; l < L; ++l) { cmp_mul_conj(&t, &h->psi[l * R + b], &h->psi[l * R + a]); cmp_add(&s, &s, &t); }
    g[a + b * m] = s;
  }
  int sw = oracle_jacobi_mp((int)m, g, v, 80);
  if (sw < 0) { free(g); free(v); free(lam); free(order); return 2; }
  oracle_finish_mp((int)m, g, v, lam, order);
  for (size_t i = 0; i < m; ++i) mp_to_words(&lam[i], out + i * w, w);
  free(g); free(v); free(lam); free(order);
  return 0;
}

/* Amplitudes of a Vidal MPS: psi(s_0..s_{n-1}) = Gamma[0]^{s_0} lam[0] Gamma[1]^{s_1} lam[1] ... Gamma[n-1]^{s_{n-1}}.
 * chi[l] = bond dimension between sites l and l+1 (l = 0..n-2).  Gamma[l] is stored row-major in
 * (s, alpha, beta) with alpha < chi[l-1] (1 for l = 0) and beta < chi[l] (1 for l = n-1), complex with
 * w words per real, concatenated over l; lam[l] (w words per value) concatenated over l.
 * amps: 2^n x 2 x w_out words. */
int oracle_mps_amplitudes(int n, const int* chi, const double* gam, const double* lam, int w,
                          double* amps, int w_out) {
  if (n < 1 || n > 22) return 1;
  size_t goff = 0, loff = 0;
  /* T: current partial contraction, rows = 2^l prefixes, cols = chi[l] */
  size_t rows = 1; int cols = 1;
  cmp_t* T = (cmp_t*)malloc(sizeof(cmp_t)); cmp_zero(&T[0]); mp_from_double(&T[0].re, 1.0);
  for (int l = 0; l < n; ++l) {
    int cl = l == 0 ? 1 : chi[l - 1], cr = l == n - 1 ? 1 : chi[l];
    if (cl != cols) { free(T); return 2; }
    mp* lw = NULL;
    if (l > 0) {                                        /* weights lam[l-1] on the left index */
      lw = (mp*)malloc(sizeof(mp) * cl);
      for (int a = 0; a < cl; ++a) mp_from_words(&lw[a], lam + (loff + a) * w, w);
      loff += cl;
    }
    cmp_t* Tn = (cmp_t*)malloc(sizeof(cmp_t) * rows * 2 * cr);
    for (size_t x = 0; x < rows; ++x) for (int s = 0; s < 2; ++s) for (int b = 0; b < cr; ++b) {
      cmp_t acc, g, t, u; cmp_zero(&acc);
      for (int a = 0; a < cl; ++a) {
        size_t gi = goff + ((size_t)s * cl + a) * cr + b;
        mp_from_words(&g.re, gam + (gi * 2 + 0) * w, w);
        mp_from_words(&g.im, gam + (gi * 2 + 1) * w, w);
        u = T[x * cl + a];
        if (lw) cmp_scale(&u, &u, &lw[a]);
        cmp_mul(&t, &u, &g); cmp_add(&acc, &acc, &t);
      }
      Tn[(x * 2 + s) * cr + b] = acc;
    }
    goff += (size_t)2 * cl * cr;
    free(T); free(lw); T = Tn; rows *= 2; cols = cr;
  }
  for (size_t x = 0; x < rows; ++x) {
    mp_to_words(&T[x].re, amps + (x * 2 + 0) * w_out, w_out);
    mp_to_words(&T[x].im, amps + (x * 2 + 1) * w_out, w_out);
  }
  free(T);
  return 0;
}

/* Canonical conditions of one site of a Vidal MPS (Section 1: the MPS is a nested Schmidt decomposition,
 * so at every bond the tensors on each side are orthonormal once weighted by the squared Schmidt
 * coefficients).  Gamma is (s, alpha, beta) row-major with alpha < a, beta < b, complex, w words per real;
 * lamL holds a weights and lamR b weights (NULL: all 1).
 *   side 0: G[beta][beta'] = sum over s, alpha of lamL_alpha^2 conj(Gamma^s[alpha][beta]) Gamma^s[alpha][beta']
 *   side 1: G[alpha][alpha'] = sum over s, beta of lamR_beta^2 Gamma^s[alpha][beta] conj(Gamma^s[alpha'][beta])
 * *defect receives max |G - I| over all entries (320 bits, rounded to double).  Returns 0, or 1 on bad
 * arguments. */
int oracle_mps_site_defect(int a, int b, const double* gam, const double* lamL, const double* lamR, int w, int side,
                           double* defect) {
  if (a < 1 || b < 1 || w < 1 || (side != 0 && side != 1) || !gam || !defect) return 1;
  const size_t ne = (size_t)2 * a * b;
  cmp_t* g = (cmp_t*)malloc(sizeof(cmp_t) * ne);
  mp* wt = (mp*)malloc(sizeof(mp) * (side == 0 ? a : b));
  for (size_t e = 0; e < ne; ++e) {
    mp_from_words(&g[e].re, gam + (e * 2 + 0) * w, w);
    mp_from_words(&g[e].im, gam + (e * 2 + 1) * w, w);
  }
  const double* lw = side == 0 ? lamL : lamR;
  const int nw = side == 0 ? a : b;
  for (int k = 0; k < nw; ++k) {
    if (lw) { mp t; mp_from_words(&t, lw + (size_t)k * w, w); mp_mul(&wt[k], &t, &t); }
    else mp_from_double(&wt[k], 1.0);
  }
  const int d = side == 0 ? b : a;                     /* the Gram matrix is d x d */
  mp worst; mp_zero(&worst);
  mp one; mp_from_double(&one, 1.0);
  for (int p = 0; p < d; ++p)
    for (int q = 0; q < d; ++q) {
      cmp_t acc; cmp_zero(&acc);
      for (int s = 0; s < 2; ++s)
        for (int k = 0; k < nw; ++k) {
          /* side 0: k = alpha, entries (alpha, p) and (alpha, q); side 1: k = beta, entries (q, beta), (p, beta) */
          const cmp_t* x = side == 0 ? &g[((size_t)s * a + k) * b + p] : &g[((size_t)s * a + q) * b + k];
          const cmp_t* y = side == 0 ? &g[((size_t)s * a + k) * b + q] : &g[((size_t)s * a + p) * b + k];
          cmp_t t;
          cmp_mul_conj(&t, x, y);                        /* conj(x) y */
          cmp_scale(&t, &t, &wt[k]);
          cmp_add(&acc, &acc, &t);
        }
      if (p == q) mp_sub(&acc.re, &acc.re, &one);
      mp m2; cmp_abs2(&m2, &acc);
      if (mp_cmp(&m2, &worst) > 0) worst = m2;
    }
  mp r; mp_sqrt(&r, &worst);
  *defect = mp_to_double(&r);
  free(g); free(wt);
  return 0;
}

/* Vidal form of the state (Section 1: the MPS is a nested Schmidt decomposition).  At every cut c = 1..n-1
 * the state is Psi[a][r] = psi[a * 2^(n-c) + r] = sum_k lambda_k u_k[a] v_k[r] with orthonormal u_k, v_k;
 * the Schmidt pairs come from the Jacobi eigensolve of the smaller Gram matrix (Psi Psi^H, eigenvectors
 * u_k; or Psi^H Psi, eigenvectors conj(v_k)), the other vector of each pair from Psi, and only values with
 * lambda_k^2 > 2^-tol_log2 lambda_0^2 are kept.  Then
 *   Gamma[l]^s[alpha][beta] = <u^(l)_alpha (x) s (x) v^(l+1)_beta | psi> / (lambda^(l)_alpha lambda^(l+1)_beta)
 * with u^(0) = v^(n) = (1) and lambda^(0) = lambda^(n) = 1, and lambda[l] = lambda^(l+1).
 * chi[l] (l = 0..n-2) receives the bond dimensions; gam and lam receive the tensors in the layout of
 * oracle_mps_amplitudes (w words), packed.  The caller sizes gam for sum over l of 2 cmax(l) cmax(l+1)
 * complex elements and lam for sum of cmax, cmax(c) = 2^min(c, n-c).  Returns 0, or 1 / 2 on bad
 * arguments / an eigensolve that did not converge. */
int oracle_sv_vidal(void* hv, int tol_log2, int* chi, double* gam, double* lam, int w) {
  sv_t* h = (sv_t*)hv;
  const int n = h->n;
  if (n < 2 || n > 14 || w < 1) return 1;
  cmp_t** U = (cmp_t**)calloc(n + 1, sizeof(cmp_t*));   /* U[c]: 2^c x chi_c, column k = u_k */
  cmp_t** V = (cmp_t**)calloc(n + 1, sizeof(cmp_t*));   /* V[c]: 2^(n-c) x chi_c, column k = v_k */
  mp** L = (mp**)calloc(n + 1, sizeof(mp*));
  int* ch = (int*)calloc(n + 1, sizeof(int));
  int rc = 0;
  ch[0] = ch[n] = 1;
  for (int c = 0; c <= n; c += n) {                     /* the trivial cuts */
    U[c] = (cmp_t*)malloc(sizeof(cmp_t) * (c == 0 ? 1 : h->dim));
    V[c] = (cmp_t*)malloc(sizeof(cmp_t) * (c == 0 ? h->dim : 1));
    L[c] = (mp*)malloc(sizeof(mp));
    mp_from_double(&L[c][0], 1.0);
  }
  cmp_zero(&U[0][0]); mp_from_double(&U[0][0].re, 1.0);
  cmp_zero(&V[n][0]); mp_from_double(&V[n][0].re, 1.0);
  for (int c = 1; c < n && !rc; ++c) {
    const size_t Ld = (size_t)1 << c, Rd = (size_t)1 << (n - c);
    const int left = Ld <= Rd;
    const size_t m = left ? Ld : Rd;
    cmp_t* g = (cmp_t*)malloc(sizeof(cmp_t) * m * m);
    cmp_t* ev = (cmp_t*)malloc(sizeof(cmp_t) * m * m);
    mp* mu = (mp*)malloc(sizeof(mp) * m);
    int* order = (int*)malloc(sizeof(int) * m);
    for (size_t a = 0; a < m; ++a) for (size_t b = 0; b < m; ++b) {
      cmp_t s, t; cmp_zero(&s);
      if (left) for (size_t r = 0; r < Rd; ++r) { cmp_mul_conj(&t, &h->psi[b * Rd + r], &h->psi[a * Rd + r]); cmp_add(&s, &s, &t); }
      else for (size_t l = 0; l < Ld; ++l) { cmp_mul_conj(&t, &h->psi[l * Rd + a], &h->psi[l * Rd + b]); cmp_add(&s, &s, &t); }
      g[a + b * m] = s;                                 /* left: (Psi Psi^H)_ab; right: (Psi^H Psi)_ab */
    }
    if (oracle_jacobi_mp((int)m, g, ev, 80) < 0) rc = 2;
    else {
      oracle_finish_mp((int)m, g, ev, mu, order);
      mp cut; mp_ldexp(&cut, &mu[0], -tol_log2);
      int k = 0;
      while (k < (int)m && mp_cmp(&mu[k], &cut) > 0) ++k;
      if (k == 0) k = 1;
      ch[c] = k;
      U[c] = (cmp_t*)malloc(sizeof(cmp_t) * Ld * k);
      V[c] = (cmp_t*)malloc(sizeof(cmp_t) * Rd * k);
      L[c] = (mp*)malloc(sizeof(mp) * k);
      for (int q = 0; q < k; ++q) {
        mp_sqrt(&L[c][q], &mu[q]);
        const cmp_t* e = ev + (size_t)order[q] * m;     /* eigenvector of mu[q] */
        if (left) {                                       /* u = e; v[r] = sum_a conj(u[a]) Psi[a][r] / lambda */
          for (size_t a = 0; a < Ld; ++a) U[c][a + Ld * q] = e[a];
          for (size_t r = 0; r < Rd; ++r) {
            cmp_t s, t; cmp_zero(&s);
            for (size_t a = 0; a < Ld; ++a) { cmp_mul_conj(&t, &e[a], &h->psi[a * Rd + r]); cmp_add(&s, &s, &t); }
            mp_div(&s.re, &s.re, &L[c][q]); mp_div(&s.im, &s.im, &L[c][q]);
            V[c][r + Rd * q] = s;
          }
        } else {                                          /* v = conj(e); u[a] = sum_r Psi[a][r] e[r] / lambda */
          for (size_t r = 0; r < Rd; ++r) cmp_conj(&V[c][r + Rd * q], &e[r]);
          for (size_t a = 0; a < Ld; ++a) {
            cmp_t s, t; cmp_zero(&s);
            for (size_t r = 0; r < Rd; ++r) { cmp_mul(&t, &h->psi[a * Rd + r], &e[r]); cmp_add(&s, &s, &t); }
            mp_div(&s.re, &s.re, &L[c][q]); mp_div(&s.im, &s.im, &L[c][q]);
            U[c][a + Ld * q] = s;
          }
        }
      }
    }
    free(g); free(ev); free(mu); free(order);
  }
  if (!rc) {
    size_t go = 0, lo = 0;
    for (int l = 0; l < n; ++l) {
      const int ca = ch[l], cb = ch[l + 1];
      const size_t La = (size_t)1 << l, Rb = (size_t)1 << (n - l - 1);
      for (int s = 0; s < 2; ++s) for (int al = 0; al < ca; ++al) for (int be = 0; be < cb; ++be) {
        cmp_t acc, t, u; cmp_zero(&acc);
        for (size_t a = 0; a < La; ++a) for (size_t r = 0; r < Rb; ++r) {
          /* conj(u_alpha[a]) conj(v_beta[r]) psi[(a, s, r)] */
          cmp_mul(&u, &U[l][a + La * al], &V[l + 1][r + Rb * be]);
          cmp_mul_conj(&t, &u, &h->psi[(a * 2 + s) * Rb + r]);
          cmp_add(&acc, &acc, &t);
        }
        mp den; mp_mul(&den, &L[l][al], &L[l + 1][be]);
        mp_div(&acc.re, &acc.re, &den); mp_div(&acc.im, &acc.im, &den);
        const size_t e = go + ((size_t)s * ca + al) * cb + be;
        mp_to_words(&acc.re, gam + (e * 2 + 0) * w, w);
        mp_to_words(&acc.im, gam + (e * 2 + 1) * w, w);
      }
      go += (size_t)2 * ca * cb;
      if (l < n - 1) {
        chi[l] = cb;
        for (int be = 0; be < cb; ++be) mp_to_words(&L[l + 1][be], lam + (lo + be) * w, w);
        lo += cb;
      }
    }
  }
  for (int c = 0; c <= n; ++c) { free(U[c]); free(V[c]); free(L[c]); }
  free(U); free(V); free(L); free(ch);
  return rc;
}

/* Expectation value of a one-qubit operator O (2x2 row-major complex, w words) on `site`:
 * <psi| O_site |psi> = sum over x of conj(psi_x) (O_site psi)_x, the plain definition.  out: re, im words. */
int oracle_sv_expect1(void* hv, int site, const double* O, int w, double* out, int w_out) {
  sv_t* h = (sv_t*)hv;
  if (site < 0 || site >= h->n) return 1;
  cmp_t g[4]; load_mat(g, O, 2, w);
  size_t bit = (size_t)1 << (h->n - 1 - site);
  cmp_t acc; cmp_zero(&acc);
  for (size_t x = 0; x < h->dim; ++x) {
    if (x & bit) continue;
    cmp_t a0 = h->psi[x], a1 = h->psi[x | bit], t, r0, r1;
    cmp_mul(&r0, &g[0], &a0); cmp_mul(&t, &g[1], &a1); cmp_add(&r0, &r0, &t);
    cmp_mul(&r1, &g[2], &a0); cmp_mul(&t, &g[3], &a1); cmp_add(&r1, &r1, &t);
    cmp_mul_conj(&t, &a0, &r0); cmp_add(&acc, &acc, &t);
    cmp_mul_conj(&t, &a1, &r1); cmp_add(&acc, &acc, &t);
  }
  mp_to_words(&acc.re, out, w_out);
  mp_to_words(&acc.im, out + w_out, w_out);
  return 0;
}

/* The same expectation value from a Vidal MPS in canonical form (the layout of oracle_mps_amplitudes):
 * the environments left of bond l-1 and right of bond l reduce to the squared Schmidt weights, so
 *   <O_l> = sum over alpha, beta, s, s' of lam[l-1]_alpha^2 lam[l]_beta^2 conj(Gamma[l]^s_{alpha beta})
 *           O_{s s'} Gamma[l]^{s'}_{alpha beta}.
 * Only site l's tensor and its two weight vectors are read.  out: re, im words. */
int oracle_mps_expect1(int n, const int* chi, const double* gam, const double* lam, int w, int site,
                       const double* O, int wo, double* out, int w_out) {
  if (n < 2 || site < 0 || site >= n) return 1;
  size_t goff = 0, loff = 0;
  for (int l = 0; l < site; ++l) {
    const int cl = l == 0 ? 1 : chi[l - 1], cr = chi[l];
    goff += (size_t)2 * cl * cr;
    if (l < site - 1) loff += cr;                     /* lam[site-1] starts after lam[0..site-2] */
  }
  const int a = site == 0 ? 1 : chi[site - 1], b = site == n - 1 ? 1 : chi[site];
  cmp_t o[4]; load_mat(o, O, 2, wo);
  mp* wl = (mp*)malloc(sizeof(mp) * a);
  mp* wr = (mp*)malloc(sizeof(mp) * b);
  for (int k = 0; k < a; ++k) {
    if (site == 0) mp_from_double(&wl[k], 1.0);
    else { mp t; mp_from_words(&t, lam + (loff + k) * w, w); mp_mul(&wl[k], &t, &t); }
  }
  const size_t roff = site == 0 ? 0 : loff + a;       /* lam[site] follows lam[site-1] */
  for (int k = 0; k < b; ++k) {
    if (site == n - 1) mp_from_double(&wr[k], 1.0);
    else { mp t; mp_from_words(&t, lam + (roff + k) * w, w); mp_mul(&wr[k], &t, &t); }
  }
  cmp_t acc; cmp_zero(&acc);
  for (int al = 0; al < a; ++al) for (int be = 0; be < b; ++be) {
    cmp_t gs[2];
    for (int s = 0; s < 2; ++s) {
      const size_t e = goff + ((size_t)s * a + al) * b + be;
      mp_from_words(&gs[s].re, gam + (e * 2 + 0) * w, w);
      mp_from_words(&gs[s].im, gam + (e * 2 + 1) * w, w);
    }
    mp wt; mp_mul(&wt, &wl[al], &wr[be]);
    for (int s = 0; s < 2; ++s) {
      cmp_t og, t, u; cmp_zero(&og);                   /* (O Gamma)^s = sum over s' of O_{s s'} Gamma^{s'} */
      for (int s2 = 0; s2 < 2; ++s2) { cmp_mul(&t, &o[s * 2 + s2], &gs[s2]); cmp_add(&og, &og, &t); }
      cmp_mul_conj(&u, &gs[s], &og);
      cmp_scale(&u, &u, &wt);
      cmp_add(&acc, &acc, &u);
    }
  }
  mp_to_words(&acc.re, out, w_out);
  mp_to_words(&acc.im, out + w_out, w_out);
  free(wl); free(wr);
  return 0;
}

/* Vidal MPS of a sum of two product states, psi = sum over t of c_t (x)_l v^t_l (t = 0, 1), at any n: the
 * footnote's state C^{n-1}-U |+...+>|-> is |+...+>|-> + 2^{-(n-1)/2} |c> (U - 1)|->, such a sum, with Schmidt
 * rank 2 at every cut.  At the cut before site l, with L^t = (x)_{k<l} v^t_k and R^t = (x)_{k>=l} v^t_k,
 * psi = sum_t c_t L^t R^t.  The Grams GL_st = <L^s|L^t> and GR_st = <R^s|R^t> are products of local inner
 * products.  In the orthonormal bases e = L Q^{-1}, f = R P^{-1} from the Cholesky factors
 * GL = Q^H Q, GR = P^H P, the coefficients are Psi = Q diag(c) P^T; its Schmidt pairs come from the
 * Jacobi eigensolve of Psi Psi^H (u_k: eigenvectors, lambda_k^2: eigenvalues, v_k = Psi^T conj(u_k) /
 * lambda_k).  Each Schmidt vector is then a combination of L^0, L^1 (or R^0, R^1), and
 *   Gamma[l]^s_{alpha beta} = sum_t c_t <u^(l)_alpha|L^t> <s|v^t_l> <v^(l+1)_beta|R^t_{l+1}> / (lambda^(l)_alpha lambda^(l+1)_beta).
 * When the two terms are parallel on one side of a cut (GL or GR singular below 2^-tol_log2 of its
 * trace) that cut has rank 1.  vecs: [t][l][amplitude 0, 1] complex, w words; coef: 2 complex, w words.
 * Output as for oracle_sv_vidal.  Returns 0, or 1 on bad arguments. */
typedef struct { cmp_t x[2][2]; } c22;

static void c22_zero(c22* m) { for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) cmp_zero(&m->x[i][j]); }

/* Cholesky-type factor of a Hermitian positive semi-definite 2x2 G = Q^H Q with Q upper triangular;
 * returns the rank (1 if the trailing pivot is below 2^-tol of the trace) */
static int chol22(const c22* G, int tol_log2, c22* Q) {
  c22_zero(Q);
  mp q00; mp_sqrt(&q00, &G->x[0][0].re);
  Q->x[0][0].re = q00;
  cmp_t q01; mp_div(&q01.re, &G->x[0][1].re, &q00); mp_div(&q01.im, &G->x[0][1].im, &q00);   /* conj(Q00) Q01 = G01 */
  Q->x[0][1] = q01;
  mp d, t, tr; cmp_abs2(&t, &q01); mp_sub(&d, &G->x[1][1].re, &t);
  mp_add(&tr, &G->x[0][0].re, &G->x[1][1].re); mp_ldexp(&tr, &tr, -tol_log2);
  if (mp_cmp(&d, &tr) <= 0) return 1;
  mp_sqrt(&Q->x[1][1].re, &d);
  return 2;
}

int oracle_mps_two_products(int n, const double* vecs, const double* coef, int w, int tol_log2, int* chi,
                            double* gam, double* lam, int w_out) {
  if (n < 2 || n > 100000 || w < 1) return 1;
  cmp_t* v = (cmp_t*)malloc(sizeof(cmp_t) * 2 * (size_t)n * 2);     /* v[(t n + l) 2 + s] */
  for (size_t e = 0; e < (size_t)4 * n; ++e) {
    mp_from_words(&v[e].re, vecs + (e * 2 + 0) * w, w);
    mp_from_words(&v[e].im, vecs + (e * 2 + 1) * w, w);
  }
  cmp_t c[2];
  for (int t = 0; t < 2; ++t) { mp_from_words(&c[t].re, coef + (t * 2 + 0) * w, w); mp_from_words(&c[t].im, coef + (t * 2 + 1) * w, w); }
  /* local inner products g_l[s][t] = <v^s_l|v^t_l>, prefix (left) and suffix (right) Gram products */
  c22* GLp = (c22*)malloc(sizeof(c22) * (n + 1));                   /* GLp[l]: sites < l */
  c22* GRs = (c22*)malloc(sizeof(c22) * (n + 1));                   /* GRs[l]: sites >= l */
  for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) {
    cmp_zero(&GLp[0].x[i][j]); mp_from_double(&GLp[0].x[i][j].re, 1.0);
    cmp_zero(&GRs[n].x[i][j]); mp_from_double(&GRs[n].x[i][j].re, 1.0);
  }
  cmp_t* gl = (cmp_t*)malloc(sizeof(cmp_t) * 4 * (size_t)n);
  for (int l = 0; l < n; ++l) for (int s = 0; s < 2; ++s) for (int t = 0; t < 2; ++t) {
    cmp_t acc, u; cmp_zero(&acc);
    for (int a = 0; a < 2; ++a) { cmp_mul_conj(&u, &v[((size_t)s * n + l) * 2 + a], &v[((size_t)t * n + l) * 2 + a]); cmp_add(&acc, &acc, &u); }
    gl[(size_t)l * 4 + s * 2 + t] = acc;
  }
  for (int l = 0; l < n; ++l) for (int s = 0; s < 2; ++s) for (int t = 0; t < 2; ++t)
    cmp_mul(&GLp[l + 1].x[s][t], &GLp[l].x[s][t], &gl[(size_t)l * 4 + s * 2 + t]);
  for (int l = n - 1; l >= 0; --l) for (int s = 0; s < 2; ++s) for (int t = 0; t < 2; ++t)
    cmp_mul(&GRs[l].x[s][t], &GRs[l + 1].x[s][t], &gl[(size_t)l * 4 + s * 2 + t]);
  /* per cut l (between sites l-1 and l, l = 1..n-1): rank k, weights, and coefficient matrices A (u_alpha =
   * sum_s A[alpha][s] L^s) and B (v_beta = sum_t B[beta][t] R^t); cuts 0 and n are the trivial ones */
  int* rk = (int*)calloc(n + 1, sizeof(int));
  c22* A = (c22*)calloc(n + 1, sizeof(c22));
  c22* B = (c22*)calloc(n + 1, sizeof(c22));
  mp* lw = (mp*)calloc((size_t)2 * (n + 1), sizeof(mp));
  rk[0] = rk[n] = 1;
  mp_from_double(&lw[0], 1.0); mp_from_double(&lw[2 * n], 1.0);
  /* trivial cuts: the "left vector" of the empty prefix is 1 = L^0 = L^1 (A = (1, 0)); the right vector of
   * the empty suffix likewise (B = (1, 0)) */
  c22_zero(&A[0]); mp_from_double(&A[0].x[0][0].re, 1.0);
  c22_zero(&B[n]); mp_from_double(&B[n].x[0][0].re, 1.0);
  for (int l = 1; l < n; ++l) {
    c22 Q, P;
    const int rl = chol22(&GLp[l], tol_log2, &Q), rr = chol22(&GRs[l], tol_log2, &P);
    /* Psi = Q diag(c) P^T restricted to the ranks (a rank-1 side keeps only row/column 0) */
    c22 Psi; c22_zero(&Psi);
    for (int a = 0; a < rl; ++a) for (int b = 0; b < rr; ++b)
      for (int t = 0; t < 2; ++t) {
        cmp_t u, z; cmp_mul(&u, &Q.x[a][t], &c[t]); cmp_mul(&z, &u, &P.x[b][t]); cmp_add(&Psi.x[a][b], &Psi.x[a][b], &z);
      }
    /* rho = Psi Psi^H (rl x rl), eigen-decomposition */
    cmp_t g[4], ev[4]; mp mu[2]; int order[2];
    for (int a = 0; a < rl; ++a) for (int b = 0; b < rl; ++b) {
      cmp_t acc, u; cmp_zero(&acc);
      for (int k = 0; k < rr; ++k) { cmp_mul_conj(&u, &Psi.x[b][k], &Psi.x[a][k]); cmp_add(&acc, &acc, &u); }
      g[a + b * rl] = acc;
    }
    oracle_jacobi_mp(rl, g, ev, 80);
    oracle_finish_mp(rl, g, ev, mu, order);
    mp cut; mp_ldexp(&cut, &mu[0], -tol_log2);
    int k = 0; while (k < rl && mp_cmp(&mu[k], &cut) > 0) ++k;
    if (k == 0) k = 1;
    rk[l] = k;
    /* Q^{-1} (upper triangular, rank rl): e_a = sum_s L^s Qinv[s][a] */
    c22 Qi, Pi; c22_zero(&Qi); c22_zero(&Pi);
    for (int side = 0; side < 2; ++side) {
      const c22* F = side == 0 ? &Q : &P; c22* Fi = side == 0 ? &Qi : &Pi; const int r = side == 0 ? rl : rr;
      mp one; mp_from_double(&one, 1.0);
      mp_div(&Fi->x[0][0].re, &one, &F->x[0][0].re);
      if (r == 2) {
        mp_div(&Fi->x[1][1].re, &one, &F->x[1][1].re);
        cmp_t t1; cmp_scale(&t1, &F->x[0][1], &Fi->x[1][1].re); cmp_scale(&t1, &t1, &Fi->x[0][0].re);
        mp_neg(&Fi->x[0][1].re, &t1.re); mp_neg(&Fi->x[0][1].im, &t1.im);                    /* -q01 / (q00 q11) */
      }
    }
    for (int q = 0; q < k; ++q) {
      mp_sqrt(&lw[2 * l + q], &mu[q]);
      const cmp_t* e = ev + (size_t)order[q] * rl;      /* u_q in the basis e_a */
      /* A[q][s] = sum_a Qinv[s][a] e[a] (coefficients on L^s) */
      for (int s = 0; s < 2; ++s) {
        cmp_t acc, u; cmp_zero(&acc);
        for (int a = 0; a < rl; ++a) { cmp_mul(&u, &Qi.x[s][a], &e[a]); cmp_add(&acc, &acc, &u); }
        A[l].x[q][s] = acc;
      }
      /* v_q = Psi^T conj(u_q) / lambda_q in the basis f_b, then B[q][t] = sum_b Pinv[t][b] v[b] */
      cmp_t vb[2];
      for (int b = 0; b < 2; ++b) {
        cmp_t acc, u; cmp_zero(&acc);
        if (b < rr) for (int a = 0; a < rl; ++a) { cmp_mul_conj(&u, &e[a], &Psi.x[a][b]); cmp_add(&acc, &acc, &u); }
        mp_div(&acc.re, &acc.re, &lw[2 * l + q]); mp_div(&acc.im, &acc.im, &lw[2 * l + q]);
        vb[b] = acc;
      }
      for (int t = 0; t < 2; ++t) {
        cmp_t acc, u; cmp_zero(&acc);
        for (int b = 0; b < rr; ++b) { cmp_mul(&u, &Pi.x[t][b], &vb[b]); cmp_add(&acc, &acc, &u); }
        B[l].x[q][t] = acc;
      }
    }
  }
  /* Gamma[l]^s_{alpha beta} = sum_t c_t <u^(l)_alpha|L^t_l> v^t_l[s] <v^(l+1)_beta|R^t_{l+1}> / (lam lam) */
  size_t go = 0, lo = 0;
  for (int l = 0; l < n; ++l) {
    const int ca = rk[l], cb = rk[l + 1];
    for (int s = 0; s < 2; ++s) for (int al = 0; al < ca; ++al) for (int be = 0; be < cb; ++be) {
      cmp_t acc; cmp_zero(&acc);
      for (int t = 0; t < 2; ++t) {
        cmp_t ul, vr, u, z;
        cmp_zero(&ul);                                 /* <u_alpha|L^t> = sum_s' conj(A[alpha][s']) GL[s'][t] */
        for (int s2 = 0; s2 < 2; ++s2) { cmp_mul_conj(&u, &A[l].x[al][s2], &GLp[l].x[s2][t]); cmp_add(&ul, &ul, &u); }
        cmp_zero(&vr);                                 /* <v_beta|R^t_{l+1}> = sum_t' conj(B[beta][t']) GR[t'][t] */
        for (int t2 = 0; t2 < 2; ++t2) { cmp_mul_conj(&u, &B[l + 1].x[be][t2], &GRs[l + 1].x[t2][t]); cmp_add(&vr, &vr, &u); }
        cmp_mul(&u, &c[t], &ul);
        cmp_mul(&z, &u, &v[((size_t)t * n + l) * 2 + s]);
        cmp_mul(&u, &z, &vr);
        cmp_add(&acc, &acc, &u);
      }
      mp den; mp_mul(&den, &lw[2 * l + al], &lw[2 * (l + 1) + be]);
      mp_div(&acc.re, &acc.re, &den); mp_div(&acc.im, &acc.im, &den);
      const size_t e = go + ((size_t)s * ca + al) * cb + be;
      mp_to_words(&acc.re, gam + (e * 2 + 0) * w_out, w_out);
      mp_to_words(&acc.im, gam + (e * 2 + 1) * w_out, w_out);
    }
    go += (size_t)2 * ca * cb;
    if (l < n - 1) {
      chi[l] = cb;
      for (int be = 0; be < cb; ++be) mp_to_words(&lw[2 * (l + 1) + be], lam + (lo + be) * w_out, w_out);
      lo += cb;
    }
  }
  free(v); free(GLp); free(GRs); free(gl); free(rk); free(A); free(B); free(lw);
  return 0;
}
