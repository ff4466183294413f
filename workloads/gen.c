/*
 * Seeded synthetic input generators (shared by the CUDA path's tests/bench and by the oracle's tests).
 *
 * This module holds none of the eigensolver's arithmetic: it draws complex Gaussians from a
 * counter-based generator, orthonormalises them by Gram-Schmidt in plain fp64 (giving a Haar-distributed
 * unitary, Mezzadri 2007: QR of a complex Gaussian with positive diagonal R), and forms
 *     A = U diag(lambda) U^H
 * EXACTLY with an integer (Kulisch-style) accumulator before rounding each real part to w doubles
 * (successive round-to-nearest).  Everything uses only IEEE +,-,*,/ and sqrt with contraction disabled,
 * plus integer operations, so the bits produced are identical on x86-64 and aarch64.
 *
 * Near-degenerate pairs: for a pair of eigen-indices (a, b) the generator builds u_b = J conj(u_a), with
 * (Jv)_{2m} = -v_{2m+1}, (Jv)_{2m+1} = v_{2m}.  Then u_a^H u_b = 0 and |u_b| = |u_a| hold exactly, so the
 * exact product keeps the prescribed split lambda_a - lambda_b even though U is unitary only to ~1e-16
 * (the remaining columns are orthogonalised against both members in the usual way).
 */
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#include <math.h>

/* ---------------- counter-based RNG: SplitMix64 finaliser over (key, counter) ---------------- */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static uint64_t rng_u64(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL); }
/* uniform in (0,1): 53 random bits, centred in their cell */
static double rng_unif(uint64_t key, uint64_t ctr) { return ((double)(rng_u64(key, ctr) >> 11) + 0.5) * 0x1p-53; }

uint64_t gen_key(uint64_t seed, uint64_t stream) { return mix64(mix64(seed ^ 0x5A17C0DEULL) + stream * 0xD1B54A32D192ED03ULL); }

/* Deterministic elementary functions from +,-,*,/ only (accuracy ~1e-16 is plenty for a generator). */
static const double LN2 = 0.6931471805599453094;
static double det_log(double x) { /* x in (0,1] */
  int e = 0;
  while (x < 0.70710678118654752) { x *= 2.0; e -= 1; }
  while (x > 1.41421356237309505) { x *= 0.5; e += 1; }
  double z = (x - 1.0) / (x + 1.0), z2 = z * z, term = z, s = 0.0;
  for (int k = 1; k < 60; k += 2) { s += term / k; term *= z2; }
  return 2.0 * s + e * LN2;
}
static void det_sincos_2pi(double u, double* s_out, double* c_out) { /* angle 2*pi*u, u in [0,1) */
  const double PI = 3.14159265358979323846;
  int q = (int)(u * 4.0); if (q > 3) q = 3;
  double th = (u - 0.25 * q) * 2.0 * PI;               /* th in [0, pi/2) */
  double s = 0.0, c = 0.0, t = th, tc = 1.0;
  for (int k = 1; k < 40; k += 2) { s += t; t *= -th * th / ((k + 1.0) * (k + 2.0)); }
  for (int k = 0; k < 40; k += 2) { c += tc; tc *= -th * th / ((k + 1.0) * (k + 2.0)); }
  double ss[4] = {s, c, -s, -c}, cc[4] = {c, -s, -c, s};
  *s_out = ss[q]; *c_out = cc[q];
}
/* standard complex Gaussian (re, im each N(0, 1/2)) number `idx` of stream `key` (Box-Muller) */
static void cgauss(uint64_t key, uint64_t idx, double* re, double* im) {
  double u1 = rng_unif(key, 2 * idx), u2 = rng_unif(key, 2 * idx + 1);
  double r = sqrt(-det_log(u1)); /* sqrt(-2 ln u1) * sqrt(1/2) */
  double s, c; det_sincos_2pi(u2, &s, &c);
  *re = r * c; *im = r * s;
}

/* uniform doubles for host-side choices (exported so Python draws from the same counter stream) */
void gen_uniform(uint64_t key, uint64_t first, int64_t count, double* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = rng_unif(key, first + (uint64_t)i);
}

/* Haar unitary columns by classical Gram-Schmidt applied twice (CGS2), column-major n x n complex,
 * interleaved (re, im).  pair_of[c] = c-1 marks column c as J conj(column c-1); -1 otherwise. */
static void haar_columns(uint64_t key, int n, const int* pair_of, double* U) {
  for (int c = 0; c < n; ++c) {
    double* u = U + 2 * (size_t)n * c;
    if (pair_of && pair_of[c] >= 0) {
      const double* v = U + 2 * (size_t)n * pair_of[c];
      for (int m = 0; m + 1 < n; m += 2) {           /* (J conj v)_{2m} = -conj(v_{2m+1}); _{2m+1} = conj(v_{2m}) */
        u[2 * m] = -v[2 * (m + 1)];     u[2 * m + 1] = v[2 * (m + 1) + 1];
        u[2 * (m + 1)] = v[2 * m];      u[2 * (m + 1) + 1] = -v[2 * m + 1];
      }
      continue;
    }
    for (int i = 0; i < n; ++i) cgauss(key, (uint64_t)c * n + i, &u[2 * i], &u[2 * i + 1]);
    for (int pass = 0; pass < 2; ++pass) {
      for (int d = 0; d < c; ++d) {
        const double* v = U + 2 * (size_t)n * d;
        double pr = 0, pi = 0;                        /* <v, u> = sum conj(v_i) u_i */
        for (int i = 0; i < n; ++i) {
          pr += v[2 * i] * u[2 * i] + v[2 * i + 1] * u[2 * i + 1];
          pi += v[2 * i] * u[2 * i + 1] - v[2 * i + 1] * u[2 * i];
        }
        for (int i = 0; i < n; ++i) {
          u[2 * i] -= pr * v[2 * i] - pi * v[2 * i + 1];
          u[2 * i + 1] -= pr * v[2 * i + 1] + pi * v[2 * i];
        }
      }
    }
    double nrm = 0;
    for (int i = 0; i < 2 * n; ++i) nrm += u[i] * u[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < 2 * n; ++i) u[i] /= nrm;
  }
}

/* ---------------- exact accumulation of products of three doubles ---------------- */
#define ACC_LIMBS 24           /* 1536 bits: bit 0 of limb 0 has weight 2^ACC_LOW */
#define ACC_LOW (-1400)
typedef struct { uint64_t pos[ACC_LIMBS], neg[ACC_LIMBS]; } acc_t;

static void acc_add_u192(uint64_t* limbs, const uint64_t v[3], int off) {
  /* add the 192-bit integer v (little-endian limbs) shifted left by `off` bits */
  if (off < 0) return;                              /* below the accumulator's range: dropped */
  int li = off >> 6, sh = off & 63;
  uint64_t w[4];
  if (sh == 0) { w[0] = v[0]; w[1] = v[1]; w[2] = v[2]; w[3] = 0; }
  else {
    w[0] = v[0] << sh; w[1] = (v[1] << sh) | (v[0] >> (64 - sh));
    w[2] = (v[2] << sh) | (v[1] >> (64 - sh)); w[3] = v[2] >> (64 - sh);
  }
  if (li + 4 > ACC_LIMBS) return;                   /* above the range: cannot happen for |values| < 2^100 */
  uint64_t c = 0;
  for (int k = 0; k < 4; ++k) {
    uint64_t a = limbs[li + k], t = a + w[k];
    uint64_t c1 = t < a;
    uint64_t t2 = t + c;
    c = c1 | (t2 < t);
    limbs[li + k] = t2;
  }
  for (int k = li + 4; c && k < ACC_LIMBS; ++k) { limbs[k] += 1; c = limbs[k] == 0; }
}
/* decompose a finite nonzero double into (mantissa integer < 2^53, exponent): x = m * 2^e */
static inline void dsplit(double x, uint64_t* m, int* e, int* neg) {
  uint64_t b; memcpy(&b, &x, 8);
  *neg = (int)(b >> 63);
  int be = (int)((b >> 52) & 0x7FF);
  uint64_t f = b & 0xFFFFFFFFFFFFFULL;
  if (be == 0) { *m = f; *e = -1074; } else { *m = f | (1ULL << 52); *e = be - 1075; }
}
/* acc += sgn * x*y*z exactly */
static void acc_add3(acc_t* acc, double x, double y, double z, int sgn) {
  if (x == 0.0 || y == 0.0 || z == 0.0) return;
  uint64_t mx, my, mz; int ex, ey, ez, nx, ny, nz;
  dsplit(x, &mx, &ex, &nx); dsplit(y, &my, &ey, &ny); dsplit(z, &mz, &ez, &nz);
  unsigned __int128 p = (unsigned __int128)mx * my;           /* < 2^106 */
  unsigned __int128 lo = (unsigned __int128)(uint64_t)p * mz;
  unsigned __int128 hi = (unsigned __int128)(uint64_t)(p >> 64) * mz;
  uint64_t v[3];
  v[0] = (uint64_t)lo;
  unsigned __int128 mid = (lo >> 64) + (uint64_t)hi;
  v[1] = (uint64_t)mid;
  v[2] = (uint64_t)(hi >> 64) + (uint64_t)(mid >> 64);
  int neg = nx ^ ny ^ nz ^ (sgn < 0);
  acc_add_u192(neg ? acc->neg : acc->pos, v, ex + ey + ez - ACC_LOW);
}
/* value = pos - neg as sign + magnitude limbs; returns sign (+1/-1/0) */
static int acc_magnitude(const acc_t* acc, uint64_t* mag) {
  int cmp = 0;
  for (int k = ACC_LIMBS - 1; k >= 0; --k) {
    if (acc->pos[k] != acc->neg[k]) { cmp = acc->pos[k] > acc->neg[k] ? 1 : -1; break; }
  }
  if (cmp == 0) { memset(mag, 0, sizeof(uint64_t) * ACC_LIMBS); return 0; }
  const uint64_t* a = cmp > 0 ? acc->pos : acc->neg;
  const uint64_t* b = cmp > 0 ? acc->neg : acc->pos;
  unsigned __int128 borrow = 0;
  for (int k = 0; k < ACC_LIMBS; ++k) {
    unsigned __int128 d = (unsigned __int128)a[k] - b[k] - borrow;
    mag[k] = (uint64_t)d; borrow = (d >> 64) ? 1 : 0;
  }
  return cmp;
}
static int top_bit(const uint64_t* mag) {
  for (int k = ACC_LIMBS - 1; k >= 0; --k) if (mag[k]) return 64 * k + 63 - __builtin_clzll(mag[k]);
  return -1;
}
static int get_bit(const uint64_t* mag, int i) { return i < 0 ? 0 : (int)((mag[i >> 6] >> (i & 63)) & 1); }
/* Round the signed big integer (sign s, magnitude mag, weight 2^ACC_LOW per unit) to nearest-even double
 * and subtract that double from it (exactly).  Returns the double. */
static double round_off_word(int* s, uint64_t* mag) {
  if (*s == 0) return 0.0;
  int t = top_bit(mag);
  if (t < 0) { *s = 0; return 0.0; }
  int lo = t - 52;                                    /* lowest kept bit index */
  uint64_t m = 0;
  for (int i = t; i >= lo; --i) m = (m << 1) | (uint64_t)get_bit(mag, i);
  int rnd = get_bit(mag, lo - 1), sticky = 0;
  for (int i = lo - 2; i >= 0 && !sticky; --i) sticky = get_bit(mag, i);
  if (lo - 1 < 0) rnd = 0;
  int up = rnd && (sticky || (m & 1));
  /* clear bits >= lo, then the remainder is mag - (m << lo) if not rounding up, else (m+1)<<lo - mag */
  double word;
  if (!up) {
    for (int i = lo < 0 ? 0 : lo; i <= t; ++i) mag[i >> 6] &= ~(1ULL << (i & 63));
    word = ldexp((double)m, lo + ACC_LOW);
  } else {
    /* remainder r = mag - (m+1)*2^lo (negative): magnitude = (m+1)*2^lo - mag = 2^lo - (mag mod 2^lo) */
    uint64_t low[ACC_LIMBS]; memset(low, 0, sizeof low);
    for (int i = 0; i < lo; ++i) if (get_bit(mag, i)) low[i >> 6] |= 1ULL << (i & 63);
    uint64_t pw[ACC_LIMBS]; memset(pw, 0, sizeof pw); pw[lo >> 6] = 1ULL << (lo & 63);
    unsigned __int128 borrow = 0;
    for (int k = 0; k < ACC_LIMBS; ++k) {
      unsigned __int128 d = (unsigned __int128)pw[k] - low[k] - borrow;
      mag[k] = (uint64_t)d; borrow = (d >> 64) ? 1 : 0;
    }
    word = ldexp((double)(m + 1), lo + ACC_LOW);
    double sgnw = *s > 0 ? word : -word;
    *s = -*s;
    if (top_bit(mag) < 0) *s = 0;
    return sgnw;
  }
  double sgnw = *s > 0 ? word : -word;
  if (top_bit(mag) < 0) *s = 0;
  return sgnw;
}
static void acc_to_words(const acc_t* acc, int w, double* out) {
  uint64_t mag[ACC_LIMBS];
  int s = acc_magnitude(acc, mag);
  for (int k = 0; k < w; ++k) out[k] = round_off_word(&s, mag);
}

/* A = U diag(lam + lam_lo) U^H (lam_lo may be NULL), written column-major complex with w words per real:
 * A[((i + j*n)*2 + part)*w + k].  pairs: npairs (a, b) index pairs of eigen-indices that must stay split
 * exactly (b gets J conj of a's column).  Returns 0 on success. */
int gen_herm_spectrum(uint64_t key, int n, const double* lam, const double* lam_lo, int npairs,
                      const int* pairs, int w, double* A, double* Uout) {
  if (n <= 0 || w < 1 || w > 8) return 1;
  double* G = (double*)malloc(sizeof(double) * 2 * (size_t)n * n);   /* columns in generation order */
  int* pair_of = (int*)malloc(sizeof(int) * n);
  int* col_of_eig = (int*)malloc(sizeof(int) * n);                     /* eigen-index -> generated column */
  int* used = (int*)calloc(n, sizeof(int));
  if (!G || !pair_of || !col_of_eig || !used) return 2;
  for (int c = 0; c < n; ++c) pair_of[c] = -1;
  int c = 0;
  for (int p = 0; p < npairs; ++p) {
    int a = pairs[2 * p], b = pairs[2 * p + 1];
    if (a < 0 || b < 0 || a >= n || b >= n || used[a] || used[b] || (n & 1)) return 3;
    used[a] = used[b] = 1;
    col_of_eig[a] = c; col_of_eig[b] = c + 1; pair_of[c + 1] = c; c += 2;
  }
  for (int k = 0; k < n; ++k) if (!used[k]) col_of_eig[k] = c++;
  haar_columns(key, n, pair_of, G);
  double* U = (double*)malloc(sizeof(double) * 2 * (size_t)n * n);     /* U[:,k] = eigenvector of lam[k] */
  for (int k = 0; k < n; ++k) memcpy(U + 2 * (size_t)n * k, G + 2 * (size_t)n * col_of_eig[k], sizeof(double) * 2 * n);
  /* Pre-split every lam_k * U_ik into an exact 106-bit integer times a power of two, and every U_jk
   * into a 53-bit one, so each term of the sum is one 106 x 53-bit integer product. */
  size_t nn = (size_t)n * n;
  unsigned __int128* Pm = (unsigned __int128*)malloc(sizeof(unsigned __int128) * 2 * nn);
  int* Pe = (int*)malloc(sizeof(int) * 2 * nn);
  uint64_t* Um = (uint64_t*)malloc(sizeof(uint64_t) * 2 * nn);
  int* Ue = (int*)malloc(sizeof(int) * 2 * nn);
  if (!Pm || !Pe || !Um || !Ue) return 2;
  for (int k = 0; k < n; ++k) {
    uint64_t ml; int el, nl; dsplit(lam[k], &ml, &el, &nl);
    for (int i = 0; i < n; ++i) {
      for (int part = 0; part < 2; ++part) {
        double u = U[2 * ((size_t)n * k + i) + part];
        size_t idx = 2 * ((size_t)i * n + k) + part;      /* row-major in (i, k) for streaming over k */
        if (u == 0.0 || lam[k] == 0.0) { Pm[idx] = 0; Pe[idx] = 0; Um[idx] = 0; Ue[idx] = 0; continue; }
        uint64_t mu; int eu, nu; dsplit(u, &mu, &eu, &nu);
        Pm[idx] = (unsigned __int128)ml * mu; Pe[idx] = (el + eu) * 2 + (nl ^ nu);  /* sign in the low bit */
        Um[idx] = mu; Ue[idx] = eu * 2 + nu;
      }
    }
  }
  acc_t* acc = (acc_t*)malloc(sizeof(acc_t));
  for (int j = 0; j < n; ++j) {
    for (int i = j; i < n; ++i) {
      /* A_ij = sum_k lam_k U_ik conj(U_jk):  re = lam(a_i a_j + b_i b_j), im = lam(b_i a_j - a_i b_j) */
      double wr[8], wi[8];
      for (int part = 0; part < 2; ++part) {
        if (part == 1 && i == j) { for (int k = 0; k < w; ++k) wi[k] = 0.0; break; }
        memset(acc, 0, sizeof(acc_t));
        for (int k = 0; k < n; ++k) {
          size_t pi_ = 2 * ((size_t)i * n + k), pj_ = 2 * ((size_t)j * n + k);
          /* part 0: P_re(i)*U_re(j) + P_im(i)*U_im(j);  part 1: P_im(i)*U_re(j) - P_re(i)*U_im(j) */
          for (int t = 0; t < 2; ++t) {
            size_t a = pi_ + (part == 0 ? t : 1 - t), b = pj_ + t;
            unsigned __int128 pm = Pm[a]; uint64_t um = Um[b];
            if (!pm || !um) continue;
            int neg = (Pe[a] & 1) ^ (Ue[b] & 1) ^ (part == 1 && t == 1);
            int e = (Pe[a] >> 1) + (Ue[b] >> 1);
            unsigned __int128 lo = (unsigned __int128)(uint64_t)pm * um;
            unsigned __int128 hi = (unsigned __int128)(uint64_t)(pm >> 64) * um;
            uint64_t v[3];
            v[0] = (uint64_t)lo;
            unsigned __int128 mid = (lo >> 64) + (uint64_t)hi;
            v[1] = (uint64_t)mid;
            v[2] = (uint64_t)(hi >> 64) + (uint64_t)(mid >> 64);
            acc_add_u192(neg ? acc->neg : acc->pos, v, e - ACC_LOW);
          }
          if (lam_lo && lam_lo[k] != 0.0) {
            const double* uk = U + 2 * (size_t)n * k;
            if (part == 0) {
              acc_add3(acc, lam_lo[k], uk[2 * i], uk[2 * j], 1);
              acc_add3(acc, lam_lo[k], uk[2 * i + 1], uk[2 * j + 1], 1);
            } else {
              acc_add3(acc, lam_lo[k], uk[2 * i + 1], uk[2 * j], 1);
              acc_add3(acc, lam_lo[k], uk[2 * i], uk[2 * j + 1], -1);
            }
          }
        }
        acc_to_words(acc, w, part == 0 ? wr : wi);
      }
      for (int k = 0; k < w; ++k) {
        A[(((size_t)i + (size_t)j * n) * 2 + 0) * w + k] = wr[k];
        A[(((size_t)i + (size_t)j * n) * 2 + 1) * w + k] = wi[k];
        A[(((size_t)j + (size_t)i * n) * 2 + 0) * w + k] = wr[k];
        A[(((size_t)j + (size_t)i * n) * 2 + 1) * w + k] = -wi[k];
      }
    }
  }
  free(Pm); free(Pe); free(Um); free(Ue);
  if (Uout) memcpy(Uout, U, sizeof(double) * 2 * (size_t)n * n);
  free(acc); free(U); free(G); free(pair_of); free(col_of_eig); free(used);
  return 0;
}

/* complex Gaussian matrix (column-major, interleaved) for tests that need raw random data */
void gen_cgauss(uint64_t key, int64_t count, double* out) {
  for (int64_t i = 0; i < count; ++i) cgauss(key, (uint64_t)i, &out[2 * i], &out[2 * i + 1]);
}
