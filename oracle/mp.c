/*
 * ORACLE (test infrastructure only).  320-bit floating point, written out plainly:
 * schoolbook multiply, aligned add/subtract with one guard limb, Newton iterations for reciprocal and
 * inverse square root.  No EFTs, no double-double: an independent path from the device arithmetic.
 */
#include "mp.h"
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

void mp_zero(mp* r) { memset(r, 0, sizeof(mp)); }
int mp_is_zero(const mp* a) { return a->m[MPL - 1] == 0; }
int mp_sign(const mp* a) { return mp_is_zero(a) ? 0 : (a->s ? -1 : 1); }
void mp_neg(mp* r, const mp* a) { *r = *a; if (!mp_is_zero(r)) r->s ^= 1; }
void mp_abs(mp* r, const mp* a) { *r = *a; r->s = 0; }
void mp_ldexp(mp* r, const mp* a, int64_t k) { *r = *a; if (!mp_is_zero(r)) r->e += k; }

/* normalise an (MPL+1)-limb magnitude x (x[0] = guard limb) with exponent e into r */
static void norm_store(mp* r, uint64_t* x, int64_t e, int s) {
  int top = -1;
  for (int k = MPL; k >= 0; --k) if (x[k]) { top = k; break; }
  if (top < 0) { mp_zero(r); return; }
  int limb_shift = MPL - top;                       /* whole limbs to shift left */
  if (limb_shift > 0) {
    for (int k = MPL; k >= 0; --k) x[k] = (k - limb_shift >= 0) ? x[k - limb_shift] : 0;
    e -= 64 * (int64_t)limb_shift;
  }
  int lz = __builtin_clzll(x[MPL]);
  if (lz) {
    for (int k = MPL; k > 0; --k) x[k] = (x[k] << lz) | (x[k - 1] >> (64 - lz));
    x[0] <<= lz;
    e -= lz;
  }
  for (int k = 0; k < MPL; ++k) r->m[k] = x[k + 1];
  r->e = e; r->s = s;
}

void mp_from_double(mp* r, double d) {
  mp_zero(r);
  if (d == 0.0) return;
  uint64_t b; memcpy(&b, &d, 8);
  int s = (int)(b >> 63), be = (int)((b >> 52) & 0x7FF);
  uint64_t f = b & 0xFFFFFFFFFFFFFULL;
  int64_t q; uint64_t m;
  if (be == 0) { m = f; q = -1074; } else { m = f | (1ULL << 52); q = be - 1075; }
  uint64_t x[MPL + 1]; memset(x, 0, sizeof x);
  x[MPL] = m;                                        /* value = m * 2^q = (x / 2^(64 MPL)) * 2^(q + 64) */
  norm_store(r, x, q + 64, s);
}

int mp_cmp_abs(const mp* a, const mp* b) {
  int za = mp_is_zero(a), zb = mp_is_zero(b);
  if (za || zb) return za && zb ? 0 : (za ? -1 : 1);
  if (a->e != b->e) return a->e > b->e ? 1 : -1;
  for (int k = MPL - 1; k >= 0; --k) if (a->m[k] != b->m[k]) return a->m[k] > b->m[k] ? 1 : -1;
  return 0;
}
int mp_cmp(const mp* a, const mp* b) {
  int sa = mp_sign(a), sb = mp_sign(b);
  if (sa != sb) return sa > sb ? 1 : -1;
  if (sa == 0) return 0;
  int c = mp_cmp_abs(a, b);
  return sa > 0 ? c : -c;
}

static void add_signed(mp* r, const mp* a, const mp* b, int bneg) {
  int sb = b->s ^ bneg;
  if (mp_is_zero(b)) { *r = *a; return; }
  if (mp_is_zero(a)) { *r = *b; r->s = sb; return; }
  const mp *big = a, *sml = b; int sbig = a->s, ssml = sb;
  if (mp_cmp_abs(a, b) < 0) { big = b; sml = a; sbig = sb; ssml = a->s; }
  int64_t d = big->e - sml->e;
  uint64_t x[MPL + 2], y[MPL + 2];                   /* one guard limb below, one carry limb above */
  memset(x, 0, sizeof x); memset(y, 0, sizeof y);
  for (int k = 0; k < MPL; ++k) x[k + 1] = big->m[k];
  if (d < 64 * (MPL + 1)) {
    int64_t ls = d >> 6; int bs = (int)(d & 63);
    for (int k = 0; k < MPL; ++k) {                  /* y = (sml.m << 64) >> d */
      int64_t dst = k + 1 - ls;
      if (dst >= 0) y[dst] |= bs ? (sml->m[k] >> bs) : sml->m[k];
      if (bs && dst - 1 >= 0) y[dst - 1] |= sml->m[k] << (64 - bs);
    }
  }
  int64_t e = big->e;
  if (sbig == ssml) {
    uint64_t c = 0;
    for (int k = 0; k <= MPL + 1; ++k) {
      u128 s = (u128)x[k] + y[k] + c; x[k] = (uint64_t)s; c = (uint64_t)(s >> 64);
    }
    if (x[MPL + 1]) {                                /* carry: shift right by one bit */
      for (int k = 0; k <= MPL; ++k) x[k] = (x[k] >> 1) | (x[k + 1] << 63);
      x[MPL + 1] = 0; e += 1;
    }
  } else {
    uint64_t br = 0;
    for (int k = 0; k <= MPL + 1; ++k) {
      u128 s = (u128)x[k] - y[k] - br; x[k] = (uint64_t)s; br = (uint64_t)(s >> 64) ? 1 : 0;
    }
  }
  norm_store(r, x, e, sbig);
}
void mp_add(mp* r, const mp* a, const mp* b) { mp t; add_signed(&t, a, b, 0); *r = t; }
void mp_sub(mp* r, const mp* a, const mp* b) { mp t; add_signed(&t, a, b, 1); *r = t; }

void mp_mul(mp* r, const mp* a, const mp* b) {
  if (mp_is_zero(a) || mp_is_zero(b)) { mp_zero(r); return; }
  uint64_t p[2 * MPL]; memset(p, 0, sizeof p);
  for (int i = 0; i < MPL; ++i) {
    uint64_t c = 0;
    for (int j = 0; j < MPL; ++j) {
      u128 t = (u128)a->m[i] * b->m[j] + p[i + j] + c;
      p[i + j] = (uint64_t)t; c = (uint64_t)(t >> 64);
    }
    p[i + MPL] = c;
  }
  uint64_t x[MPL + 1];
  for (int k = 0; k <= MPL; ++k) x[k] = p[MPL - 1 + k];  /* keep one guard limb */
  mp t; norm_store(&t, x, a->e + b->e, a->s ^ b->s);
  *r = t;
}

/* top 64 bits as a double in [0.5, 1) (approximation used only to seed Newton iterations) */
static double mant_approx(const mp* a) { return ldexp((double)a->m[MPL - 1], -64) + ldexp((double)a->m[MPL - 2], -128); }

void mp_div(mp* r, const mp* a, const mp* b) {
  if (mp_is_zero(b)) { mp_zero(r); r->m[MPL - 1] = 1ULL << 63; r->e = 1 << 30; return; }  /* "infinity" */
  if (mp_is_zero(a)) { mp_zero(r); return; }
  mp bb = *b; bb.s = 0; bb.e = 0;                   /* |b| scaled into [0.5, 1) */
  mp x, t, one;
  mp_from_double(&x, 1.0 / mant_approx(&bb));
  mp_from_double(&one, 1.0);
  for (int it = 0; it < 5; ++it) {                   /* x <- x + x (1 - b x): 2^-50 -> 2^-100 -> ... */
    mp_mul(&t, &bb, &x); mp_sub(&t, &one, &t); mp_mul(&t, &x, &t); mp_add(&x, &x, &t);
  }
  mp q, aa = *a; aa.s = 0;
  mp_mul(&q, &aa, &x);                               /* q ~ |a| / |bb| */
  mp_mul(&t, &bb, &q); mp_sub(&t, &aa, &t); mp_mul(&t, &x, &t); mp_add(&q, &q, &t);   /* one correction */
  q.e -= b->e; q.s = a->s ^ b->s;
  if (mp_is_zero(&q)) mp_zero(&q);
  *r = q;
}

void mp_sqrt(mp* r, const mp* a) {
  if (mp_is_zero(a) || a->s) { mp_zero(r); return; }
  mp aa = *a; int64_t e = a->e;
  aa.e = (e & 1) ? 1 : 0;                            /* aa in [0.5, 2): a = aa * 2^(e - aa.e), e - aa.e even */
  int64_t half = (e - aa.e) / 2;
  double f = ldexp(mant_approx(a), (int)aa.e);
  mp y, t, one, three_half;
  mp_from_double(&y, 1.0 / sqrt(f));
  mp_from_double(&one, 1.0);
  for (int it = 0; it < 5; ++it) {                   /* y <- y + y (1 - aa y^2) / 2 */
    mp_mul(&t, &y, &y); mp_mul(&t, &aa, &t); mp_sub(&t, &one, &t); mp_mul(&t, &y, &t);
    mp_ldexp(&t, &t, -1); mp_add(&y, &y, &t);
  }
  (void)three_half;
  mp s;
  mp_mul(&s, &aa, &y);                               /* s ~ sqrt(aa) */
  mp_mul(&t, &s, &s); mp_sub(&t, &aa, &t); mp_mul(&t, &y, &t); mp_ldexp(&t, &t, -1); mp_add(&s, &s, &t);
  s.e += half;
  *r = s;
}

void mp_from_words(mp* r, const double* w, int n) {
  mp acc, t; mp_zero(&acc);
  for (int k = 0; k < n; ++k) { mp_from_double(&t, w[k]); mp_add(&acc, &acc, &t); }
  *r = acc;
}

/* round |a| to the nearest double (ties to even), honouring all lower limbs as sticky bits */
double mp_to_double(const mp* a) {
  if (mp_is_zero(a)) return 0.0;
  uint64_t top = a->m[MPL - 1];
  uint64_t m53 = top >> 11;                          /* 53 bits */
  uint64_t rest = top & 0x7FF;                       /* 11 bits below */
  int rnd = (int)((rest >> 10) & 1);
  int sticky = (rest & 0x3FF) != 0;
  for (int k = 0; k < MPL - 1 && !sticky; ++k) sticky = a->m[k] != 0;
  if (rnd && (sticky || (m53 & 1))) m53 += 1;
  /* value = m53 * 2^(e - 53); exponents far outside double range saturate via ldexp */
  int64_t e = a->e - 53;
  double v;
  if (e > 2000) v = INFINITY; else if (e < -2200) v = 0.0; else v = ldexp((double)m53, (int)e);
  return a->s ? -v : v;
}

void mp_to_words(const mp* a, double* w, int n) {
  mp rem = *a, t;
  for (int k = 0; k < n; ++k) {
    w[k] = mp_to_double(&rem);
    mp_from_double(&t, w[k]);
    mp_sub(&rem, &rem, &t);
  }
}

void cmp_zero(cmp_t* r) { mp_zero(&r->re); mp_zero(&r->im); }
void cmp_add(cmp_t* r, const cmp_t* a, const cmp_t* b) { mp_add(&r->re, &a->re, &b->re); mp_add(&r->im, &a->im, &b->im); }
void cmp_sub(cmp_t* r, const cmp_t* a, const cmp_t* b) { mp_sub(&r->re, &a->re, &b->re); mp_sub(&r->im, &a->im, &b->im); }
void cmp_mul(cmp_t* r, const cmp_t* a, const cmp_t* b) {
  mp t1, t2, re, im;
  mp_mul(&t1, &a->re, &b->re); mp_mul(&t2, &a->im, &b->im); mp_sub(&re, &t1, &t2);
  mp_mul(&t1, &a->re, &b->im); mp_mul(&t2, &a->im, &b->re); mp_add(&im, &t1, &t2);
  r->re = re; r->im = im;
}
void cmp_mul_conj(cmp_t* r, const cmp_t* a, const cmp_t* b) {
  cmp_t c; c.re = a->re; mp_neg(&c.im, &a->im); cmp_mul(r, &c, b);
}
void cmp_scale(cmp_t* r, const cmp_t* a, const mp* s) { mp_mul(&r->re, &a->re, s); mp_mul(&r->im, &a->im, s); }
void cmp_conj(cmp_t* r, const cmp_t* a) { r->re = a->re; mp_neg(&r->im, &a->im); }
void cmp_abs2(mp* r, const cmp_t* a) { mp t1, t2; mp_mul(&t1, &a->re, &a->re); mp_mul(&t2, &a->im, &a->im); mp_add(r, &t1, &t2); }
