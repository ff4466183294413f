/*
 * ORACLE (test infrastructure only; never part of the product path).
 * Plain 320-bit binary floating point used by the oracle's eigensolver and statevector simulator.
 * value = (-1)^s * (M / 2^(64*MPL)) * 2^e, M = little-endian limbs m[0..MPL-1] with the top bit of
 * m[MPL-1] set (zero: all limbs zero).  Every operation truncates toward zero after keeping one guard
 * limb, so each result is within a few units of 2^-318 relative of the exact one.
 */
#ifndef ORACLE_MP_H
#define ORACLE_MP_H
#include <stdint.h>
#define MPL 5
typedef struct { uint64_t m[MPL]; int64_t e; int s; } mp;
typedef struct { mp re, im; } cmp_t;

void mp_zero(mp* r);
int mp_is_zero(const mp* a);
void mp_from_double(mp* r, double d);
void mp_from_words(mp* r, const double* w, int n);        /* exact sum of n doubles (if span <= 320 bits) */
double mp_to_double(const mp* a);                         /* round to nearest */
void mp_to_words(const mp* a, double* w, int n);          /* successive round-to-nearest expansion */
void mp_add(mp* r, const mp* a, const mp* b);
void mp_sub(mp* r, const mp* a, const mp* b);
void mp_mul(mp* r, const mp* a, const mp* b);
void mp_div(mp* r, const mp* a, const mp* b);
void mp_sqrt(mp* r, const mp* a);
void mp_neg(mp* r, const mp* a);
void mp_abs(mp* r, const mp* a);
void mp_ldexp(mp* r, const mp* a, int64_t k);
int mp_cmp(const mp* a, const mp* b);                     /* sign of a - b */
int mp_cmp_abs(const mp* a, const mp* b);                 /* sign of |a| - |b| */
int mp_sign(const mp* a);                                 /* -1, 0, 1 */

/* complex helpers */
void cmp_zero(cmp_t* r);
void cmp_add(cmp_t* r, const cmp_t* a, const cmp_t* b);
void cmp_sub(cmp_t* r, const cmp_t* a, const cmp_t* b);
void cmp_mul(cmp_t* r, const cmp_t* a, const cmp_t* b);
void cmp_mul_conj(cmp_t* r, const cmp_t* a, const cmp_t* b);  /* conj(a) * b */
void cmp_scale(cmp_t* r, const cmp_t* a, const mp* s);
void cmp_conj(cmp_t* r, const cmp_t* a);
void cmp_abs2(mp* r, const cmp_t* a);
#endif
