// Multi-word floating point built from FP64 error-free transformations (the "multiple-precision"
// arithmetic the paper relies on to keep Schmidt coefficients of size ~2^{-(n-1)/2}, Section 1 and
// its footnote).  A value is an unevaluated sum of W doubles, highest first, kept non-overlapping:
//   W = 1: plain double; W = 2: double-double (~106 bits); W = 4: quad-double (~212 bits).
// Building blocks (Knuth TwoSum, Dekker FastTwoSum, TwoProd through one FMA) and the level-by-level
// accumulation of partial products follow the published descriptions of double-double
// (Dekker 1971; Joldes-Muller-Popescu 2017) and quad-double arithmetic (Hida-Li-Bailey 2001).
// Host-compilable so the same code can be checked on the CPU.
#pragma once
#include <cmath>

#if defined(__CUDACC__)
#define MW_HD __host__ __device__ __forceinline__
#define MW_FMA(a, b, c) fma(a, b, c)
#else
#define MW_HD inline
#define MW_FMA(a, b, c) std::fma(a, b, c)
#endif

namespace zkq {

// ---- error-free transformations --------------------------------------------------------------
MW_HD double two_sum(double a, double b, double& e) {    // a + b = s + e exactly
  double s = a + b;
  double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}
MW_HD double fast_two_sum(double a, double b, double& e) {  // needs exponent(a) >= exponent(b) or a == 0
  double s = a + b;
  e = b - (s - a);
  return s;
}
MW_HD double two_prod(double a, double b, double& e) {   // a * b = p + e exactly (FMA)
  double p = a * b;
  e = MW_FMA(a, b, -p);
  return p;
}
// (a, b, c) -> (s, e1, e2), s + e1 + e2 = a + b + c exactly
MW_HD void three_sum(double& a, double& b, double& c) {
  double t1, t2, t3;
  t1 = two_sum(a, b, t2);
  a = two_sum(c, t1, t3);
  b = two_sum(t2, t3, c);
}
// (a, b, c) -> (s, e) with s + e ~ a + b + c (the second error word is rounded in)
MW_HD void three_sum2(double& a, double& b, double c) {
  double t1, t2, t3;
  t1 = two_sum(a, b, t2);
  a = two_sum(c, t1, t3);
  b = t2 + t3;
}

template <int W> struct mw { double x[W]; };
using dd = mw<2>;
using qd = mw<4>;

// ---- renormalisation ------------------------------------------------------------------------
// five words (any order of magnitude after cancellation) -> four non-overlapping words:
// a bottom-up TwoSum pass (exact regardless of ordering) and a top-down pass.
MW_HD void renorm5(double c0, double c1, double c2, double c3, double c4, double* o) {
  double e;
  c3 = two_sum(c3, c4, c4);
  c2 = two_sum(c2, c3, c3);
  c1 = two_sum(c1, c2, c2);
  c0 = two_sum(c0, c1, c1);
  c1 = two_sum(c1, c2, c2);
  c2 = two_sum(c2, c3, c3);
  c3 = c3 + c4;
  c0 = fast_two_sum(c0, c1, e); c1 = e;
  c1 = fast_two_sum(c1, c2, e); c2 = e;
  c2 = fast_two_sum(c2, c3, e); c3 = e;
  o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

// ---- generic interface ------------------------------------------------------------------------
template <int W> MW_HD mw<W> mw_from(double a) { mw<W> r; r.x[0] = a; for (int k = 1; k < W; ++k) r.x[k] = 0.0; return r; }
template <int W> MW_HD mw<W> mw_zero() { return mw_from<W>(0.0); }
template <int W> MW_HD mw<W> mw_neg(const mw<W>& a) { mw<W> r; for (int k = 0; k < W; ++k) r.x[k] = -a.x[k]; return r; }
template <int W> MW_HD double mw_hi(const mw<W>& a) { return a.x[0]; }
template <int W> MW_HD mw<W> mw_ldexp(const mw<W>& a, int e) { mw<W> r; for (int k = 0; k < W; ++k) r.x[k] = ldexp(a.x[k], e); return r; }

// ---- W = 1 ----
MW_HD mw<1> mw_add(const mw<1>& a, const mw<1>& b) { mw<1> r; r.x[0] = a.x[0] + b.x[0]; return r; }
MW_HD mw<1> mw_mul(const mw<1>& a, const mw<1>& b) { mw<1> r; r.x[0] = a.x[0] * b.x[0]; return r; }
MW_HD mw<1> mw_mul_d(const mw<1>& a, double b) { mw<1> r; r.x[0] = a.x[0] * b; return r; }
MW_HD mw<1> mw_add_d(const mw<1>& a, double b) { mw<1> r; r.x[0] = a.x[0] + b; return r; }
MW_HD mw<1> mw_div(const mw<1>& a, const mw<1>& b) { mw<1> r; r.x[0] = a.x[0] / b.x[0]; return r; }
MW_HD mw<1> mw_sqrt(const mw<1>& a) { mw<1> r; r.x[0] = sqrt(a.x[0]); return r; }
MW_HD mw<1> mw_fma(const mw<1>& a, const mw<1>& b, const mw<1>& c) { mw<1> r; r.x[0] = MW_FMA(a.x[0], b.x[0], c.x[0]); return r; }

// ---- W = 2: double-double ----
MW_HD dd dd_make(double hi, double lo) { dd r; r.x[0] = hi; r.x[1] = lo; return r; }
MW_HD dd mw_add(const dd& a, const dd& b) {          // accurate (both words' errors kept)
  double t1, t2, e1, e2;
  double s1 = two_sum(a.x[0], b.x[0], e1);
  t1 = two_sum(a.x[1], b.x[1], t2);
  e1 += t1;
  s1 = fast_two_sum(s1, e1, e1);
  e1 += t2;
  s1 = fast_two_sum(s1, e1, e2);
  return dd_make(s1, e2);
}
MW_HD dd mw_add_d(const dd& a, double b) {
  double e, s = two_sum(a.x[0], b, e);
  e += a.x[1];
  s = fast_two_sum(s, e, e);
  return dd_make(s, e);
}
MW_HD dd mw_mul(const dd& a, const dd& b) {
  double e, p = two_prod(a.x[0], b.x[0], e);
  e = MW_FMA(a.x[0], b.x[1], e);
  e = MW_FMA(a.x[1], b.x[0], e);
  p = fast_two_sum(p, e, e);
  return dd_make(p, e);
}
MW_HD dd mw_mul_d(const dd& a, double b) {
  double e, p = two_prod(a.x[0], b, e);
  e = MW_FMA(a.x[1], b, e);
  p = fast_two_sum(p, e, e);
  return dd_make(p, e);
}
MW_HD dd mw_div(const dd& a, const dd& b) {           // three-step long division
  double q1 = a.x[0] / b.x[0];
  dd r = mw_add(a, mw_neg(mw_mul_d(b, q1)));
  double q2 = r.x[0] / b.x[0];
  r = mw_add(r, mw_neg(mw_mul_d(b, q2)));
  double q3 = r.x[0] / b.x[0];
  double e;
  q1 = fast_two_sum(q1, q2, e);
  dd s = dd_make(q1, e);
  return mw_add_d(s, q3);
}
MW_HD dd mw_sqrt(const dd& a) {                        // one Newton step from the double root
  if (a.x[0] <= 0.0) return dd_make(0.0, 0.0);
  double x = 1.0 / sqrt(a.x[0]);
  double ax = a.x[0] * x;
  dd ax2 = mw_mul(dd_make(ax, 0.0), dd_make(ax, 0.0));
  double d = mw_add(a, mw_neg(ax2)).x[0] * (x * 0.5);
  double e, s = two_sum(ax, d, e);
  return dd_make(s, e);
}
MW_HD dd mw_fma(const dd& a, const dd& b, const dd& c) { return mw_add(mw_mul(a, b), c); }

// ---- W = 4: quad-double ----
MW_HD qd qd_make(double a, double b, double c, double d) { qd r; r.x[0] = a; r.x[1] = b; r.x[2] = c; r.x[3] = d; return r; }
MW_HD qd mw_add(const qd& a, const qd& b) {
  // level-by-level: TwoSum each pair of words, carry the errors down one level at a time
  double t0, t1, t2, t3;
  double s0 = two_sum(a.x[0], b.x[0], t0);
  double s1 = two_sum(a.x[1], b.x[1], t1);
  double s2 = two_sum(a.x[2], b.x[2], t2);
  double s3 = two_sum(a.x[3], b.x[3], t3);
  s1 = two_sum(s1, t0, t0);                     // level 1 done; t0 -> level 2
  three_sum(s2, t0, t1);                        // level 2: s2; errors t0 -> level 3, t1 -> level 4
  three_sum2(s3, t0, t2);                       // level 3: s3; error t0 -> level 4
  t0 = t0 + t1 + t3;
  qd r; renorm5(s0, s1, s2, s3, t0, r.x);
  return r;
}
MW_HD qd mw_add_d(const qd& a, double b) {
  double e0, e1, e2, e3;
  double s0 = two_sum(a.x[0], b, e0);
  double s1 = two_sum(a.x[1], e0, e1);
  double s2 = two_sum(a.x[2], e1, e2);
  double s3 = two_sum(a.x[3], e2, e3);
  qd r; renorm5(s0, s1, s2, s3, e3, r.x);
  return r;
}
MW_HD qd mw_mul(const qd& a, const qd& b) {
  // partial products grouped by order: O(1): a0b0; O(e): a0b1, a1b0; O(e^2): a0b2, a1b1, a2b0;
  // O(e^3): a0b3, a1b2, a2b1, a3b0 (plain products) plus the TwoProd errors of the O(e^2) terms.
  double q0, q1, q2, q3, q4, q5;
  double p0 = two_prod(a.x[0], b.x[0], q0);
  double p1 = two_prod(a.x[0], b.x[1], q1);
  double p2 = two_prod(a.x[1], b.x[0], q2);
  double p3 = two_prod(a.x[0], b.x[2], q3);
  double p4 = two_prod(a.x[1], b.x[1], q4);
  double p5 = two_prod(a.x[2], b.x[0], q5);
  three_sum(p1, p2, q0);                        // O(e): p1; errors p2, q0 -> O(e^2)
  three_sum(p2, q1, q2);                        // O(e^2) pieces: p2, q1, q2 ...
  three_sum(p3, p4, p5);                        // ... and p3, p4, p5
  double t0, t1;
  double s0 = two_sum(p2, p3, t0);
  double s1 = two_sum(q1, p4, t1);
  double s2 = q2 + p5;
  s1 = two_sum(s1, t0, t0);
  s2 += t0 + t1;
  s1 += a.x[0] * b.x[3] + a.x[1] * b.x[2] + a.x[2] * b.x[1] + a.x[3] * b.x[0] + q0 + q3 + q4 + q5;
  qd r; renorm5(p0, p1, s0, s1, s2, r.x);
  return r;
}
MW_HD qd mw_mul_d(const qd& a, double b) {
  double q0, q1, q2;
  double p0 = two_prod(a.x[0], b, q0);
  double p1 = two_prod(a.x[1], b, q1);
  double p2 = two_prod(a.x[2], b, q2);
  double p3 = a.x[3] * b;
  double s0 = p0;
  double s1 = two_sum(q0, p1, q0);
  double t;
  three_sum(q0, q1, p2);
  double s2 = q0;
  three_sum2(q1, q2, p3);
  double s3 = q1 + p2, s4 = q2;
  (void)t;
  qd r; renorm5(s0, s1, s2, s3, s4, r.x);
  return r;
}
MW_HD qd mw_div(const qd& a, const qd& b) {            // five-step long division
  double q[5];
  qd r = a;
  for (int k = 0; k < 5; ++k) {
    q[k] = r.x[0] / b.x[0];
    if (k < 4) r = mw_add(r, mw_neg(mw_mul_d(b, q[k])));
  }
  qd o; renorm5(q[0], q[1], q[2], q[3], q[4], o.x);
  return o;
}
MW_HD qd mw_sqrt(const qd& a) {                        // Newton on 1/sqrt(a), three steps, then a * y
  if (a.x[0] <= 0.0) return qd_make(0, 0, 0, 0);
  qd y = qd_make(1.0 / sqrt(a.x[0]), 0, 0, 0);
  for (int it = 0; it < 3; ++it) {
    qd t = mw_mul(a, mw_mul(y, y));                   // a y^2
    t = mw_add_d(mw_neg(t), 1.0);                     // 1 - a y^2
    y = mw_add(y, mw_mul_d(mw_mul(y, t), 0.5));
  }
  qd s = mw_mul(a, y);
  qd d = mw_add(a, mw_neg(mw_mul(s, s)));              // correction s + (a - s^2) y / 2
  return mw_add(s, mw_mul_d(mw_mul(d, y), 0.5));
}
MW_HD qd mw_fma(const qd& a, const qd& b, const qd& c) { return mw_add(mw_mul(a, b), c); }

template <int W> MW_HD mw<W> mw_sub(const mw<W>& a, const mw<W>& b) { return mw_add(a, mw_neg(b)); }
template <int W> MW_HD mw<W> mw_abs(const mw<W>& a) { return a.x[0] < 0 ? mw_neg(a) : a; }
template <int W> MW_HD mw<W> mw_recip(const mw<W>& a) { return mw_div(mw_from<W>(1.0), a); }

// round a longer expansion (K words) into W words
template <int W, int K> MW_HD mw<W> mw_from_words(const double* w) {
  mw<W> r = mw_from<W>(w[0]);
  if constexpr (W >= K) {
    for (int k = 1; k < K; ++k) r.x[k] = w[k];
  } else {
    for (int k = 1; k < K; ++k) r = mw_add_d(r, w[k]);
  }
  return r;
}

// ---- complex ---------------------------------------------------------------------------------
template <int W> struct cmw { mw<W> re, im; };
template <int W> MW_HD cmw<W> c_make(const mw<W>& re, const mw<W>& im) { cmw<W> z; z.re = re; z.im = im; return z; }
template <int W> MW_HD cmw<W> c_zero() { return c_make(mw_zero<W>(), mw_zero<W>()); }
template <int W> MW_HD cmw<W> c_add(const cmw<W>& a, const cmw<W>& b) { return c_make(mw_add(a.re, b.re), mw_add(a.im, b.im)); }
template <int W> MW_HD cmw<W> c_sub(const cmw<W>& a, const cmw<W>& b) { return c_make(mw_sub(a.re, b.re), mw_sub(a.im, b.im)); }
template <int W> MW_HD cmw<W> c_conj(const cmw<W>& a) { return c_make(a.re, mw_neg(a.im)); }
template <int W> MW_HD cmw<W> c_mul(const cmw<W>& a, const cmw<W>& b) {
  return c_make(mw_sub(mw_mul(a.re, b.re), mw_mul(a.im, b.im)), mw_add(mw_mul(a.re, b.im), mw_mul(a.im, b.re)));
}
template <int W> MW_HD cmw<W> c_mul_conj(const cmw<W>& a, const cmw<W>& b) {   // conj(a) * b
  return c_make(mw_add(mw_mul(a.re, b.re), mw_mul(a.im, b.im)), mw_sub(mw_mul(a.re, b.im), mw_mul(a.im, b.re)));
}
template <int W> MW_HD cmw<W> c_scale(const cmw<W>& a, const mw<W>& s) { return c_make(mw_mul(a.re, s), mw_mul(a.im, s)); }
template <int W> MW_HD cmw<W> c_scale_d(const cmw<W>& a, double s) { return c_make(mw_mul_d(a.re, s), mw_mul_d(a.im, s)); }
template <int W> MW_HD mw<W> c_abs2(const cmw<W>& a) { return mw_add(mw_mul(a.re, a.re), mw_mul(a.im, a.im)); }
template <int W> MW_HD cmw<W> c_div(const cmw<W>& a, const cmw<W>& b) {
  mw<W> d = c_abs2(b);
  cmw<W> n = c_mul_conj(b, a);                        // conj(b) a
  return c_make(mw_div(n.re, d), mw_div(n.im, d));
}

// element I/O in the library layout: element e holds re words then im words
template <int W, int K> MW_HD cmw<W> c_load(const double* p, size_t e) {
  const double* q = p + e * 2 * K;
  return c_make(mw_from_words<W, K>(q), mw_from_words<W, K>(q + K));
}
template <int W> MW_HD void c_store(double* p, size_t e, const cmw<W>& z) {
  double* q = p + e * 2 * W;
  for (int k = 0; k < W; ++k) { q[k] = z.re.x[k]; q[W + k] = z.im.x[k]; }
}
template <int W> MW_HD void mw_store(double* p, size_t i, const mw<W>& v) { for (int k = 0; k < W; ++k) p[i * W + k] = v.x[k]; }
template <int W, int K> MW_HD mw<W> mw_load(const double* p, size_t i) { return mw_from_words<W, K>(p + i * K); }

}  // namespace zkq
