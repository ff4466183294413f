// Precision recovery by block Ogita-Aishima refinement (Ogita & Aishima 2018; clustered eigenvalues:
// Ogita & Aishima 2019), the build's chosen form of the paper's precision-recovery step (Section 2,
// ZKCM_CUS paragraph).  With X the current eigenvector matrix (target precision, W words per real):
//   P = A X,  S = X^H P,  R = I - X^H X                                  (split products, ozaki.cu)
//   lambda_i = s_ii / (1 - r_ii)
//   delta = 2 (||S - diag(lambda)||_F + ||A|| ||R||_F)   (used here in a local form, oa_cluster_kernel)
//   e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)   if |lambda_i - lambda_j| > delta
//   e_ij = r_ij / 2                                         otherwise (and on the diagonal)
//   X <- X + X E
// (E is evaluated as R/2 plus an exactly anti-Hermitian part, see oa_E_kernel.)
// Columns stay sorted by eigenvalue, so a cluster is a maximal run of consecutive columns whose
// neighbouring lambdas are within delta.  A cluster J whose block S_JJ is not yet diagonal is separated
// after the update: T = X_J^H (A - mu I) X_J is formed from the updated X (mu = mean lambda over J), rounded
// to FP64, diagonalised with the FP64 Jacobi kernel, and X_J <- X_J W.  For spectra graded far below 2^-53 ||A|| each pass resolves
// about 53 more bits of the small eigenvalues.  E only needs double-double: its entries are of the size of
// the current error, so their relative accuracy requirement is at most ~106 bits.
// A problem is converged once every coupling |s_ij + (lambda_i + lambda_j)/2 r_ij| <= 2^-(53W-6) ||A||
// (E itself can stay at noise / gap for near-degenerate pairs); after one more ordinary iteration it takes
// re-orthonormalising steps (E = R/2) until |r_ij| <= 2^-(53W-10), and lambda, X of the following
// evaluation are reported.
#include <vector>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include "common.cuh"
#include "mw.cuh"
#include "reduce.cuh"
#include "ozaki.cuh"
#include "prof.cuh"
#include "internal.cuh"

namespace zkq {

struct OaProb {
  int n; int64_t xoff;         // element offset of the problem's n x n matrices in X, P, S, R, E
  int64_t loff;                // offset (in eigenpairs) of lambda, cluster arrays
  int64_t a_off;               // element offset of A, V, V_out
};

// ---- X <- promote(V) -------------------------------------------------------------------------
template <int W>
__global__ void oa_init_kernel(const OaProb* __restrict__ pr, const double* __restrict__ V, double* __restrict__ X) {
  const OaProb p = pr[blockIdx.y];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.n * p.n) return;
  const double* v = V + (p.a_off + e) * 2;
  c_store(X + p.xoff * 2 * W, e, c_make(mw_from<W>(v[0]), mw_from<W>(v[1])));
}

// ---- per-problem statistics: lambda, couplings, clusters ----------------------------------------
struct OaStat { double maxE; double delta; double anorm; int nclusters; int clustered; double cl_off; double maxNum; double maxR; };

// lambda_i = s_ii / (1 - r_ii); anorm = max |lambda|; reset the per-iteration accumulators
template <int W>
__global__ void __launch_bounds__(256) oa_lambda_kernel(const OaProb* __restrict__ pr, const double* __restrict__ S,
                                                        const double* __restrict__ R, double* __restrict__ lam,
                                                        double* __restrict__ colnum, OaStat* __restrict__ st) {
  const OaProb p = pr[blockIdx.x];
  const int n = p.n, tid = threadIdx.x;
  __shared__ double sbuf[32];
  const double* Sb = S + p.xoff * 2 * W;
  const double* Rb = R + p.xoff * 2 * W;
  double* lb = lam + p.loff * W;
  double amax = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    mw<W> sv = c_load<W, W>(Sb, (size_t)i + (size_t)i * n).re;
    mw<W> rv = c_load<W, W>(Rb, (size_t)i + (size_t)i * n).re;
    mw<W> l = mw_div(sv, mw_add_d(mw_neg(rv), 1.0));
    mw_store(lb, i, l);
    amax = fmax(amax, fabs(l.x[0]));
    colnum[p.loff + i] = 0.0;
  }
  amax = block_max_d(amax, sbuf);
  if (tid == 0) {
    OaStat z; z.maxE = 0; z.delta = 0; z.anorm = amax; z.nclusters = 0; z.clustered = 0; z.cl_off = 0; z.maxNum = 0; z.maxR = 0;
    st[blockIdx.x] = z;
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* a, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// couplings num_ij = s_ij + (lambda_i + lambda_j)/2 r_ij (i != j): first-order insensitive to the
// non-orthonormality of X, (lambda_i - lambda_j)/2 times the rotation error of the pair.  Accumulates
// column norms ||num_{:,c}||^2, max |num| and max |r|.
// The column sums go through shared memory first (a block of 256 consecutive elements touches at most
// 256/n + 2 columns), then one global atomic per touched column.
template <int W>
__global__ void __launch_bounds__(256) oa_coupling_kernel(const OaProb* __restrict__ pr, const double* __restrict__ S,
                                                          const double* __restrict__ R, const double* __restrict__ lam,
                                                          double* __restrict__ colnum, double* __restrict__ NUM,
                                                          OaStat* __restrict__ st) {
  __shared__ double csum[258];
  const OaProb p = pr[blockIdx.y];
  const int e0 = blockIdx.x * blockDim.x;
  if (e0 >= p.n * p.n) return;                         // whole block past this problem
  const int j0 = e0 / p.n;
  const int jn = min(p.n - 1, (e0 + (int)blockDim.x - 1) / p.n) - j0 + 1;   // columns touched (<= 258)
  for (int t = threadIdx.x; t < jn; t += blockDim.x) csum[t] = 0.0;
  __syncthreads();
  int e = e0 + threadIdx.x;
  double cpl = 0.0, rmag = 0.0;
  if (e < p.n * p.n) {
    const int n = p.n, i = e % n, j = e / n;
    cmw<W> r = c_load<W, W>(R + p.xoff * 2 * W, e);
    rmag = hypot(r.re.x[0], r.im.x[0]);
    cmw<2> num2 = c_zero<2>();
    if (i != j) {
      cmw<W> sv = c_load<W, W>(S + p.xoff * 2 * W, e);
      const double* lw = lam + p.loff * W;
      // num is needed to an absolute 2^-(53 W) ||A|| (the residual it leaves is about its error).  When
      // both terms are below 2^-(53 W - 100) ||A||, double-double (relative error about 2^-104) already
      // reaches that, whatever the cancellation; otherwise the sum takes the working precision.
      bool dd = false;
      if constexpr (W > 2) {
        const double hm = 0.5 * fabs(lw[(size_t)i * W] + lw[(size_t)j * W]);
        const double mag = fmax(fmax(fabs(sv.re.x[0]), fabs(sv.im.x[0])), hm * fmax(fabs(r.re.x[0]), fabs(r.im.x[0])));
        dd = mag <= ldexp(st[blockIdx.y].anorm, -(53 * W - 100));
      }
      if (dd) {
        // the two leading words of a normalised expansion are a double-double within 2^-105 of it
        auto lead2 = [](const double* w) { mw<2> t; t.x[0] = w[0]; t.x[1] = w[1]; return t; };
        const cmw<2> s2 = c_make(lead2(sv.re.x), lead2(sv.im.x));
        const cmw<2> r2 = c_make(lead2(r.re.x), lead2(r.im.x));
        const mw<2> h2 = mw_mul_d(mw_add(lead2(lw + (size_t)i * W), lead2(lw + (size_t)j * W)), 0.5);
        num2 = c_add(s2, c_scale(r2, h2));
        cpl = hypot(num2.re.x[0], num2.im.x[0]);
      } else {
        mw<W> hs = mw_mul_d(mw_add(mw_load<W, W>(lw, i), mw_load<W, W>(lw, j)), 0.5);
        cmw<W> num = c_add(sv, c_scale(r, hs));     // cancellation-sensitive: working precision
        cpl = hypot(num.re.x[0], num.im.x[0]);
        num2 = c_make(mw_from_words<2, W>(num.re.x), mw_from_words<2, W>(num.im.x));
      }
      if (cpl > 0) atomicAdd(&csum[j - j0], cpl * cpl);
    }
    c_store(NUM + p.xoff * 2 * 2, e, num2);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < jn; t += blockDim.x)
    if (csum[t] > 0) atomicAdd(&colnum[p.loff + j0 + t], csum[t]);
  for (int o = 16; o > 0; o >>= 1) {
    cpl = fmax(cpl, __shfl_down_sync(0xffffffffu, cpl, o));
    rmag = fmax(rmag, __shfl_down_sync(0xffffffffu, rmag, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (cpl > 0) atomic_max_nonneg(&st[blockIdx.y].maxNum, cpl);
    if (rmag > 0) atomic_max_nonneg(&st[blockIdx.y].maxR, rmag);
  }
}

// clusters: consecutive columns c, c+1 stay together while
//   |lambda_c - lambda_{c+1}| <= delta_c = g (||num_{:,c}|| + ||num_{:,c+1}||) + 2^-(53W/2+4) max(|lambda_c|, |lambda_{c+1}|),
// a local version of the Ogita-Aishima threshold: the couplings bound the eigenvalue errors of the two
// columns, so a non-orthonormality confined to tiny-eigenvalue columns cannot merge the whole spectrum.
// The margin g = 2^16 keeps every rotation k = num / gap outside the clusters below 2^-16: the first-order
// update X + X K then leaves non-orthonormality k^H k < 2^-32, and the iteration stays in its quadratic
// regime (with g = 2, k reached 1/4 and the first iterations made little progress).  Measured on the
// 256-problem quad-double batch, the refinement took 5.86, 5.53, 5.41, 5.38 and 5.45 s for g = 2^7, 2^10,
// 2^13, 2^16 and 2^20: a wider margin makes the clusters a few columns larger but the separated pairs
// converge in fewer iterations.
// The relative floor keeps pairs closer than ~2^-(53W/2) apart together: for them the computed coupling
// (noise ~2^-53W |lambda|) over the gap would give rotations k whose second-order term k^H k exceeds the
// working precision; the cluster step (exactly unitary rotation) separates them instead.
constexpr double kClusterMargin = 65536.0;

template <int W>
__global__ void oa_cluster_kernel(const OaProb* __restrict__ pr, const double* __restrict__ lam,
                                  const double* __restrict__ colnum, int32_t* __restrict__ cl_start,
                                  int32_t* __restrict__ cl_len, OaStat* __restrict__ st, double margin) {
  const OaProb p = pr[blockIdx.x];
  if (threadIdx.x != 0) return;
  const int n = p.n;
  const double* lb = lam + p.loff * W;
  const double floor_rel = ldexp(1.0, -(53 * W / 2 + 4));
  int ncl = 0, clustered = 0, start = 0;
  double dmax = 0.0;
  for (int i = 1; i <= n; ++i) {
    bool brk = (i == n);
    if (!brk) {
      mw<W> a = mw_load<W, W>(lb, i - 1), b = mw_load<W, W>(lb, i);
      double gap = fabs(mw_sub(a, b).x[0]);
      double d = margin * (sqrt(colnum[p.loff + i - 1]) + sqrt(colnum[p.loff + i])) +
                 floor_rel * fmax(fabs(a.x[0]), fabs(b.x[0]));
      dmax = fmax(dmax, d);
      brk = gap > d;
    }
    if (brk) {
      int len = i - start;
      for (int c = start; c < i; ++c) { cl_start[p.loff + c] = start; cl_len[p.loff + c] = len; }
      if (len > 1) { ++ncl; clustered += len; }
      start = i;
    }
  }
  st[blockIdx.x].delta = dmax;
  st[blockIdx.x].nclusters = ncl;
  st[blockIdx.x].clustered = clustered;
}

// ---- E (double-double) -----------------------------------------------------------------------------
// E = R/2 + K with K anti-Hermitian:  k_ij = (s_ij + (lambda_i + lambda_j)/2 r_ij) / (lambda_j - lambda_i)
// for separated pairs (the Ogita-Aishima e_ij minus r_ij/2), k_ij = 0 inside clusters.  k is evaluated
// once per unordered pair from the upper-triangle entries (i < j) and mirrored as k_ji = -conj(k_ij), so
// E + E^H = R holds to rounding even where the computed S carries noise / gap for near-degenerate pairs;
// that noise then only rotates inside the pair's span.
template <int W>
__global__ void oa_E_kernel(const OaProb* __restrict__ pr, const double* __restrict__ NUM, const double* __restrict__ R,
                            const double* __restrict__ lam, const int32_t* __restrict__ cl_start,
                            const int32_t* __restrict__ orth_only, double* __restrict__ E, OaStat* __restrict__ st) {
  const OaProb p = pr[blockIdx.y];
  const bool no_rot = orth_only[blockIdx.y] != 0;     // polishing step: E = R/2 (orthonormalisation only)
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  double mag = 0.0, cpl = 0.0, rmag = 0.0, incl = 0.0;
  if (e < p.n * p.n) {
    const int n = p.n, i = e % n, j = e / n;
    const int a = i < j ? i : j, b = i < j ? j : i;           // upper-triangle representative (a, b)
    const size_t eu = (size_t)a + (size_t)b * n;
    // the two leading words of a normalised expansion are a double-double within 2^-105 of it
    auto lead2 = [](const double* w) { mw<2> t; t.x[0] = w[0]; t.x[1] = w[1]; return t; };
    const double* rp = R + (p.xoff + eu) * 2 * W;
    const cmw<2> r2 = c_make(lead2(rp), lead2(rp + W));
    rmag = hypot(rp[0], rp[W]);
    cmw<2> out;
    if (i == j) {
      out = c_scale_d(r2, 0.5);
      out.im = mw_zero<2>();
      rmag = fabs(rp[0]);
    } else {
      // coupling num_ab (gap-free), evaluated in working precision by the coupling pass, kept as DD
      cmw<2> n2 = c_load<2, 2>(NUM + p.xoff * 2 * 2, eu);
      cpl = hypot(n2.re.x[0], n2.im.x[0]);
      cmw<2> k = c_zero<2>();
      if (cl_start[p.loff + a] == cl_start[p.loff + b]) {
        incl = cpl;
      } else if (!no_rot) {
        // gap lambda_b - lambda_a: in double-double when its error (2^-104 max|lambda| at most) moves
        // k (gap) = num by less than 2^-(53 W + 2) ||A||, else in the working precision
        const double* lw = lam + p.loff * W;
        mw<2> den2 = mw_sub(lead2(lw + (size_t)b * W), lead2(lw + (size_t)a * W));
        if constexpr (W > 2) {
          const double lmax = fmax(fabs(lw[(size_t)a * W]), fabs(lw[(size_t)b * W]));
          const double margin = fabs(den2.x[0]) - ldexp(lmax, -103);
          if (!(margin > 0 && cpl * ldexp(lmax, -104) <= ldexp(st[blockIdx.y].anorm, -(53 * W + 2)) * margin)) {
            const mw<W> den = mw_sub(mw_load<W, W>(lw, b), mw_load<W, W>(lw, a));
            den2 = lead2(den.x);
          }
        }
        k = c_scale(n2, mw_recip(den2));
      }
      cmw<2> half_r = c_scale_d(r2, 0.5);
      if (i < j) out = c_add(half_r, k);                       // e_ab = r_ab/2 + k_ab
      else out = c_sub(c_conj(half_r), c_conj(k));             // e_ba = conj(r_ab)/2 - conj(k_ab)
    }
    c_store(E + p.xoff * 2 * 2, e, out);
    mag = fmax(fabs(out.re.x[0]), fabs(out.im.x[0]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mag = fmax(mag, __shfl_down_sync(0xffffffffu, mag, o));
    cpl = fmax(cpl, __shfl_down_sync(0xffffffffu, cpl, o));
    rmag = fmax(rmag, __shfl_down_sync(0xffffffffu, rmag, o));
    incl = fmax(incl, __shfl_down_sync(0xffffffffu, incl, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mag > 0) atomic_max_nonneg(&st[blockIdx.y].maxE, mag);
    if (incl > 0) atomic_max_nonneg(&st[blockIdx.y].cl_off, incl);
  }
}

// ---- cluster blocks: T = X_J^H (A - mu I) X_J  (FP64), from the updated X ---------------------------
struct OaCluster { int prob; int start; int len; int64_t toff; int64_t woff; };

// CT = X_J^H A X_J and CG = X_J^H X_J (W words, len x len at toff) were formed by split products from the
// updated X, so the components of X_J outside the cluster are second order and do not blur the small
// splittings; mu = mean of the current lambdas over J.
// mu of every cluster (one thread per cluster)
template <int W>
__global__ void oa_cluster_mu_kernel(const OaProb* __restrict__ pr, const OaCluster* __restrict__ cl, int ncl,
                                     const double* __restrict__ lam, double* __restrict__ MU) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncl) return;
  const OaCluster c = cl[k];
  const OaProb p = pr[c.prob];
  mw<W> mu = mw_zero<W>();
  for (int q = 0; q < c.len; ++q) mu = mw_add(mu, mw_load<W, W>(lam + p.loff * W, c.start + q));
  mw_store(MU, k, mw_mul_d(mu, 1.0 / c.len));
}

template <int W>
__global__ void oa_cluster_T_kernel(const OaProb* __restrict__ pr, const OaCluster* __restrict__ cl,
                                    const double* __restrict__ CT, const double* __restrict__ CG,
                                    const double* __restrict__ MU, double* __restrict__ T) {
  const OaCluster c = cl[blockIdx.y];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c.len * c.len) return;
  int a = e % c.len, b = e / c.len;
  const mw<W> mu = mw_load<W, W>(MU, blockIdx.y);
  cmw<W> t = c_load<W, W>(CT + c.toff * 2 * W, e);
  cmw<W> g = c_load<W, W>(CG + c.toff * 2 * W, e);
  t = c_sub(t, c_scale(g, mu));
  T[(c.toff + e) * 2 + 0] = t.re.x[0] + (W > 1 ? t.re.x[1] : 0.0);
  T[(c.toff + e) * 2 + 1] = a == b ? 0.0 : t.im.x[0] + (W > 1 ? t.im.x[1] : 0.0);
}

// W (FP64 Jacobi eigenvectors of a cluster block) promoted to W words
template <int W>
__global__ void oa_promote_kernel(const OaCluster* __restrict__ cl, const double* __restrict__ V64, double* __restrict__ Wm) {
  const OaCluster c = cl[blockIdx.y];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c.len * c.len) return;
  const double* v = V64 + (c.toff + e) * 2;
  c_store(Wm + c.toff * 2 * W, e, c_make(mw_from<W>(v[0]), mw_from<W>(v[1])));
}
// out = coef R (+ I): the terms of the polar (Loewdin) factor (X^H X)^{-1/2} = (I - R)^{-1/2} of a finishing
// problem, evaluated by Horner's rule in R (see oa_refine_t); one grid row per listed problem
template <int W>
__global__ void oa_polar_term_kernel(const OaProb* __restrict__ pr, const double* __restrict__ R, double* __restrict__ out,
                                     double coef, int add_identity) {
  const OaProb p = pr[blockIdx.y];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.n * p.n) return;
  cmw<W> v = c_scale_d(c_load<W, W>(R + p.xoff * 2 * W, e), coef);
  if (add_identity && e % p.n == e / p.n) v.re = mw_add_d(v.re, 1.0);
  c_store(out + p.xoff * 2 * W, e, v);
}

// copy rotated cluster columns (from Y = old X buffer) back into X
template <int W>
__global__ void oa_cluster_copy_kernel(const OaProb* __restrict__ pr, const OaCluster* __restrict__ cl,
                                       const double* __restrict__ Y, double* __restrict__ X) {
  const OaCluster c = cl[blockIdx.y];
  const OaProb p = pr[c.prob];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.n * c.len) return;
  size_t idx = (size_t)c.start * p.n + e;
  const double* s = Y + (p.xoff + idx) * 2 * W;
  double* d = X + (p.xoff + idx) * 2 * W;
  for (int k = 0; k < 2 * W; ++k) d[k] = s[k];
}

// ---- output: sort, phase, residual estimate --------------------------------------------------------
template <int W>
__device__ __forceinline__ bool mw_greater(const mw<W>& a, const mw<W>& b) {
  mw<W> d = mw_sub(a, b);
  return d.x[0] > 0.0;
}

// One warp per output column c (8 per block): rank of lambda_c (descending, ties by index), residual
// estimate ||P_c - lambda_c X_c|| / ||A|| (the residual in W words, its norm in double), and X_c with its
// first largest-modulus component made real and positive, written to column `rank`.  Lanes stride the
// rows, so the column reads and writes are coalesced.
template <int W>
__global__ void __launch_bounds__(256) oa_output_kernel(const OaProb* __restrict__ pr, const int32_t* __restrict__ which,
                                                        const double* __restrict__ X, const double* __restrict__ P,
                                                        const double* __restrict__ lam, const OaStat* __restrict__ st,
                                                        double* __restrict__ W_out, double* __restrict__ V_out,
                                                        double* __restrict__ err) {
  const int b = which[blockIdx.y];
  const OaProb p = pr[b];
  const int n = p.n;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= n) return;                                  // whole warps leave
  const double* lb = lam + p.loff * W;
  const double anorm = fmax(st[b].anorm, 1e-300);
  const mw<W> lc = mw_load<W, W>(lb, c);
  int rank = 0;
  for (int d = lane; d < n; d += 32) {
    if (d == c) continue;
    mw<W> df = mw_sub(mw_load<W, W>(lb, d), lc);
    rank += (df.x[0] > 0.0) || (df.x[0] == 0.0 && d < c);
  }
  const double* xc = X + (p.xoff + (size_t)c * n) * 2 * W;
  const double* pc = P + (p.xoff + (size_t)c * n) * 2 * W;
  int best = n; double bm = -1.0, rr = 0.0;
  for (int r = lane; r < n; r += 32) {
    const double m2 = xc[r * 2 * W] * xc[r * 2 * W] + xc[r * 2 * W + W] * xc[r * 2 * W + W];
    if (m2 > bm) { bm = m2; best = r; }                // rows ascend per lane: the first largest
    cmw<W> res = c_sub(c_load<W, W>(pc, r), c_scale(c_load<W, W>(xc, r), lc));
    rr += res.re.x[0] * res.re.x[0] + res.im.x[0] * res.im.x[0];
  }
  for (int o = 16; o > 0; o >>= 1) {
    rank += __shfl_xor_sync(0xffffffffu, rank, o);
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    const double obm = __shfl_xor_sync(0xffffffffu, bm, o);
    const int obest = __shfl_xor_sync(0xffffffffu, best, o);
    if (obm > bm || (obm == bm && obest < best)) { bm = obm; best = obest; }
  }
  if (lane == 0) {
    mw_store(W_out, p.loff + rank, lc);
    err[p.loff + rank] = sqrt(rr) / anorm;
  }
  const cmw<W> xb = c_load<W, W>(xc, best);
  const mw<W> mag = mw_sqrt(c_abs2(xb));
  const cmw<W> ph = c_make(mw_div(xb.re, mag), mw_neg(mw_div(xb.im, mag)));
  double* vo = V_out + (p.a_off + (size_t)rank * n) * 2 * W;
  for (int r = lane; r < n; r += 32) {
    cmw<W> v = c_mul(c_load<W, W>(xc, r), ph);
    if (r == best) v.im = mw_zero<W>();
    c_store(vo, r, v);
  }
}

// --------------------------------------------------------------------------------------------------

static size_t alg(size_t x) { return (x + 255) & ~(size_t)255; }

// ZKQ_DEBUG=1 in the environment prints per-iteration refinement statistics to stderr
static bool debug_log() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("ZKQ_DEBUG"); v = (e && e[0] == '1') ? 1 : 0; }
  return v == 1;
}

static zkq_status grow_buf(void** p, size_t* have, size_t need) {
  if (need <= *have) return ZKQ_OK;
  if (*p) { cudaFree(*p); *p = nullptr; *have = 0; }
  size_t want = std::max(need + need / 8, (size_t)1 << 20);
  cudaError_t e = cudaMalloc(p, want);
  if (e != cudaSuccess) { set_last_cuda_error(e); *p = nullptr; return ZKQ_ENOMEM; }
  *have = want;
  return ZKQ_OK;
}

// Bytes of the refinement state that oa_refine_t lays out for a batch (the same regions in the same order,
// each rounded to 256 bytes): xe = sum n^2 elements, le = sum n eigenpairs, W words per real.
size_t oa_state_bytes(int batch, int64_t xe, int64_t le, int W) {
  const size_t mat = (size_t)xe * 2 * W * sizeof(double);
  const size_t ddm = (size_t)xe * 2 * 2 * sizeof(double), fp = (size_t)xe * 2 * sizeof(double);
  size_t off = 0;
  for (size_t b : {mat, mat, mat, mat, mat, ddm,                                   // X, X2, P, S, R, E
                   (size_t)le * W * sizeof(double), (size_t)le * 4, (size_t)le * 4,   // lambda, cluster starts, lengths
                   sizeof(OaStat) * batch, sizeof(OaProb) * batch, sizeof(int32_t) * batch,
                   fp, (size_t)le * sizeof(double), fp, (size_t)le * sizeof(int32_t),   // T, its eigenpairs, info
                   sizeof(OaCluster) * le, mat, mat, mat,                               // clusters, CT, CG, CW
                   (size_t)le * sizeof(double), sizeof(int32_t) * batch,                 // coupling norms, flags
                   (size_t)le * W * sizeof(double), ddm})                                // cluster means, couplings
    off += alg(b);
  return off;
}

// Bytes of the kept residue planes of A (one entry per problem, at the modulus count of the largest order):
// nothing unless the products take the CRT form
size_t oa_cache_bytes(int batch, const int32_t* n, int W, int prod_method) {
  if (prod_method != 1 || batch <= 0) return 0;
  int nmax = 0;
  for (int b = 0; b < batch; ++b) nmax = std::max(nmax, n[b]);
  const int r = crt_moduli(nmax, 53 * W + 6);
  if (r == 0) return 0;
  size_t total = 0;
  for (int b = 0; b < batch; ++b) total += plane_cache_entry_bytes(n[b], n[b], r);
  return total;
}

// Terms k (1..4) of the series (I - R)^{-1/2} = I + R/2 + 3R^2/8 + 5R^3/16 + 35R^4/128 + ... needed for the
// polar factor of an n x n matrix with non-orthonormality max|r_ij| = maxR: with ||R||_2 <= n maxR, the first
// dropped term is below (n maxR)^(k+1), which must be below 2^-(53W - 8); 0 when more than four terms would
// be needed (the problem then takes orthonormalising steps E = R/2 instead).
static int polar_term_count(double maxR, int n, int W) {
  const double lim = ldexp(1.0, -(53 * W - 8));
  const double r = maxR * n;
  double pw = r;
  for (int k = 1; k <= 4; ++k) {
    pw *= r;
    if (pw <= lim) return k;
  }
  return 0;
}

// device bytes grow_buf holds after growing to `need` bytes from nothing
size_t oa_grow_bytes(size_t need) { return std::max(need + need / 8, (size_t)1 << 20); }

template <int W>
zkq_status oa_refine_t(void* ctx, const OaBuffers& buf, int batch, const int32_t* n, const int64_t* a_off,
                       const double* A, int wa, const double* V, double* W_out, double* V_out, double* err,
                       int32_t* info, int max_iter, int prod_method, cudaStream_t st) {
  std::vector<OaProb> probs(batch);
  int64_t xe = 0, le = 0; int nmax = 0;
  for (int b = 0; b < batch; ++b) {
    probs[b] = {n[b], xe, le, a_off[b]};
    xe += (int64_t)n[b] * n[b]; le += n[b]; nmax = std::max(nmax, n[b]);
  }
  const size_t mat = (size_t)xe * 2 * W * sizeof(double);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += alg(bytes); return o; };
  size_t oX = take(mat), oX2 = take(mat), oP = take(mat), oS = take(mat), oR = take(mat);
  size_t oE = take((size_t)xe * 2 * 2 * sizeof(double));
  size_t oL = take((size_t)le * W * sizeof(double));
  size_t oCS = take((size_t)le * 4), oCL = take((size_t)le * 4);
  size_t oST = take(sizeof(OaStat) * batch);
  size_t oPR = take(sizeof(OaProb) * batch);
  size_t oWH = take(sizeof(int32_t) * batch);
  size_t oT = take((size_t)xe * 2 * sizeof(double));          // cluster T blocks (FP64), bounded by sum n^2
  size_t oTW = take((size_t)le * sizeof(double));              // cluster eigenvalues
  size_t oTV = take((size_t)xe * 2 * sizeof(double));         // cluster eigenvectors
  size_t oTI = take((size_t)le * sizeof(int32_t));
  size_t oCLD = take(sizeof(OaCluster) * le);
  size_t oCT = take(mat), oCG = take(mat), oCW = take(mat);   // cluster blocks X_J^H A X_J, X_J^H X_J; rotation
  size_t oCN = take((size_t)le * sizeof(double));              // column coupling norms
  size_t oOO = take(sizeof(int32_t) * batch);                  // per active problem: orthonormalise only
  size_t oMU = take((size_t)le * W * sizeof(double));           // cluster means
  size_t oNUM = take((size_t)xe * 2 * 2 * sizeof(double));      // couplings (double-double)
  // residue planes of A, which every iteration's P = A X and cluster products A X_J take as their left
  // operand: split once and kept for the whole refinement (CRT form)
  const size_t cache_bytes = oa_cache_bytes(batch, n, W, prod_method);
  size_t oPC = take(cache_bytes);
  // and those of X^H, shared within an iteration by R = I - X^H X (first call) and S = X^H P (second call)
  size_t oXC = take(cache_bytes);
  zkq_status s = grow_buf(buf.ws, buf.ws_bytes, off);
  if (s != ZKQ_OK) return s;
  char* base = (char*)*buf.ws;
  PlaneCache pcache, xcache;
  pcache.buf = base + oPC; pcache.bytes = cache_bytes;
  xcache.buf = base + oXC; xcache.bytes = cache_bytes;
  double *X = (double*)(base + oX), *X2 = (double*)(base + oX2), *Pm = (double*)(base + oP), *Sm = (double*)(base + oS),
         *Rm = (double*)(base + oR), *Em = (double*)(base + oE), *Lm = (double*)(base + oL);
  int32_t *CS = (int32_t*)(base + oCS), *CL = (int32_t*)(base + oCL), *WH = (int32_t*)(base + oWH), *TI = (int32_t*)(base + oTI);
  OaStat* ST = (OaStat*)(base + oST);
  OaProb* PR = (OaProb*)(base + oPR);
  double *T = (double*)(base + oT), *TW = (double*)(base + oTW), *TV = (double*)(base + oTV);
  OaCluster* CLD = (OaCluster*)(base + oCLD);
  double *CT = (double*)(base + oCT), *CG = (double*)(base + oCG), *CW = (double*)(base + oCW);
  double* CN = (double*)(base + oCN);
  int32_t* OO = (int32_t*)(base + oOO);
  double* MUb = (double*)(base + oMU);
  double* NUM = (double*)(base + oNUM);
  HostStage& hs = *buf.stage;
  ZKQ_CUDA_TRY(hs.upload(PR, probs.data(), sizeof(OaProb) * batch, st));
  ZKQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t) * batch, st));
  {
    dim3 g((nmax * nmax + 255) / 256, batch);
    { ProfScope ps_(PC_OA, st); oa_init_kernel<W><<<g, 256, 0, st>>>(PR, V, X); }
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  const double tol = ldexp(1.0, -(53 * W - 6));
  std::vector<int> active(batch, 1), polish(batch, 0), iters(batch, 0), orth_steps(batch, 0), near_conv(batch, 0);
  std::vector<OaStat> hst(batch);
  std::vector<int32_t> hcl_len(le);
  const int p_bits = 53 * W + 6;
  for (int it = 0; it <= max_iter; ++it) {
    std::vector<int> act;
    for (int b = 0; b < batch; ++b) if (active[b]) act.push_back(b);
    if (act.empty()) break;
    // P = A X ; S = X^H P ; R = I - X^H X
    // re-orthonormalising steps (polish 1) need R only: their lambda and couplings are not used, and the
    // final evaluation (polish 2) forms P and S again
    // When A has the working precision's words, R joins the first call: X is then split once as the right
    // operand of both A X and X^H X (the call splits an operand shared by several products once).
    std::vector<MwProd> p1, p2;
    const bool r_first = wa == W;
    for (int b : act) {
      const OaProb& q = probs[b];
      double* Xb = X + q.xoff * 2 * W;
      if (polish[b] != 1) {
        MwProd pa{q.n, q.n, q.n, 0, A + q.a_off * 2 * wa, Xb, Pm + q.xoff * 2 * W, nullptr, 1.0, 0};
        pa.keepA = 1;                                // A does not change: its planes are split once
        p1.push_back(pa);
      }
      MwProd pr_{q.n, q.n, q.n, 1, Xb, Xb, Rm + q.xoff * 2 * W, nullptr, -1.0, 1};
      pr_.hermitian = 1;                           // R = I - X^H X is Hermitian
      pr_.keepA = r_first ? 2 : 0;                 // X^H's planes (xcache) serve S = X^H P in the second call
      (r_first ? p1 : p2).push_back(pr_);
    }
    xcache.clear();                                // X changed since the last iteration
    PlaneCache* const caches[2] = {&pcache, &xcache};   // keepA 1: A's planes, 2: this iteration's X^H
    s = mw_gemm_batched(p1.data(), (int)p1.size(), wa, W, W, p_bits, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage, caches, 2);
    if (s != ZKQ_OK) return s;
    for (int b : act) {
      const OaProb& q = probs[b];
      if (polish[b] == 1) continue;
      double* Xb = X + q.xoff * 2 * W;
      MwProd ps_{q.n, q.n, q.n, 1, Xb, Pm + q.xoff * 2 * W, Sm + q.xoff * 2 * W, nullptr, 1.0, 0};
      ps_.hermitian = 1;                           // S = X^H A X is Hermitian
      ps_.keepA = 2;                               // X^H's planes from the first call
      p2.push_back(ps_);
    }
    s = mw_gemm_batched(p2.data(), (int)p2.size(), W, W, W, p_bits, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage, caches, 2);
    if (s != ZKQ_OK) return s;
    // statistics for every problem (inactive ones keep their last values: recompute is harmless but skipped)
    std::vector<OaProb> ap; for (int b : act) ap.push_back(probs[b]);
    OaProb* APR = PR;   // the stats/E kernels index PR by the active list
    std::vector<int32_t> actv(act.begin(), act.end());
    std::vector<int32_t> oo; for (int b : act) oo.push_back(polish[b] == 1 ? 1 : 0);
    // pack the active problems' descriptors at the front of a scratch copy
    OaProb* PRA = (OaProb*)(base + oCLD);   // reuse: cluster list is built after these kernels
    hs.add(WH, actv.data(), sizeof(int32_t) * actv.size());
    hs.add(PRA, ap.data(), sizeof(OaProb) * ap.size());
    hs.add(OO, oo.data(), sizeof(int32_t) * oo.size());
    ZKQ_CUDA_TRY(hs.flush(st));
    {
      int mx = 0; for (auto& q : ap) mx = std::max(mx, q.n * q.n);
      dim3 g((mx + 255) / 256, (unsigned)ap.size());
      { ProfScope ps_(PC_OA, st); oa_lambda_kernel<W><<<(unsigned)ap.size(), 256, 0, st>>>(PRA, Sm, Rm, Lm, CN, ST); }
      { ProfScope ps_(PC_OA, st); oa_coupling_kernel<W><<<g, 256, 0, st>>>(PRA, Sm, Rm, Lm, CN, NUM, ST); }
      { ProfScope ps_(PC_OA, st); oa_cluster_kernel<W><<<(unsigned)ap.size(), 32, 0, st>>>(PRA, Lm, CN, CS, CL, ST, kClusterMargin); }
      { ProfScope ps_(PC_OA, st); oa_E_kernel<W><<<g, 256, 0, st>>>(PRA, NUM, Rm, Lm, CS, OO, Em, ST); }
      ZKQ_CUDA_TRY(cudaGetLastError());
    }
    std::vector<OaStat> ast(ap.size());
    ZKQ_CUDA_TRY(hs.download_sync(ast.data(), ST, sizeof(OaStat) * ap.size(), st));
    ZKQ_CUDA_TRY(hs.download_sync(hcl_len.data(), CL, sizeof(int32_t) * le, st));
    (void)APR;
    if (debug_log()) {
      for (size_t a = 0; a < act.size(); ++a)
        fprintf(stderr, "[zkq oa] it %d prob %d n %d maxE %.3e coupling %.3e maxR %.3e delta %.3e clusters %d (%d cols) cl_off %.3e\n",
                it, act[a], probs[act[a]].n, ast[a].maxE, ast[a].maxNum / (ast[a].anorm > 0 ? ast[a].anorm : 1.0), ast[a].maxR,
                ast[a].delta, ast[a].nclusters, ast[a].clustered, ast[a].cl_off / (ast[a].anorm > 0 ? ast[a].anorm : 1.0));
    }
    // convergence decisions
    std::vector<int> finish, upd, polar;
    std::vector<int> polar_terms(batch, 0);
    for (size_t a = 0; a < act.size(); ++a) {
      int b = act[a];
      hst[b] = ast[a];
      iters[b] = it;
      const double an = ast[a].anorm > 0 ? ast[a].anorm : 1.0;
      // converged: every coupling (the residual proxy) at the working-precision level; near-degenerate
      // noise may leave (noise/gap)^2 in R, which the orthonormalising steps below remove
      bool conv = ast[a].maxNum <= tol * an;
      const bool orth_ok = ast[a].maxR <= ldexp(1.0, -(53 * W - 10));
      // polish: 0 iterating; 1 converged: updates only re-orthonormalise (E = R/2) until R is at working
      // precision (at most 4 such steps); 2 report lambda and X of this evaluation
      // A converged problem finishes at once (polar step below) when its couplings are so small that every
      // column's residual, about the column norm of the couplings (<= sqrt(n) max|num|), is 16x below the
      // convergence tolerance, and R needs at most four polar terms.  Otherwise it takes one more ordinary
      // update (which squares the couplings); if that does not get there either (couplings at the noise
      // level), it takes the orthonormalising steps.
      const bool polar_ok = ast[a].maxNum * sqrt((double)probs[b].n) <= tol * an / 16.0 &&
                            (polar_terms[b] = polar_term_count(ast[a].maxR, probs[b].n, W)) > 0;
      if (polish[b] == 2 || it == max_iter) finish.push_back(b);
      else if (polish[b] == 0 && conv && polar_ok) {
        polar.push_back(b);     // finish now: lambda from this evaluation, X made orthonormal by its polar factor
      } else {
        if (polish[b] == 1) { if (orth_ok || ++orth_steps[b] >= 4) polish[b] = 2; }
        else if (conv && ++near_conv[b] >= 2) polish[b] = 1;
        upd.push_back(b);
      }
    }
    if (!finish.empty()) {
      // statistics of finishing problems are in ST at their active index: copy to a per-problem array
      std::vector<OaStat> fst(batch);
      for (size_t a = 0; a < act.size(); ++a) fst[act[a]] = ast[a];
      hs.add(ST, fst.data(), sizeof(OaStat) * batch);
      hs.add(WH, finish.data(), sizeof(int32_t) * finish.size());
      hs.add(PR, probs.data(), sizeof(OaProb) * batch);
      ZKQ_CUDA_TRY(hs.flush(st));
      {
        ProfScope ps_(PC_OA, st);
        oa_output_kernel<W><<<dim3((unsigned)((nmax + 7) / 8), (unsigned)finish.size()), 256, 0, st>>>(PR, WH, X, Pm, Lm, ST, W_out, V_out, err);
      }
      ZKQ_CUDA_TRY(cudaGetLastError());
      std::vector<int32_t> hinfo(batch, 0);
      bool any = false;
      for (int b : finish) {
        active[b] = 0;
        if (polish[b] != 2) { hinfo[b] = it > 0 ? it : 1; any = true; }
      }
      if (any) {
        for (int b : finish) if (hinfo[b]) hs.add(info + b, &hinfo[b], sizeof(int32_t));
        ZKQ_CUDA_TRY(hs.flush(st));
      }
    }
    if (!polar.empty()) {
      // Converged problems whose non-orthonormality R = I - X^H X is small enough finish in this iteration.
      // lambda = s_ii / (1 - r_ii) is already the Rayleigh quotient of X's columns.  X is replaced by its polar
      // (Loewdin) factor X (X^H X)^{-1/2} = X (I - R)^{-1/2} = X (I + F), the symmetric orthonormalisation that
      // removes the symmetric part of the pairwise tilts and leaves the couplings (already below tolerance):
      //   F = c1 R + c2 R^2 + ... + ck R^k,  (c1, c2, c3, c4) = (1/2, 3/8, 5/16, 35/128),
      // with k terms such that the dropped ones are below the working precision (polar_term_count), by
      // Horner's rule F = (R/2) G_1, G_j = I + (c_{j+1}/c_j) R G_{j+1}, G_{k-1} = I + (c_k/c_{k-1}) R.  Then
      // X_out = X + X F and P_out = P + P F = A X_out give the output and its residual estimate.  This replaces
      // the orthonormalising steps E = R/2 and the final evaluation of the products.
      // Buffers at each problem's own offset: G ping-pong in CT / CG, scaled R in CW, X_out in X2, P_out in S
      // (S is consumed); the cluster step of this iteration reuses CT / CG / CW afterwards, in stream order.
      // All problems finishing in this iteration take the largest term count among them (more terms only
      // make the factor more accurate).
      static const double cfr[4] = {0.5, 0.75, 5.0 / 6.0, 0.875};   // c_1, then c_{j+1} / c_j
      std::vector<OaProb> pp; int k = 0, mxe = 0;
      for (int b : polar) { pp.push_back(probs[b]); k = std::max(k, polar_terms[b]); mxe = std::max(mxe, probs[b].n * probs[b].n); }
      std::vector<int32_t> pw(polar.begin(), polar.end());
      OaProb* PRP = (OaProb*)(base + oCLD);
      hs.add(PRP, pp.data(), sizeof(OaProb) * pp.size());
      ZKQ_CUDA_TRY(hs.flush(st));
      const dim3 gp((mxe + 255) / 256, (unsigned)pp.size());
      double* Gcur = CT; double* Gnext = CG;
      auto term = [&](double* out, double coef, int add_identity) -> zkq_status {
        { ProfScope ps_(PC_OA, st); oa_polar_term_kernel<W><<<gp, 256, 0, st>>>(PRP, Rm, out, coef, add_identity); }
        ZKQ_CUDA_TRY(cudaGetLastError());
        return ZKQ_OK;
      };
      auto prod = [&](const double* Aop, const double* Bop, double* Cop, int identity) -> zkq_status {
        std::vector<MwProd> v;
        for (auto& q : pp) {
          MwProd m_{q.n, q.n, q.n, 0, Aop + q.xoff * 2 * W, Bop + q.xoff * 2 * W, Cop + q.xoff * 2 * W, nullptr, 1.0, identity};
          m_.hermitian = 1;                            // polynomials in the Hermitian R are Hermitian
          v.push_back(m_);
        }
        return mw_gemm_batched(v.data(), (int)v.size(), W, W, W, p_bits, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage);
      };
      const double* F = CW;
      if (k == 1) {
        s = term(CW, cfr[0], 0);                      // F = R/2
        if (s != ZKQ_OK) return s;
      } else {
        s = term(Gcur, cfr[k - 1], 1);                // G_{k-1} = I + (c_k / c_{k-1}) R
        if (s != ZKQ_OK) return s;
        for (int j = k - 2; j >= 1; --j) {            // G_j = I + (c_{j+1} / c_j) R G_{j+1}
          s = term(CW, cfr[j], 0);
          if (s != ZKQ_OK) return s;
          s = prod(CW, Gcur, Gnext, 1);
          if (s != ZKQ_OK) return s;
          std::swap(Gcur, Gnext);
        }
        s = term(CW, cfr[0], 0);                      // F = (R/2) G_1
        if (s != ZKQ_OK) return s;
        s = prod(CW, Gcur, Gnext, 0);
        if (s != ZKQ_OK) return s;
        F = Gnext;
      }
      {
        std::vector<MwProd> po;
        for (auto& q : pp) {
          double* Xb = X + q.xoff * 2 * W;
          double* Pb = Pm + q.xoff * 2 * W;
          po.push_back({q.n, q.n, q.n, 0, Xb, F + q.xoff * 2 * W, X2 + q.xoff * 2 * W, Xb, 1.0, 0});
          po.push_back({q.n, q.n, q.n, 0, Pb, F + q.xoff * 2 * W, Sm + q.xoff * 2 * W, Pb, 1.0, 0});
        }
        s = mw_gemm_batched(po.data(), (int)po.size(), W, W, W, p_bits, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage);
        if (s != ZKQ_OK) return s;
      }
      std::vector<OaStat> fst(batch);
      for (size_t a = 0; a < act.size(); ++a) fst[act[a]] = ast[a];
      hs.add(ST, fst.data(), sizeof(OaStat) * batch);
      hs.add(WH, pw.data(), sizeof(int32_t) * pw.size());
      hs.add(PR, probs.data(), sizeof(OaProb) * batch);
      ZKQ_CUDA_TRY(hs.flush(st));
      {
        ProfScope ps_(PC_OA, st);
        oa_output_kernel<W><<<dim3((unsigned)((nmax + 7) / 8), (unsigned)polar.size()), 256, 0, st>>>(PR, WH, X2, Sm, Lm, ST, W_out, V_out, err);
      }
      ZKQ_CUDA_TRY(cudaGetLastError());
      for (int b : polar) active[b] = 0;
    }
    if (upd.empty()) continue;
    // X2 = X + X E  (E double-double)
    std::vector<MwProd> p3;
    for (int b : upd) {
      const OaProb& q = probs[b];
      double* Xb = X + q.xoff * 2 * W;
      p3.push_back({q.n, q.n, q.n, 0, Xb, Em + q.xoff * 2 * 2, X2 + q.xoff * 2 * W, Xb, 1.0, 0});
    }
    // E is indexed by the active order in the E kernel: it wrote at each problem's own xoff, so p3 is direct.
    // X E is added to X, so it needs the working precision of X's scale only: its error is 2^-p of the
    // scale of E's columns (at most sqrt(2) max|e|), and the product takes log2(1 / (2 max|e|)) bits fewer.
    double emax = 0.0;
    for (int b : upd) emax = std::max(emax, hst[b].maxE);
    int p_xe = p_bits;
    if (emax > 0 && emax < 0.25) p_xe = std::max(64, p_bits - (int)std::floor(-std::log2(2.0 * emax)));
    s = mw_gemm_batched(p3.data(), (int)p3.size(), W, 2, W, p_xe, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage);
    if (s != ZKQ_OK) return s;
    // clusters that still need separation
    std::vector<OaCluster> cls;
    int64_t toff = 0, woff = 0;
    for (int b : upd) {
      const OaProb& q = probs[b];
      // rotate only clusters whose members are still coupled (gap-free measure |s_ij + lambda_j r_ij|);
      // non-orthonormality alone is removed by the r/2 part of E.  The bar is the one the polar finish sets
      // for every coupling (sqrt(n) max|num| <= tol ||A|| / 16): a cluster left coupled just below tol would
      // keep its problem from finishing and send it through the orthonormalising steps.
      bool need = hst[b].cl_off * sqrt((double)q.n) > tol * (hst[b].anorm > 0 ? hst[b].anorm : 1.0) / 16.0 &&
                  hst[b].nclusters > 0 && polish[b] == 0;
      if (!need) continue;
      for (int c = 0; c < q.n;) {
        int len = hcl_len[q.loff + c];
        if (len > 1) { cls.push_back({b, c, len, toff, woff}); toff += (int64_t)len * len; woff += len; }
        c += std::max(len, 1);
      }
    }
    if (!cls.empty()) {
      int maxl = 0; for (auto& c : cls) maxl = std::max(maxl, c.len);
      hs.add(PR, probs.data(), sizeof(OaProb) * batch);
      hs.add(CLD, cls.data(), sizeof(OaCluster) * cls.size());
      ZKQ_CUDA_TRY(hs.flush(st));
      // Q_J = A X2_J (into the P buffer's cluster columns), then CT = X2_J^H Q_J, CG = X2_J^H X2_J.
      // T = CT - mu CG is rounded to FP64, so it needs an absolute accuracy of about 2^-57 times the
      // cluster's spread of eigenvalues; the products' error is 2^-p of the scale of A (times sqrt(n) for
      // the inner dimension).  A cluster whose spread is 2^-d ||A|| therefore takes p = 64 + d +
      // log2(n)/2 bits (rounded up to a multiple of 16, at most the working precision): the wide
      // clusters of the first peeling steps of a graded spectrum need less than half the moduli.
      std::vector<double> lam_h((size_t)le * W);
      ZKQ_CUDA_TRY(hs.download_sync(lam_h.data(), Lm, sizeof(double) * lam_h.size(), st));
      std::vector<int> cp(cls.size());
      for (size_t k = 0; k < cls.size(); ++k) {
        const OaCluster& c = cls[k];
        const OaProb& q = probs[c.prob];
        double lo = 0, hi = 0;
        for (int t = 0; t < c.len; ++t) {
          const double l = lam_h[(size_t)(q.loff + c.start + t) * W];
          if (t == 0 || l < lo) lo = l;
          if (t == 0 || l > hi) hi = l;
        }
        const double an = hst[c.prob].anorm > 0 ? hst[c.prob].anorm : 1.0, spread = hi - lo;
        int need = p_bits;
        if (spread > 0) {
          need = 64 + (int)std::ceil(std::log2(an / spread)) + (int)std::ceil(0.5 * std::log2((double)q.n));
          need = std::min(p_bits, (need + 15) / 16 * 16);
        }
        cp[k] = std::max(need, 64);
      }
      std::vector<int> levels(cp.begin(), cp.end());
      std::sort(levels.begin(), levels.end());
      levels.erase(std::unique(levels.begin(), levels.end()), levels.end());
      PlaneCache* const acache[1] = {&pcache};
      for (int pl : levels) {
        std::vector<MwProd> p5, p6;
        for (size_t k = 0; k < cls.size(); ++k) {
          if (cp[k] != pl) continue;
          const OaCluster& c = cls[k];
          const OaProb& q = probs[c.prob];
          double* XJ = X2 + (q.xoff + (int64_t)c.start * q.n) * 2 * W;
          double* QJ = Pm + (q.xoff + (int64_t)c.start * q.n) * 2 * W;
          MwProd pa{q.n, c.len, q.n, 0, A + q.a_off * 2 * wa, XJ, QJ, nullptr, 1.0, 0};
          pa.keepA = 1;
          p5.push_back(pa);
          MwProd pt_{c.len, c.len, q.n, 1, XJ, QJ, CT + c.toff * 2 * W, nullptr, 1.0, 0};
          MwProd pg_{c.len, c.len, q.n, 1, XJ, XJ, CG + c.toff * 2 * W, nullptr, 1.0, 0};
          pt_.hermitian = 1; pg_.hermitian = 1;
          p6.push_back(pt_);
          p6.push_back(pg_);
        }
        s = mw_gemm_batched(p5.data(), (int)p5.size(), wa, W, W, pl, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage, acache, 1);
        if (s != ZKQ_OK) return s;
        s = mw_gemm_batched(p6.data(), (int)p6.size(), W, W, W, pl, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage);
        if (s != ZKQ_OK) return s;
      }
      dim3 g((maxl * maxl + 255) / 256, (unsigned)cls.size());
      { ProfScope ps_(PC_OA, st); oa_cluster_mu_kernel<W><<<(unsigned)((cls.size() + 127) / 128), 128, 0, st>>>(PR, CLD, (int)cls.size(), Lm, MUb); }
      { ProfScope ps_(PC_OA, st); oa_cluster_T_kernel<W><<<g, 256, 0, st>>>(PR, CLD, CT, CG, MUb, T); }
      ZKQ_CUDA_TRY(cudaGetLastError());
      std::vector<int32_t> cn(cls.size()); std::vector<int64_t> co(cls.size());
      for (size_t c = 0; c < cls.size(); ++c) { cn[c] = cls[c].len; co[c] = cls[c].toff; }
      s = eigh_internal(ctx, (int)cls.size(), cn.data(), co.data(), T, 1, TW, TV, TI, st, PC_JACOBI_CLUSTER);
      if (s != ZKQ_OK) return s;
      // The FP64 eigenvector matrix W is unitary only to about 2^-53 sqrt(len).  It rotates X_J as it is: its
      // departure from unitarity adds non-orthonormality to X_J, which the couplings do not see (they are
      // insensitive to it at first order) and the next update's R/2 removes, and which is far below what
      // every update leaves anyway (about E^H E, 10^-13 to 10^-10 in the peeling iterations of a graded
      // spectrum).  Two Newton-Schulz steps making W unitary to the working precision cost four len^3
      // products per cluster and changed neither the iterations nor the peeling.
      { ProfScope ps_(PC_OA, st); oa_promote_kernel<W><<<g, 256, 0, st>>>(CLD, TV, CT); }
      ZKQ_CUDA_TRY(cudaGetLastError());
      const double* Wcur = CT;
      // Y_J = X2_J W_J into the X buffer (free now), then copy back into X2
      std::vector<MwProd> p4;
      for (auto& c : cls) {
        const OaProb& q = probs[c.prob];
        p4.push_back({q.n, c.len, c.len, 0, X2 + (q.xoff + (int64_t)c.start * q.n) * 2 * W, Wcur + c.toff * 2 * W,
                      X + (q.xoff + (int64_t)c.start * q.n) * 2 * W, nullptr, 1.0, 0});
      }
      s = mw_gemm_batched(p4.data(), (int)p4.size(), W, W, W, p_bits, prod_method, buf.oz_ws, buf.oz_bytes, buf.oz_meta, buf.oz_meta_bytes, st, buf.stage);
      if (s != ZKQ_OK) return s;
      dim3 g2((nmax * maxl + 255) / 256, (unsigned)cls.size());
      { ProfScope ps_(PC_OA, st); oa_cluster_copy_kernel<W><<<g2, 256, 0, st>>>(PR, CLD, X, X2); }
      ZKQ_CUDA_TRY(cudaGetLastError());
    }
    // X <- X2: every active problem was either finished (its output is written) or updated into X2
    std::swap(X, X2);
  }
  return ZKQ_OK;
}

zkq_status oa_refine(void* ctx, const OaBuffers& buf, int batch, const int32_t* n, const int64_t* a_off,
                     const double* A, int wa, const double* V, int W, double* W_out, double* V_out, double* err,
                     int32_t* info, int max_iter, int prod_method, cudaStream_t st) {
  if (W == 2) return oa_refine_t<2>(ctx, buf, batch, n, a_off, A, wa, V, W_out, V_out, err, info, max_iter, prod_method, st);
  if (W == 4) return oa_refine_t<4>(ctx, buf, batch, n, a_off, A, wa, V, W_out, V_out, err, info, max_iter, prod_method, st);
  return ZKQ_EINVAL;
}

}  // namespace zkq
