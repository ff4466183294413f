// Plain precision recovery by Rayleigh quotient iteration (Section 2, ZKCM_CUS paragraph: RQI recovers
// the precision after the double-precision eigensolve).  One CTA per eigenpair, all arithmetic in the
// target multi-word precision:
//   x <- v (FP64), normalised;
//   repeat: y = A x;  mu = x^H y / x^H x;  r = y - mu x;  stop if ||r|| <= 2^-p ||A||;
//           solve (A - mu I) z = x by LU with partial pivoting;  x <- z / ||z||;
//   finally mu = x^H A x / x^H x, and the phase of x makes its first largest-modulus entry real > 0.
// The LU works on the augmented matrix [A - mu I | x] so the forward substitution happens during the
// elimination; back substitution is column oriented.  A zero pivot (mu equal to an eigenvalue at working
// precision) is replaced by 2^-(53W+8) ||A||, the usual inverse-iteration safeguard.
#include "common.cuh"
#include "mw.cuh"
#include "reduce.cuh"
#include "prof.cuh"
#include "internal.cuh"

namespace zkq {


// Convergence: the computed residual cannot drop below the rounding floor ~ n 2^(-53W) ||A||, so the
// iteration counts as converged at 16 n 2^(-53W) ||A|| and then takes one more (cubically convergent)
// step to settle at the floor.
template <int W> __device__ __forceinline__ int word_bits() { return 53 * W; }

template <int W, int WA>
__global__ void __launch_bounds__(256) rqi_kernel(RqiBatch rb) {
  extern __shared__ __align__(16) unsigned char smem[];
  cmw<W>* red = reinterpret_cast<cmw<W>*>(smem);
  __shared__ double s_dbl[32];
  __shared__ int s_piv;
  __shared__ long long s_item;
  double* ws = rb.ws + (size_t)blockIdx.x * rb.ws_stride;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(rb.counter, 1);
    __syncthreads();
    const long long item = s_item;
    __syncthreads();
    if (item >= rb.total_pairs) break;
    // locate (problem, column) of this eigenpair
    const int b = rb.pair_prob[item];
    const int n = rb.n[b];
    const int col = (int)(item - rb.w_off[b]);
    const double* Ab = rb.A + rb.a_off[b] * 2 * WA;
    const size_t ldb = (size_t)n;                 // augmented matrix: n x (n + 1), column-major
    double* B = ws;                                // (n*(n+1)) complex W-word elements
    double* x = B + (size_t)n * (n + 1) * 2 * W;   // n complex W-word elements
    double* y = x + (size_t)n * 2 * W;
    // ||A|| estimate: max |lambda| from the FP64 stage (eigenvalues are sorted)
    const double* Wb = rb.W + rb.w_off[b];
    const double anorm = fmax(fabs(Wb[0]), fabs(Wb[n - 1]));
    const double thresh = ldexp(anorm * n, 4 - word_bits<W>());
    // x <- v, normalised
    mw<W> nrm2 = mw_zero<W>();
    for (int i = tid; i < n; i += nth) {
      const double* vp = rb.V + (rb.a_off[b] + (size_t)i + (size_t)col * n) * 2;
      cmw<W> v = c_make(mw_from<W>(vp[0]), mw_from<W>(vp[1]));
      c_store(x, i, v);
      nrm2 = mw_add(nrm2, c_abs2(v));
    }
    nrm2 = block_sum_r(nrm2, reinterpret_cast<mw<W>*>(red));
    {
      mw<W> inv = mw_recip(mw_sqrt(nrm2));
      for (int i = tid; i < n; i += nth) c_store(x, i, c_scale(c_load<W, W>(x, i), inv));
    }
    __syncthreads();
    mw<W> mu = mw_from<W>(Wb[col]);
    int converged = 0, it = 0;
    double res = 0.0;
    for (it = 0; it <= rb.max_iter; ++it) {
      // y = A x ; partial sums of x^H y and x^H x
      cmw<W> xy = c_zero<W>();
      mw<W> xx = mw_zero<W>();
      for (int i = tid; i < n; i += nth) {
        cmw<W> s = c_zero<W>();
        for (int j = 0; j < n; ++j) s = c_add(s, c_mul(c_load<W, WA>(Ab, (size_t)i + (size_t)j * n), c_load<W, W>(x, j)));
        c_store(y, i, s);
        cmw<W> xi = c_load<W, W>(x, i);
        xy = c_add(xy, c_mul_conj(xi, s));
        xx = mw_add(xx, c_abs2(xi));
      }
      xy = block_sum_c(xy, red);
      xx = block_sum_r(xx, reinterpret_cast<mw<W>*>(red));
      mu = mw_div(xy.re, xx);                      // Hermitian: the imaginary part is rounding noise
      // residual
      mw<W> rr = mw_zero<W>();
      for (int i = tid; i < n; i += nth) {
        cmw<W> r = c_sub(c_load<W, W>(y, i), c_scale(c_load<W, W>(x, i), mu));
        rr = mw_add(rr, c_abs2(r));
      }
      rr = block_sum_r(rr, reinterpret_cast<mw<W>*>(red));
      res = sqrt(fmax(rr.x[0], 0.0)) / sqrt(xx.x[0]);
      if (converged) break;                        // the polishing step has been taken
      if (res <= thresh) converged = 1;
      if (it == rb.max_iter) break;
      // B = [A - mu I | x]
      for (size_t e = tid; e < (size_t)n * (n + 1); e += nth) {
        int i = (int)(e % ldb), j = (int)(e / ldb);
        cmw<W> v = j < n ? c_load<W, WA>(Ab, (size_t)i + (size_t)j * n) : c_load<W, W>(x, i);
        if (i == j) v.re = mw_sub(v.re, mu);
        c_store(B, e, v);
      }
      __syncthreads();
      const double tiny = ldexp(anorm, -(53 * W + 8));
      for (int k = 0; k < n; ++k) {
        // pivot: largest |B_ik| (leading words) for i >= k; ties keep the smallest index
        double best = -1.0; int bi = k;
        for (int i = k + tid; i < n; i += nth) {
          const double* p = B + ((size_t)i + (size_t)k * ldb) * 2 * W;
          double m2 = p[0] * p[0] + p[W] * p[W];
          if (m2 > best) { best = m2; bi = i; }
        }
        // block argmax
        for (int o = 16; o > 0; o >>= 1) {
          double ob = __shfl_down_sync(0xffffffffu, best, o);
          int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((tid & 31) == 0) { s_dbl[tid >> 5] = best; reinterpret_cast<int*>(red)[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
          double bb = s_dbl[0]; int ii = reinterpret_cast<int*>(red)[0];
          for (int w = 1; w < nth / 32; ++w) {
            double ob = s_dbl[w]; int oi = reinterpret_cast<int*>(red)[w];
            if (ob > bb || (ob == bb && oi < ii)) { bb = ob; ii = oi; }
          }
          s_piv = ii;
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != k) {                                     // swap rows k and piv (columns k..n)
          for (int j = k + tid; j <= n; j += nth) {
            cmw<W> a = c_load<W, W>(B, (size_t)k + (size_t)j * ldb), c = c_load<W, W>(B, (size_t)piv + (size_t)j * ldb);
            c_store(B, (size_t)k + (size_t)j * ldb, c); c_store(B, (size_t)piv + (size_t)j * ldb, a);
          }
        }
        __syncthreads();
        cmw<W> ukk = c_load<W, W>(B, (size_t)k + (size_t)k * ldb);
        if (ukk.re.x[0] == 0.0 && ukk.im.x[0] == 0.0) {
          ukk.re = mw_from<W>(tiny);
          __syncthreads();
          if (tid == 0) c_store(B, (size_t)k + (size_t)k * ldb, ukk);
        }
        const cmw<W> rinv = c_div(c_make(mw_from<W>(1.0), mw_zero<W>()), ukk);
        __syncthreads();
        // multipliers l_ik = B_ik / u_kk stored in place
        for (int i = k + 1 + tid; i < n; i += nth)
          c_store(B, (size_t)i + (size_t)k * ldb, c_mul(c_load<W, W>(B, (size_t)i + (size_t)k * ldb), rinv));
        __syncthreads();
        // trailing update (columns k+1..n, the last one is the right-hand side)
        const int rows = n - k - 1, cols = n - k;
        for (int e = tid; e < rows * cols; e += nth) {
          int i = k + 1 + e % rows, j = k + 1 + e / rows;
          cmw<W> l = c_load<W, W>(B, (size_t)i + (size_t)k * ldb);
          cmw<W> u = c_load<W, W>(B, (size_t)k + (size_t)j * ldb);
          c_store(B, (size_t)i + (size_t)j * ldb, c_sub(c_load<W, W>(B, (size_t)i + (size_t)j * ldb), c_mul(l, u)));
        }
        __syncthreads();
      }
      // back substitution U z = c (c = last column), column oriented, z overwrites the last column
      for (int k = n - 1; k >= 0; --k) {
        cmw<W> zk = c_div(c_load<W, W>(B, (size_t)k + (size_t)n * ldb), c_load<W, W>(B, (size_t)k + (size_t)k * ldb));
        __syncthreads();
        for (int i = tid; i < k; i += nth)
          c_store(B, (size_t)i + (size_t)n * ldb, c_sub(c_load<W, W>(B, (size_t)i + (size_t)n * ldb), c_mul(c_load<W, W>(B, (size_t)i + (size_t)k * ldb), zk)));
        if (tid == 0) c_store(B, (size_t)k + (size_t)n * ldb, zk);
        __syncthreads();
      }
      // x <- z / ||z||  (scale by the leading-word max first to stay in range)
      double zmax = 0.0;
      for (int i = tid; i < n; i += nth) {
        const double* p = B + ((size_t)i + (size_t)n * ldb) * 2 * W;
        zmax = fmax(zmax, fmax(fabs(p[0]), fabs(p[W])));
      }
      zmax = block_max_d(zmax, s_dbl);
      int ez; frexp(zmax, &ez);
      mw<W> zz = mw_zero<W>();
      for (int i = tid; i < n; i += nth) {
        cmw<W> z = c_load<W, W>(B, (size_t)i + (size_t)n * ldb);
        z.re = mw_ldexp(z.re, -ez); z.im = mw_ldexp(z.im, -ez);
        c_store(x, i, z);
        zz = mw_add(zz, c_abs2(z));
      }
      zz = block_sum_r(zz, reinterpret_cast<mw<W>*>(red));
      mw<W> inv = mw_recip(mw_sqrt(zz));
      for (int i = tid; i < n; i += nth) c_store(x, i, c_scale(c_load<W, W>(x, i), inv));
      __syncthreads();
    }
    // phase normalisation and output
    double bm = -1.0; int bi = 0;
    for (int i = tid; i < n; i += nth) {
      const double* p = x + (size_t)i * 2 * W;
      double m2 = p[0] * p[0] + p[W] * p[W];
      if (m2 > bm) { bm = m2; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, bm, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > bm || (ob == bm && oi < bi)) { bm = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { s_dbl[tid >> 5] = bm; reinterpret_cast<int*>(red)[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bb = s_dbl[0]; int ii = reinterpret_cast<int*>(red)[0];
      for (int w = 1; w < nth / 32; ++w) {
        double ob = s_dbl[w]; int oi = reinterpret_cast<int*>(red)[w];
        if (ob > bb || (ob == bb && oi < ii)) { bb = ob; ii = oi; }
      }
      s_piv = ii;
    }
    __syncthreads();
    cmw<W> xb = c_load<W, W>(x, s_piv);
    mw<W> mag = mw_sqrt(c_abs2(xb));
    cmw<W> ph = c_make(mw_div(xb.re, mag), mw_neg(mw_div(xb.im, mag)));   // conj(x_b)/|x_b|
    __syncthreads();
    double* Vo = rb.V_out + (rb.a_off[b] + (size_t)col * n) * 2 * W;
    for (int i = tid; i < n; i += nth) {
      cmw<W> v = c_mul(c_load<W, W>(x, i), ph);
      if (i == s_piv) v.im = mw_zero<W>();
      c_store(Vo, i, v);
    }
    if (tid == 0) {
      mw_store(rb.W_out, rb.w_off[b] + col, mu);
      rb.err[rb.w_off[b] + col] = res / anorm;
      if (!converged) atomicAdd(rb.info + b, 1);
    }
    __syncthreads();
  }
}

template <int W, int WA>
static zkq_status launch_rqi_t(const RqiBatch& rb, int grid, cudaStream_t st) {
  size_t sm = 256 * sizeof(cmw<W>);
  ZKQ_CUDA_TRY((smem_limit_max<rqi_kernel<W, WA>>()));
  ProfScope ps(PC_RQI, st);
  rqi_kernel<W, WA><<<grid, 256, sm, st>>>(rb);
  ZKQ_CUDA_TRY(cudaGetLastError());
  return ZKQ_OK;
}

size_t rqi_slot_doubles(int nmax, int W) { return ((size_t)nmax * (nmax + 1) + 2 * (size_t)nmax) * 2 * W; }

zkq_status launch_rqi(const RqiBatch& rb, int W, int WA, int grid, cudaStream_t st) {
#define ZKQ_RQI_CASE(w, wa) if (W == w && WA == wa) return launch_rqi_t<w, wa>(rb, grid, st);
  ZKQ_RQI_CASE(2, 1) ZKQ_RQI_CASE(2, 2) ZKQ_RQI_CASE(2, 4)
  ZKQ_RQI_CASE(4, 1) ZKQ_RQI_CASE(4, 2) ZKQ_RQI_CASE(4, 4)
#undef ZKQ_RQI_CASE
  return ZKQ_EINVAL;
}

}  // namespace zkq
