// Batched complex singular value decomposition in FP64 by one-sided (Hestenes) Jacobi: the SVD the paper's
// ZKCM_CUS offers beside the Hermitian diagonalisation (Section 2, ZKCM_CUS paragraph: singular value
// decomposition through cuSOLVER with the precision then recovered; here a hand-written kernel).  In the
// MPS gate update it replaces the FP64 eigensolve of rho = M M^H by the SVD of M itself, which does not
// square the conditioning: on a matrix whose rows are graded (M carries the Schmidt weights of the bond to
// its left), the small singular values come out with high relative accuracy instead of drowning below
// 2^-53 ||rho|| in the Gram matrix.
//
// For A (m x n) let G = A if m >= n, else G = A^H, so G is R x K with R = max(m, n) >= K = min(m, n).  The
// columns of G are orthogonalised pairwise: for columns p, q with Gram entries alpha = |g_p|^2,
// beta = |g_q|^2, gamma = g_p^H g_q = |gamma| e^{i phi}, the rotation that diagonalises the 2 x 2 Gram matrix
//   zeta = (beta - alpha) / (2 |gamma|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2),
//   s = t c, J = [[c, s e^{i phi}], [-s e^{-i phi}, c]]
// is applied as G <- G J and accumulated in V <- V J, pairs taken in the parallel (circle) order of the
// FP64 eigensolver.  A pair is rotated while |gamma| > 2^-51 sqrt(alpha beta); a sweep without rotation
// ends the iteration.  Then G = U_G Sigma with sigma_j = |g_j| and G_in = U_G Sigma V^H, so
//   m >= n: A = U_G Sigma V^H;   m < n: A = V Sigma U_G^H.
// Output: sigma descending (ties by index); the left singular vectors with their first largest-modulus
// component real and positive, the right ones carrying the same phase.  One CTA per problem; the working
// copies of G and V live in the context's workspace (L2-resident for the sizes of a gate update).
#include <vector>
#include <algorithm>
#include "common.cuh"
#include "prof.cuh"
#include "internal.cuh"

namespace zkq {

struct SvdProb { int m, n; int64_t a_off, u_off, v_off, s_off, ws_off; };

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int WA>
__global__ void __launch_bounds__(256) svd_onesided_kernel(const SvdProb* __restrict__ pr, const double* __restrict__ A,
                                                          double* __restrict__ ws, double* __restrict__ S,
                                                          double* __restrict__ U, double* __restrict__ V,
                                                          int32_t* __restrict__ info, int max_sweeps) {
  const SvdProb p = pr[blockIdx.x];
  const bool tr = p.m < p.n;
  const int R = tr ? p.n : p.m, K = tr ? p.m : p.n;
  c64* G = reinterpret_cast<c64*>(ws + p.ws_off);          // R x K, column-major
  c64* Vc = G + (size_t)R * K;                              // K x K
  double* nrm = reinterpret_cast<double*>(Vc + (size_t)K * K);   // K column norms
  int* rnk = reinterpret_cast<int*>(nrm + K);               // K ranks
  const double* Ab = A + p.a_off * 2 * WA;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  for (int e = tid; e < R * K; e += nth) {
    const int i = e % R, j = e / R;
    // G[i, j] = A[i, j] or conj(A[j, i]); only the leading word of each real is used
    const double* q = tr ? Ab + ((size_t)j + (size_t)i * p.m) * 2 * WA : Ab + ((size_t)i + (size_t)j * p.m) * 2 * WA;
    G[e] = c64{q[0], tr ? -q[WA] : q[WA]};
  }
  for (int e = tid; e < K * K; e += nth) Vc[e] = c64{(e % K) == (e / K) ? 1.0 : 0.0, 0.0};
  __shared__ int s_rot;
  __syncthreads();
  const int mm = K + (K & 1), P = mm / 2;
  int sweep = 0, converged = 0;
  for (sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    int my_rot = 0;
    for (int r = 0; r < mm - 1; ++r) {
      for (int k = warp; k < P; k += nwarp) {
        int pp, qq; rr_pair(mm, r, k, pp, qq);
        if (qq >= K) continue;
        c64* gp = G + (size_t)pp * R; c64* gq = G + (size_t)qq * R;
        double al = 0, be = 0, gr = 0, gi = 0;
        for (int i = lane; i < R; i += 32) {
          const c64 x = gp[i], y = gq[i];
          al += x.re * x.re + x.im * x.im;
          be += y.re * y.re + y.im * y.im;
          gr += x.re * y.re + x.im * y.im;           // conj(x) y
          gi += x.re * y.im - x.im * y.re;
        }
        al = warp_sum(al); be = warp_sum(be); gr = warp_sum(gr); gi = warp_sum(gi);
        const double ag = hypot(gr, gi);
        if (!(ag > 0x1p-51 * sqrt(al * be))) continue;   // also skips zero columns
        const double zeta = (be - al) / (2.0 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        const double er = gr / ag, ei = gi / ag;
        const c64 z2{s * er, s * ei}, z1{s * er, -s * ei};   // s e^{i phi}, s e^{-i phi}
        ++my_rot;
        for (int i = lane; i < R; i += 32) {
          const c64 x = gp[i], y = gq[i];
          const c64 u = cmul(z1, y), v = cmul(z2, x);
          gp[i] = c64{c * x.re - u.re, c * x.im - u.im};
          gq[i] = c64{v.re + c * y.re, v.im + c * y.im};
        }
        c64* vp = Vc + (size_t)pp * K; c64* vq = Vc + (size_t)qq * K;
        for (int i = lane; i < K; i += 32) {
          const c64 x = vp[i], y = vq[i];
          const c64 u = cmul(z1, y), v = cmul(z2, x);
          vp[i] = c64{c * x.re - u.re, c * x.im - u.im};
          vq[i] = c64{v.re + c * y.re, v.im + c * y.im};
        }
      }
      __syncthreads();
    }
    if (lane == 0 && my_rot) atomicAdd(&s_rot, my_rot);
    __syncthreads();
    converged = (s_rot == 0);
    __syncthreads();
  }
  // column norms, ranks (descending, ties by index)
  for (int j = warp; j < K; j += nwarp) {
    double a = 0;
    for (int i = lane; i < R; i += 32) { const c64 x = G[(size_t)j * R + i]; a += x.re * x.re + x.im * x.im; }
    a = warp_sum(a);
    if (lane == 0) nrm[j] = sqrt(a);
  }
  __syncthreads();
  for (int j = tid; j < K; j += nth) {
    int rk = 0;
    for (int d = 0; d < K; ++d) rk += (nrm[d] > nrm[j]) || (nrm[d] == nrm[j] && d < j);
    rnk[j] = rk;
    S[p.s_off + rk] = nrm[j];
  }
  __syncthreads();
  // outputs: column j goes to position rnk[j]; left vectors of A are U_G (m >= n) or V (m < n)
  const int um = p.m, vn = p.n;
  for (int j = warp; j < K; j += nwarp) {
    const int rk = rnk[j];
    const double sj = nrm[j];
    const double inv = sj > 0 ? 1.0 / sj : 0.0;
    const c64* lc = tr ? Vc + (size_t)j * K : G + (size_t)j * R;      // left vector (length m), unnormalised for G
    const c64* rc = tr ? G + (size_t)j * R : Vc + (size_t)j * K;      // right vector (length n)
    const double ls = tr ? 1.0 : inv, rs = tr ? inv : 1.0;
    // phase from the left vector's first largest-modulus component
    int best = um; double bm = -1.0;
    for (int i = lane; i < um; i += 32) {
      const double m2 = lc[i].re * lc[i].re + lc[i].im * lc[i].im;
      if (m2 > bm) { bm = m2; best = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, bm, o);
      const int oi = __shfl_xor_sync(0xffffffffu, best, o);
      if (ob > bm || (ob == bm && oi < best)) { bm = ob; best = oi; }
    }
    c64 ph{1.0, 0.0};
    if (bm > 0) { const double a = sqrt(bm); ph = c64{lc[best].re / a, -lc[best].im / a}; }   // conj(x)/|x|
    double* uo = U + (p.u_off + (size_t)rk * um) * 2;
    for (int i = lane; i < um; i += 32) {
      c64 v = cmul(lc[i], ph);
      if (i == best) v.im = 0.0;
      uo[2 * i] = v.re * ls; uo[2 * i + 1] = v.im * ls;
    }
    double* vo = V + (p.v_off + (size_t)rk * vn) * 2;
    for (int i = lane; i < vn; i += 32) {
      const c64 v = cmul(rc[i], ph);
      vo[2 * i] = v.re * rs; vo[2 * i + 1] = v.im * rs;
    }
  }
  if (tid == 0) info[blockIdx.x] = converged ? 0 : sweep;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// doubles of workspace per problem: G (R K complex), V (K K complex), norms, ranks
static size_t svd_ws_doubles(int m, int n) {
  const size_t R = std::max(m, n), K = std::min(m, n);
  return al256((2 * R * K + 2 * K * K + 2 * K) * sizeof(double)) / sizeof(double);
}

zkq_status svd_internal(void* ctx, int batch, const int32_t* m, const int32_t* n, const int64_t* a_off, const double* A,
                        int a_words, double* S, double* U, const int64_t* u_off, double* V, const int64_t* v_off,
                        int32_t* info, cudaStream_t st, void** ws, size_t* ws_bytes, void** meta, size_t* meta_bytes) {
  std::vector<SvdProb> pr(batch);
  int64_t so = 0, wo = 0;
  for (int b = 0; b < batch; ++b) {
    pr[b] = {m[b], n[b], a_off[b], u_off[b], v_off[b], so, wo};
    so += std::min(m[b], n[b]);
    wo += (int64_t)svd_ws_doubles(m[b], n[b]);
  }
  auto grow = [](void** p, size_t* have, size_t need) -> zkq_status {
    if (need <= *have) return ZKQ_OK;
    if (*p) { cudaFree(*p); *p = nullptr; *have = 0; }
    const size_t want = std::max(need, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) { set_last_cuda_error(e); *p = nullptr; return ZKQ_ENOMEM; }
    *have = want;
    return ZKQ_OK;
  };
  zkq_status s = grow(ws, ws_bytes, (size_t)wo * sizeof(double));
  if (s != ZKQ_OK) return s;
  s = grow(meta, meta_bytes, al256(sizeof(SvdProb) * batch));
  if (s != ZKQ_OK) return s;
  ZKQ_CUDA_TRY(ctx_stage(ctx)->upload(*meta, pr.data(), sizeof(SvdProb) * batch, st));
  const int ms = ctx_config(ctx).max_sweeps > 0 ? ctx_config(ctx).max_sweeps : 40;
  ProfScope ps(PC_JACOBI, st);
  const SvdProb* d = (const SvdProb*)*meta;
  switch (a_words) {
    case 1: svd_onesided_kernel<1><<<batch, 256, 0, st>>>(d, A, (double*)*ws, S, U, V, info, ms); break;
    case 2: svd_onesided_kernel<2><<<batch, 256, 0, st>>>(d, A, (double*)*ws, S, U, V, info, ms); break;
    default: svd_onesided_kernel<4><<<batch, 256, 0, st>>>(d, A, (double*)*ws, S, U, V, info, ms); break;
  }
  ZKQ_CUDA_TRY(cudaGetLastError());
  return ZKQ_OK;
}

}  // namespace zkq
