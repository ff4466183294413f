// Measurements on the device-resident Vidal MPS, in its working precision (Section 1: the MPS is a nested
// Schmidt decomposition, kept to a precision that resolves Schmidt coefficients ~2^{-(n-1)/2}, footnote;
// what a simulation reads out of it must keep that precision).
//
// One-qubit expectation values.  In canonical Vidal form the environments to the left of bond l-1 and to the
// right of bond l reduce to the squared Schmidt weights, so
//   <O_l> = sum over alpha, beta, s, s' of lam[l-1]_alpha^2 lam[l]_beta^2 conj(Gamma[l]^s_{alpha beta})
//           O_{s s'} Gamma[l]^{s'}_{alpha beta}
// (lam = 1 beyond the ends): a reduction over site l's tensor only.  One CTA per (site, operator) pair.
//
// Sampling.  Bits are drawn site by site by the chain rule of the Born probabilities.  With the prefix vector
// v^(k)_beta = (Gamma[0]^{s_0} lam[0] Gamma[1]^{s_1} ... lam[k-1] Gamma[k]^{s_k})_beta, the marginal of a prefix
// is sum over beta of |v^(k)_beta|^2 lam[k]_beta^2, because the sites to the right are orthonormal in the
// weights.  Site k takes s_k = 1 when the uniform number u_k >= p(prefix, 0) / p(prefix), else 0 (inverse
// CDF; the uniforms are inputs).  The prefix vector is renormalised after every site (divided by the square
// root of its marginal), so p(prefix) is 1 at every step and the probability of the string is the product of
// the chosen conditional marginals.  One CTA per shot; the prefix vectors live in the context's MPS
// workspace.
#include <vector>
#include <algorithm>
#include "common.cuh"
#include "mw.cuh"
#include "reduce.cuh"
#include "prof.cuh"
#include "internal.cuh"
#include "mps.cuh"

namespace zkq {

template <int W>
__global__ void __launch_bounds__(256) mps_expect1_kernel(const double* const* __restrict__ tab, int n,
                                                         const int32_t* __restrict__ sites, const double* __restrict__ O,
                                                         double* __restrict__ out) {
  __shared__ cmw<W> buf[256];
  const int32_t* dims = reinterpret_cast<const int32_t*>(tab + 2 * n);
  const int q = blockIdx.x, l = sites[q];
  const int a = dims[l], b = dims[l + 1];
  const double* G = tab[l];
  const double* lL = l > 0 ? tab[n + l - 1] : nullptr;
  const double* lR = l < n - 1 ? tab[n + l] : nullptr;
  const double* Oq = O + (size_t)q * 4 * 2 * W;
  const cmw<W> o0 = c_load<W, W>(Oq, 0), o1 = c_load<W, W>(Oq, 1), o2 = c_load<W, W>(Oq, 2), o3 = c_load<W, W>(Oq, 3);
  cmw<W> acc = c_zero<W>();
  for (int e = threadIdx.x; e < a * b; e += blockDim.x) {
    const int al = e / b, be = e % b;
    const cmw<W> g0 = c_load<W, W>(G, (size_t)al * b + be);
    const cmw<W> g1 = c_load<W, W>(G, ((size_t)a + al) * b + be);
    const cmw<W> og0 = c_add(c_mul(o0, g0), c_mul(o1, g1));       // (O Gamma)^0
    const cmw<W> og1 = c_add(c_mul(o2, g0), c_mul(o3, g1));       // (O Gamma)^1
    cmw<W> u = c_add(c_mul_conj(g0, og0), c_mul_conj(g1, og1));
    mw<W> wt = mw_from<W>(1.0);
    if (lL) { const mw<W> x = mw_load<W, W>(lL, al); wt = mw_mul(x, x); }
    if (lR) { const mw<W> x = mw_load<W, W>(lR, be); wt = mw_mul(wt, mw_mul(x, x)); }
    acc = c_add(acc, c_scale(u, wt));
  }
  const cmw<W> tot = block_sum_c(acc, buf);
  if (threadIdx.x == 0) c_store(out, q, tot);
}

template <int W>
__global__ void __launch_bounds__(256) mps_sample_kernel(const double* const* __restrict__ tab, int n,
                                                        const double* __restrict__ u, int shot0, double* __restrict__ scratch,
                                                        int maxc, int32_t* __restrict__ bits, double* __restrict__ prob) {
  __shared__ mw<W> rbuf[256];
  const int32_t* dims = reinterpret_cast<const int32_t*>(tab + 2 * n);
  const size_t shot = (size_t)shot0 + blockIdx.x;
  const size_t vec = (size_t)maxc * 2 * W;
  double* lv = scratch + (size_t)blockIdx.x * 3 * vec;
  double* nv[2] = {lv + vec, lv + 2 * vec};
  if (threadIdx.x == 0) { cmw<W> one = c_zero<W>(); one.re = mw_from<W>(1.0); c_store(lv, 0, one); }
  mw<W> pstr = mw_from<W>(1.0);                     // probability of the prefix drawn so far
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const int a = dims[k], b = dims[k + 1];
    const double* G = tab[k];
    const double* lk = k < n - 1 ? tab[n + k] : nullptr;
    mw<W> p[2] = {mw_zero<W>(), mw_zero<W>()};
    for (int be = threadIdx.x; be < b; be += blockDim.x) {
      cmw<W> acc[2] = {c_zero<W>(), c_zero<W>()};
      for (int al = 0; al < a; ++al) {
        const cmw<W> x = c_load<W, W>(lv, al);
        acc[0] = c_add(acc[0], c_mul(x, c_load<W, W>(G, (size_t)al * b + be)));
        acc[1] = c_add(acc[1], c_mul(x, c_load<W, W>(G, ((size_t)a + al) * b + be)));
      }
      mw<W> wt = mw_from<W>(1.0);
      if (lk) { const mw<W> x = mw_load<W, W>(lk, be); wt = mw_mul(x, x); }
      for (int s = 0; s < 2; ++s) {
        c_store(nv[s], be, acc[s]);
        p[s] = mw_add(p[s], mw_mul(c_abs2(acc[s]), wt));
      }
    }
    p[0] = block_sum_r(p[0], rbuf);                  // every thread receives the same totals
    p[1] = block_sum_r(p[1], rbuf);
    // the prefix is normalised, so p(prefix) = 1: s_k = 1 iff u_k >= p(prefix, 0)
    const int s = mw_sub(mw_from<W>(u[shot * n + k]), p[0]).x[0] >= 0.0 ? 1 : 0;
    pstr = mw_mul(pstr, p[s]);
    if (threadIdx.x == 0) bits[shot * n + k] = s;
    if (k < n - 1) {
      const mw<W> inv = mw_recip(mw_sqrt(p[s]));
      for (int be = threadIdx.x; be < b; be += blockDim.x) {
        cmw<W> v = c_load<W, W>(nv[s], be);
        c_store(lv, be, c_scale(v, mw_mul(mw_load<W, W>(lk, be), inv)));
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) mw_store(prob, shot, pstr);
}

// rewrite the bond-dimension table behind the pointer table (host -> device, stream-ordered)
static zkq_status upload_dims(const zkq_mps* m, cudaStream_t st, std::vector<int32_t>* hd) {
  hd->assign(m->n + 1, 1);
  for (int l = 1; l < m->n; ++l) (*hd)[l] = m->chi[l - 1];
  int32_t* dd = reinterpret_cast<int32_t*>(m->d_ptrs + 2 * m->n);
  ZKQ_CUDA_TRY(cudaMemcpyAsync(dd, hd->data(), hd->size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  return ZKQ_OK;
}

}  // namespace zkq

using namespace zkq;

extern "C" zkq_status zkq_mps_expect1(zkq_ctx* ctx, const zkq_mps* m, int count, const int32_t* sites, const double* O,
                                      double* out, void* stream) try {
  if (!ctx || !m || count < 0 || (count > 0 && (!sites || !O || !out)) || ctx_device(ctx) != m->device) return ZKQ_EINVAL;
  if (count == 0) return ZKQ_OK;
  for (int q = 0; q < count; ++q) if (sites[q] < 0 || sites[q] >= m->n) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int W = m->W;
  // workspace: sites, operators, results
  const size_t b_sites = ((size_t)count * 4 + 255) & ~(size_t)255;
  const size_t b_ops = (size_t)count * 4 * 2 * W * sizeof(double);
  const size_t b_out = (size_t)count * 2 * W * sizeof(double);
  size_t* cap = nullptr;
  void** ws = ctx_mps_ws(ctx, &cap);
  const size_t need = b_sites + b_ops + b_out;
  if (need > *cap) {
    if (*ws) { cudaFree(*ws); *ws = nullptr; *cap = 0; }
    cudaError_t e = cudaMalloc(ws, need + need / 4);
    if (e != cudaSuccess) { set_last_cuda_error(e); *ws = nullptr; return ZKQ_ENOMEM; }
    *cap = need + need / 4;
  }
  char* base = (char*)*ws;
  int32_t* d_sites = (int32_t*)base;
  double* d_ops = (double*)(base + b_sites);
  double* d_out = (double*)(base + b_sites + b_ops);
  std::vector<int32_t> hd;
  zkq_status s = upload_dims(m, st, &hd);
  if (s != ZKQ_OK) return s;
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_sites, sites, (size_t)count * 4, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_ops, O, b_ops, cudaMemcpyHostToDevice, st));
  {
    ProfScope ps(PC_MPS, st);
    if (W == 2) mps_expect1_kernel<2><<<count, 256, 0, st>>>(m->d_ptrs, m->n, d_sites, d_ops, d_out);
    else mps_expect1_kernel<4><<<count, 256, 0, st>>>(m->d_ptrs, m->n, d_sites, d_ops, d_out);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  ZKQ_CUDA_TRY(cudaMemcpyAsync(out, d_out, b_out, cudaMemcpyDeviceToHost, st));
  ZKQ_CUDA_TRY(cudaStreamSynchronize(st));
  return ZKQ_OK;
} catch (...) {
  return api_exception(ctx);
}

extern "C" zkq_status zkq_mps_sample(zkq_ctx* ctx, const zkq_mps* m, int shots, const double* u, int32_t* bits,
                                     double* prob, void* stream) try {
  if (!ctx || !m || shots < 0 || (shots > 0 && (!u || !bits || !prob)) || ctx_device(ctx) != m->device) return ZKQ_EINVAL;
  if (shots == 0) return ZKQ_OK;
  const int n = m->n, W = m->W;
  for (size_t i = 0; i < (size_t)shots * n; ++i) if (!(u[i] >= 0.0 && u[i] < 1.0)) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  int maxc = 1;
  for (int c : m->chi) maxc = std::max(maxc, c);
  const int chunk = std::min(shots, 4 * std::max(1, ctx_num_sms(ctx)));
  const size_t b_u = (((size_t)shots * n * sizeof(double)) + 255) & ~(size_t)255;
  const size_t b_bits = (((size_t)shots * n * 4) + 255) & ~(size_t)255;
  const size_t b_prob = (((size_t)shots * W * sizeof(double)) + 255) & ~(size_t)255;
  const size_t b_vec = (size_t)chunk * 3 * maxc * 2 * W * sizeof(double);
  size_t* cap = nullptr;
  void** ws = ctx_mps_ws(ctx, &cap);
  const size_t need = b_u + b_bits + b_prob + b_vec;
  if (need > *cap) {
    if (*ws) { cudaFree(*ws); *ws = nullptr; *cap = 0; }
    cudaError_t e = cudaMalloc(ws, need + need / 4);
    if (e != cudaSuccess) { set_last_cuda_error(e); *ws = nullptr; return ZKQ_ENOMEM; }
    *cap = need + need / 4;
  }
  char* base = (char*)*ws;
  double* d_u = (double*)base;
  int32_t* d_bits = (int32_t*)(base + b_u);
  double* d_prob = (double*)(base + b_u + b_bits);
  double* d_vec = (double*)(base + b_u + b_bits + b_prob);
  std::vector<int32_t> hd;
  zkq_status s = upload_dims(m, st, &hd);
  if (s != ZKQ_OK) return s;
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_u, u, (size_t)shots * n * sizeof(double), cudaMemcpyHostToDevice, st));
  for (int s0 = 0; s0 < shots; s0 += chunk) {
    const int cnt = std::min(chunk, shots - s0);
    ProfScope ps(PC_MPS, st);
    if (W == 2) mps_sample_kernel<2><<<cnt, 256, 0, st>>>(m->d_ptrs, n, d_u, s0, d_vec, maxc, d_bits, d_prob);
    else mps_sample_kernel<4><<<cnt, 256, 0, st>>>(m->d_ptrs, n, d_u, s0, d_vec, maxc, d_bits, d_prob);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  ZKQ_CUDA_TRY(cudaMemcpyAsync(bits, d_bits, (size_t)shots * n * 4, cudaMemcpyDeviceToHost, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(prob, d_prob, (size_t)shots * W * sizeof(double), cudaMemcpyDeviceToHost, st));
  ZKQ_CUDA_TRY(cudaStreamSynchronize(st));
  return ZKQ_OK;
} catch (...) {
  return api_exception(ctx);
}
