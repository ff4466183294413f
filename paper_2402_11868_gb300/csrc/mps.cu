// Device-resident matrix-product state in Vidal's form and its two-site gate update (Section 1: an MPS
// is a nested Schmidt decomposition evolved without leaving that form; the diagonalisation at each gate
// is the dominant cost, Section 2.1; the working precision must resolve Schmidt coefficients ~2^{-(n-1)/2},
// footnote).  State: Gamma[l] (2 x chi_{l-1} x chi_l, complex, W words) and lambda[l] (chi_l, real).
//
// Gate G (4x4, row-major in (i j) x (k m), i the bit of `site`) on (site, site+1) = (l, l+1):
//   theta_{ij}[alpha, gamma] = sum_{k,m} G_{ij,km} (L_{l-1} Gamma[l]^k L_l Gamma[l+1]^m L_{l+1})[alpha, gamma]
//   M[(i, alpha), (j, gamma)] = theta_{ij}[alpha, gamma]            (2a x 2d; a = chi_{l-1}, d = chi_{l+1})
//   left Gram (2a <= 2d):  rho = M M^H = U diag(sigma^2) U^H
//       Gamma'[l]^i_{alpha beta} = U[(i,alpha), beta] / lambda_{l-1, alpha}
//       Gamma'[l+1]^j_{beta gamma} = (U^H M)[beta, (j,gamma)] / (sigma_beta lambda_{l+1, gamma})
//   right Gram (2d < 2a): rho = M^H M = V diag(sigma^2) V^H
//       Gamma'[l+1]^j_{beta gamma} = conj(V[(j,gamma), beta]) / lambda_{l+1, gamma}
//       Gamma'[l]^i_{alpha beta} = (M V)[(i,alpha), beta] / (lambda_{l-1, alpha} sigma_beta)
//   keep beta with sigma_beta^2 > tau sum sigma^2, at most r_max; lambda'_beta = sigma_beta / sqrt(sum kept).
// The eigensolve of rho is the library's FP64 Jacobi + refinement to W words; products are split products.
#include <new>
#include <mutex>
#include <vector>
#include <algorithm>
#include <cstring>
#include "common.cuh"
#include "mw.cuh"
#include "ozaki.cuh"
#include "prof.cuh"
#include "internal.cuh"
#include "mps.cuh"

namespace zkq {


// ------------------------------------------------------------------------------------------------------
// kernels (one thread per element)
template <int W>
__global__ void mps_scale_kernel(const double* __restrict__ G, const double* __restrict__ lamL,
                                 const double* __restrict__ lamR, int rows, int cols, double* __restrict__ out) {
  // out[s][r][c] = lamL[r] * G[s][r][c] * lamR[c]   (lamL / lamR may be null = 1); G row-major (s, r, c)
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * rows * cols) return;
  int c = e % cols, r = (e / cols) % rows;
  cmw<W> v = c_load<W, W>(G, e);
  if (lamL) v = c_scale(v, mw_load<W, W>(lamL, r));
  if (lamR) v = c_scale(v, mw_load<W, W>(lamR, c));
  c_store(out, e, v);
}
// column-major copies of the four k/m slices for the products:  Mk (a x c) and Nm (c x d)
template <int W>
__global__ void mps_to_colmajor_kernel(const double* __restrict__ src, int rows, int cols, double* __restrict__ dst) {
  // src row-major (s, r, c) -> dst column-major per s: dst[s][r + c rows]
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * rows * cols) return;
  int c = e % cols, r = (e / cols) % rows, s = e / (rows * cols);
  c_store(dst, (size_t)s * rows * cols + r + (size_t)c * rows, c_load<W, W>(src, e));
}
// M[(i, alpha), (j, gamma)] = sum_{km} G[ij, km] T_km[alpha, gamma];  T_km column-major a x d at T + km*a*d
template <int W>
__global__ void mps_theta_kernel(const double* __restrict__ T, const double* __restrict__ Gd, int a, int d,
                                 double* __restrict__ M) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * a * d) return;
  const int R = 2 * a;
  int row = e % R, col = e / R;
  int i = row / a, alpha = row % a, j = col / d, gamma = col % d;
  cmw<W> s = c_zero<W>();
  for (int km = 0; km < 4; ++km) {
    cmw<W> g = c_load<W, W>(Gd, (size_t)(2 * i + j) * 4 + km);
    s = c_add(s, c_mul(g, c_load<W, W>(T, (size_t)km * a * d + alpha + (size_t)gamma * a)));
  }
  c_store(M, (size_t)row + (size_t)col * R, s);
}
template <int W>
__global__ void mps_conj_transpose_kernel(const double* __restrict__ M, int rows, int cols, double* __restrict__ MH) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int r = e % rows, c = e / rows;
  c_store(MH, (size_t)c + (size_t)r * cols, c_conj(c_load<W, W>(M, e)));
}
// Gamma'[l]^i_{alpha beta} = Y[(i,alpha), beta] * rowscale  with Y column-major (2a x chi), rowscale 1/lambda_{l-1}
// colscale (optional) 1/sigma_beta; conj_src: Y holds V (right Gram) used as conj(V)^T for Gamma'[l+1]
template <int W>
__global__ void mps_split_left_kernel(const double* __restrict__ Y, int a, int chi, const double* __restrict__ lamL,
                                      const double* __restrict__ sig, double* __restrict__ Gout) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * a * chi) return;
  int beta = e % chi, alpha = (e / chi) % a, i = e / (a * chi);
  cmw<W> v = c_load<W, W>(Y, (size_t)(i * a + alpha) + (size_t)beta * 2 * a);
  if (lamL) v = c_make(mw_div(v.re, mw_load<W, W>(lamL, alpha)), mw_div(v.im, mw_load<W, W>(lamL, alpha)));
  if (sig) v = c_make(mw_div(v.re, mw_load<W, W>(sig, beta)), mw_div(v.im, mw_load<W, W>(sig, beta)));
  c_store(Gout, e, v);   // row-major (i, alpha, beta)
}
// Gamma'[l+1]^j_{beta gamma} from Z[beta, (j,gamma)] (Z column-major chi x 2d)  or from conj(V[(j,gamma), beta])
template <int W>
__global__ void mps_split_right_kernel(const double* __restrict__ Z, int chi, int d, int from_v,
                                       const double* __restrict__ lamR, const double* __restrict__ sig,
                                       double* __restrict__ Gout) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * chi * d) return;
  int gamma = e % d, beta = (e / d) % chi, j = e / (chi * d);
  cmw<W> v = from_v ? c_conj(c_load<W, W>(Z, (size_t)(j * d + gamma) + (size_t)beta * 2 * d))
                    : c_load<W, W>(Z, (size_t)beta + (size_t)(j * d + gamma) * chi);
  if (lamR) v = c_make(mw_div(v.re, mw_load<W, W>(lamR, gamma)), mw_div(v.im, mw_load<W, W>(lamR, gamma)));
  if (sig) v = c_make(mw_div(v.re, mw_load<W, W>(sig, beta)), mw_div(v.im, mw_load<W, W>(sig, beta)));
  c_store(Gout, e, v);   // row-major (j, beta, gamma)
}
// sigma_beta = sqrt(max(eig, 0)), lambda'_beta = sigma_beta / sqrt(kept weight); one thread per beta
template <int W>
__global__ void mps_sigma_kernel(const double* __restrict__ eig, int chi, const double* __restrict__ norm2,
                                 double* __restrict__ sig, double* __restrict__ lam_new) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= chi) return;
  mw<W> e = mw_load<W, W>(eig, b);
  if (e.x[0] < 0) e = mw_zero<W>();
  mw<W> s = mw_sqrt(e);
  mw_store(sig, b, s);
  mw_store(lam_new, b, mw_div(s, mw_sqrt(mw_load<W, W>(norm2, 0))));
}
// kept weight = sum of the first chi eigenvalues (one thread, chi <= 4096)
template <int W>
__global__ void mps_weight_kernel(const double* __restrict__ eig, int chi, int ntot, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  mw<W> k = mw_zero<W>(), t = mw_zero<W>();
  for (int b = 0; b < ntot; ++b) {
    mw<W> e = mw_load<W, W>(eig, b);
    if (e.x[0] < 0) e = mw_zero<W>();
    t = mw_add(t, e);
    if (b < chi) k = mw_add(k, e);
  }
  mw_store(out, 0, k);
  mw_store(out, 1, t);
}
// one-qubit gate on a Gamma tensor (row-major (s, r, c)): Gamma^i <- sum_k U_ik Gamma^k
template <int W>
__global__ void mps_apply1_kernel(double* __restrict__ G, int rows, int cols, const double* __restrict__ Ud) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  cmw<W> g0 = c_load<W, W>(G, e), g1 = c_load<W, W>(G, (size_t)rows * cols + e);
  cmw<W> n0 = c_add(c_mul(c_load<W, W>(Ud, 0), g0), c_mul(c_load<W, W>(Ud, 1), g1));
  cmw<W> n1 = c_add(c_mul(c_load<W, W>(Ud, 2), g0), c_mul(c_load<W, W>(Ud, 3), g1));
  c_store(G, e, n0);
  c_store(G, (size_t)rows * cols + e, n1);
}
template <int W>
__global__ void mps_init_kernel(double* __restrict__ G, size_t elems) {   // Gamma^0 = 1, Gamma^1 = 0 (1x1)
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= elems) return;
  c_store(G, e, c_zero<W>());
  if (e == 0) { cmw<W> one = c_zero<W>(); one.re = mw_from<W>(1.0); c_store(G, 0, one); }
}

}  // namespace zkq

using namespace zkq;


static inline int left_dim(const zkq_mps* m, int l) { return l == 0 ? 1 : m->chi[l - 1]; }
static inline int right_dim(const zkq_mps* m, int l) { return l == m->n - 1 ? 1 : m->chi[l]; }
static inline int left_cap(const zkq_mps* m, int l) { return l == 0 ? 1 : m->cap[l - 1]; }
static inline int right_cap(const zkq_mps* m, int l) { return l == m->n - 1 ? 1 : m->cap[l]; }

template <int W> static unsigned blocks(size_t n) { return (unsigned)((n + 255) / 256); }

// Bond capacities: the Schmidt rank across bond l is at most 2^min(l+1, n-l-1), and at most r_max.
static std::vector<int> mps_caps(int n_qubits, int r_max) {
  std::vector<int> cap(n_qubits - 1);
  for (int l = 0; l < n_qubits - 1; ++l) {
    long long lim = 1;
    int e = std::min(l + 1, n_qubits - l - 1);
    for (int k = 0; k < e && lim < r_max; ++k) lim *= 2;
    cap[l] = (int)std::min<long long>(lim, r_max);
  }
  return cap;
}

// Device bytes an MPS handle allocates: Gamma per site at capacity, lambda per bond, the gate buffer and the
// pointer table (the allocations of mps_build).
static size_t mps_state_bytes(int n_qubits, int words, const std::vector<int>& cap) {
  const size_t wb = (size_t)words * sizeof(double);
  size_t tot = 0;
  for (int l = 0; l < n_qubits; ++l) {
    const size_t a = l == 0 ? 1 : cap[l - 1], b = l == n_qubits - 1 ? 1 : cap[l];
    tot += 2 * a * b * 2 * wb;
  }
  for (int l = 0; l < n_qubits - 1; ++l) tot += (size_t)cap[l] * wb;
  tot += 16 * 2 * wb;
  tot += (size_t)(2 * n_qubits) * sizeof(double*) + (size_t)(n_qubits + 1) * sizeof(int32_t);
  return tot;
}

// Scratch layout of one two-site gate update (offsets in doubles) for bond dimensions a (left), c (middle),
// d (right): theta operands, M and M^H, rho, the FP64 and refined eigenpairs, the split-back product, and
// the SVD variant's buffers.
struct GateScratch {
  size_t Mk, Nm, Mc, Nc, T, M, MH, Rho, W64, V64, Wq, Vq, Err, Info, Y, Sig, Norm, SvdX, SvdS, total;
};
static GateScratch gate_scratch(int a, int c, int d, int W, bool svd) {
  const size_t E = 2 * W;
  const int R = 2 * a, C = 2 * d, g = std::min(R, C);
  GateScratch L{};
  size_t off = 0;
  auto take = [&](size_t doubles) { size_t o = off; off += (doubles + 31) & ~(size_t)31; return o; };
  L.Mk = take(2 * (size_t)a * c * E); L.Nm = take(2 * (size_t)c * d * E);
  L.Mc = take(2 * (size_t)a * c * E); L.Nc = take(2 * (size_t)c * d * E);
  L.T = take(4 * (size_t)a * d * E); L.M = take((size_t)R * C * E); L.MH = take((size_t)R * C * E);
  L.Rho = take((size_t)g * g * E); L.W64 = take(g); L.V64 = take(2 * (size_t)g * g);
  L.Wq = take((size_t)g * W); L.Vq = take((size_t)g * g * E); L.Err = take(g); L.Info = take(8);
  L.Y = take((size_t)std::max(R, C) * g * E);
  L.Sig = take((size_t)g * W); L.Norm = take(2 * W);
  L.SvdX = svd ? take(2 * (size_t)std::max(R, C) * g) : 0;   // the SVD's vectors of the larger side
  L.SvdS = svd ? take(g) : 0;
  L.total = off;
  return L;
}

// |0...0> on the context's device; on failure the caller frees m (whatever it holds by then)
// The MPS's buffers come from the device's stream-ordered pool (cudaMallocAsync / cudaFreeAsync), so that
// creating or destroying a simulation does not synchronise the whole device: a serving loop admits and
// retires simulations while other streams keep computing.  Freed memory stays cached in the pool for the
// next simulation (release threshold raised once per device).
static zkq_status pool_keep_memory(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> g(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return ZKQ_OK;
  cudaMemPool_t pool;
  ZKQ_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = ~0ULL;
  ZKQ_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  done.push_back(dev);
  return ZKQ_OK;
}

namespace {
struct TempStream {                       // a private stream, synchronised and destroyed on every exit path
  cudaStream_t s = nullptr;
  ~TempStream() { if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); } }
};
}  // namespace

static zkq_status mps_build(zkq_ctx* ctx, zkq_mps* m, int n_qubits, int r_max, int words) {
  m->n = n_qubits; m->r_max = r_max; m->W = words;
  m->device = ctx_device(ctx);
  ZKQ_CUDA_TRY(cudaSetDevice(m->device));
  zkq_status ps = pool_keep_memory(m->device);
  if (ps != ZKQ_OK) return ps;
  m->chi.assign(n_qubits - 1, 1);
  m->cap = mps_caps(n_qubits, r_max);
  m->gamma.reserve(n_qubits);                  // the push_backs below cannot throw and lose a device buffer
  m->lam.reserve(n_qubits - 1);
  const std::vector<double> one = [&] { std::vector<double> v(words, 0.0); v[0] = 1.0; return v; }();
  std::vector<double*> tab(2 * n_qubits, nullptr);
  TempStream ts;
  ZKQ_CUDA_TRY(cudaStreamCreateWithFlags(&ts.s, cudaStreamNonBlocking));
  const cudaStream_t st = ts.s;
  size_t wb = (size_t)words * sizeof(double);
  for (int l = 0; l < n_qubits; ++l) {
    size_t elems = (size_t)2 * left_cap(m, l) * right_cap(m, l);
    double* g = nullptr;
    cudaError_t e = cudaMallocAsync(&g, elems * 2 * wb, st);
    if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ENOMEM; }
    m->gamma.push_back(g);
    if (words == 2) mps_init_kernel<2><<<blocks<2>(elems), 256, 0, st>>>(g, elems);
    else mps_init_kernel<4><<<blocks<4>(elems), 256, 0, st>>>(g, elems);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  for (int l = 0; l < n_qubits - 1; ++l) {
    double* v = nullptr;
    cudaError_t e = cudaMallocAsync(&v, (size_t)m->cap[l] * wb, st);
    if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ENOMEM; }
    m->lam.push_back(v);
    ZKQ_CUDA_TRY(cudaMemcpyAsync(v, one.data(), wb, cudaMemcpyHostToDevice, st));
  }
  cudaError_t e = cudaMallocAsync(&m->gate, 16 * 2 * wb, st);
  if (e != cudaSuccess) { set_last_cuda_error(e); m->gate = nullptr; return ZKQ_ENOMEM; }
  // device tables of the site and bond pointers (fixed for the life of the MPS) and of the bond dimensions
  e = cudaMallocAsync(&m->d_ptrs, (size_t)(2 * n_qubits) * sizeof(double*) + (size_t)(n_qubits + 1) * sizeof(int32_t), st);
  if (e != cudaSuccess) { set_last_cuda_error(e); m->d_ptrs = nullptr; return ZKQ_ENOMEM; }
  for (int l = 0; l < n_qubits; ++l) tab[l] = m->gamma[l];
  for (int l = 0; l < n_qubits - 1; ++l) tab[n_qubits + l] = m->lam[l];
  ZKQ_CUDA_TRY(cudaMemcpyAsync(m->d_ptrs, tab.data(), tab.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaStreamSynchronize(st));    // the buffers are ready for any stream from here on
  return ZKQ_OK;
}

extern "C" {

zkq_status zkq_mps_create(zkq_ctx* ctx, int n_qubits, int r_max, int words, zkq_mps** out) {
  if (!ctx || !out || n_qubits < 2 || n_qubits > 4096 || r_max < 1 || r_max > 2048 || (words != 2 && words != 4))
    return ZKQ_EINVAL;
  *out = nullptr;
  zkq_mps* m = new (std::nothrow) zkq_mps();
  if (!m) return ZKQ_ENOMEM;
  zkq_status s;
  try { s = mps_build(ctx, m, n_qubits, r_max, words); } catch (...) { s = api_exception(nullptr); }
  if (s != ZKQ_OK) { zkq_mps_destroy(m); return s; }
  *out = m;
  return ZKQ_OK;
}

// Every MPS call but apply1q synchronises its stream before returning; apply1q records an event behind its
// kernel.  Destroy orders the frees after that event on a private stream, so no device-wide
// synchronisation is needed.
zkq_status zkq_mps_destroy(zkq_mps* m) {
  if (!m) return ZKQ_OK;
  cudaSetDevice(m->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  if (st && m->done) cudaStreamWaitEvent(st, m->done, 0);
  if (!st) cudaDeviceSynchronize();            // fallback: no stream could be made
  for (double* p : m->gamma) if (p) cudaFreeAsync(p, st);
  for (double* p : m->lam) if (p) cudaFreeAsync(p, st);
  if (m->gate) cudaFreeAsync(m->gate, st);
  if (m->d_ptrs) cudaFreeAsync(m->d_ptrs, st);
  if (st) cudaStreamDestroy(st);               // released once its frees have run
  if (m->done) cudaEventDestroy(m->done);
  delete m;
  return ZKQ_OK;
}

zkq_status zkq_mps_bond_dims(const zkq_mps* m, int32_t* chi) {
  if (!m || !chi) return ZKQ_EINVAL;
  for (int l = 0; l < m->n - 1; ++l) chi[l] = m->chi[l];
  return ZKQ_OK;
}

// Host copies in the oracle's layout: Gamma[l] row-major (s, alpha, beta) concatenated over l; lambda[l]
// concatenated over l; W words per real.
zkq_status zkq_mps_download(const zkq_mps* m, double* gammas, double* lambdas, void* stream) {
  if (!m || !gammas || !lambdas) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  size_t go = 0, lo = 0, wb = (size_t)m->W * sizeof(double);
  for (int l = 0; l < m->n; ++l) {
    size_t elems = (size_t)2 * left_dim(m, l) * right_dim(m, l);
    ZKQ_CUDA_TRY(cudaMemcpyAsync(gammas + go * 2 * m->W, m->gamma[l], elems * 2 * wb, cudaMemcpyDeviceToHost, st));
    go += elems;
  }
  for (int l = 0; l < m->n - 1; ++l) {
    ZKQ_CUDA_TRY(cudaMemcpyAsync(lambdas + lo * m->W, m->lam[l], (size_t)m->chi[l] * wb, cudaMemcpyDeviceToHost, st));
    lo += m->chi[l];
  }
  ZKQ_CUDA_TRY(cudaStreamSynchronize(st));
  return ZKQ_OK;
}

zkq_status zkq_mps_upload(zkq_mps* m, const int32_t* chi, const double* gammas, const double* lambdas, void* stream) {
  if (!m || !chi || !gammas || !lambdas) return ZKQ_EINVAL;
  for (int l = 0; l < m->n - 1; ++l) if (chi[l] < 1 || chi[l] > m->cap[l]) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  for (int l = 0; l < m->n - 1; ++l) m->chi[l] = chi[l];
  size_t go = 0, lo = 0, wb = (size_t)m->W * sizeof(double);
  for (int l = 0; l < m->n; ++l) {
    size_t elems = (size_t)2 * left_dim(m, l) * right_dim(m, l);
    ZKQ_CUDA_TRY(cudaMemcpyAsync(m->gamma[l], gammas + go * 2 * m->W, elems * 2 * wb, cudaMemcpyHostToDevice, st));
    go += elems;
  }
  for (int l = 0; l < m->n - 1; ++l) {
    ZKQ_CUDA_TRY(cudaMemcpyAsync(m->lam[l], lambdas + lo * m->W, (size_t)chi[l] * wb, cudaMemcpyHostToDevice, st));
    lo += chi[l];
  }
  ZKQ_CUDA_TRY(cudaStreamSynchronize(st));
  return ZKQ_OK;
}

zkq_status zkq_mps_apply1q(zkq_ctx* ctx, zkq_mps* m, int site, const double* U, void* stream) {
  if (!ctx || !m || !U || site < 0 || site >= m->n || ctx_device(ctx) != m->device) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int W = m->W;
  ZKQ_CUDA_TRY(cudaMemcpyAsync(m->gate, U, 4 * 2 * W * sizeof(double), cudaMemcpyHostToDevice, st));
  int rows = left_dim(m, site), cols = right_dim(m, site);
  {
    ProfScope ps(PC_MPS, st);
    if (W == 2) mps_apply1_kernel<2><<<blocks<2>((size_t)rows * cols), 256, 0, st>>>(m->gamma[site], rows, cols, m->gate);
    else mps_apply1_kernel<4><<<blocks<4>((size_t)rows * cols), 256, 0, st>>>(m->gamma[site], rows, cols, m->gate);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  if (!m->done) ZKQ_CUDA_TRY(cudaEventCreateWithFlags(&m->done, cudaEventDisableTiming));
  ZKQ_CUDA_TRY(cudaEventRecord(m->done, st));   // destroy waits for this
  return ZKQ_OK;
}

}  // extern "C"

template <int W>
static zkq_status apply2q_t(zkq_ctx* ctx, zkq_mps* m, int l, const double* G, double tau, int method,
                            int32_t* new_bond, double* discarded, cudaStream_t st) {
  const int a = left_dim(m, l), c = m->chi[l], d = right_dim(m, l + 1);
  const double* lamL = l > 0 ? m->lam[l - 1] : nullptr;
  const double* lamC = m->lam[l];
  const double* lamR = (l + 1 < m->n - 1) ? m->lam[l + 1] : nullptr;
  const size_t E = 2 * W;                                   // doubles per complex element
  const int R = 2 * a, C = 2 * d;
  const bool left = R <= C;                                 // Gram matrix of the smaller side (ties: left)
  const int g = left ? R : C;
  const bool svd = method == ZKQ_SVD_OA;
  const GateScratch gs = gate_scratch(a, c, d, W, svd);
  const size_t oMk = gs.Mk, oNm = gs.Nm, oMc = gs.Mc, oNc = gs.Nc, oT = gs.T, oM = gs.M, oMH = gs.MH, oRho = gs.Rho;
  const size_t oW64 = gs.W64, oV64 = gs.V64, oWq = gs.Wq, oVq = gs.Vq, oErr = gs.Err, oInfo = gs.Info, oY = gs.Y;
  const size_t oSig = gs.Sig, oNorm = gs.Norm, oSvdX = gs.SvdX, oSvdS = gs.SvdS;
  const size_t off = gs.total;
  size_t* cap_bytes = nullptr;
  void** ws = ctx_mps_ws(ctx, &cap_bytes);
  size_t need = off * sizeof(double);
  if (need > *cap_bytes) {
    if (*ws) { cudaFree(*ws); *ws = nullptr; *cap_bytes = 0; }
    cudaError_t e = cudaMalloc(ws, need + need / 4);
    if (e != cudaSuccess) { set_last_cuda_error(e); *ws = nullptr; return ZKQ_ENOMEM; }
    *cap_bytes = need + need / 4;
  }
  double* b = (double*)*ws;
  double *Mk = b + oMk, *Nm = b + oNm, *Mc = b + oMc, *Nc = b + oNc, *T = b + oT, *M = b + oM, *MH = b + oMH;
  double *Rho = b + oRho, *W64 = b + oW64, *V64 = b + oV64, *Wq = b + oWq, *Vq = b + oVq, *Err = b + oErr;
  int32_t* Info = (int32_t*)(b + oInfo);
  double *Y = b + oY, *Sig = b + oSig, *Norm = b + oNorm;
  ZKQ_CUDA_TRY(cudaMemcpyAsync(m->gate, G, 16 * E * sizeof(double), cudaMemcpyHostToDevice, st));
  {
    ProfScope ps(PC_MPS, st);
    // Mk = L_{l-1} Gamma[l]^k L_l, Nm = Gamma[l+1]^m L_{l+1}; to column-major
    mps_scale_kernel<W><<<blocks<W>(2 * (size_t)a * c), 256, 0, st>>>(m->gamma[l], lamL, lamC, a, c, Mk);
    mps_scale_kernel<W><<<blocks<W>(2 * (size_t)c * d), 256, 0, st>>>(m->gamma[l + 1], nullptr, lamR, c, d, Nm);
    mps_to_colmajor_kernel<W><<<blocks<W>(2 * (size_t)a * c), 256, 0, st>>>(Mk, a, c, Mc);
    mps_to_colmajor_kernel<W><<<blocks<W>(2 * (size_t)c * d), 256, 0, st>>>(Nm, c, d, Nc);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  OaBuffers ob = ctx_oa_buffers(ctx);
  const int p_bits = 53 * W + 6;
  // T_km = Mc_k Nc_m (4 products a x c x d)
  std::vector<MwProd> pr;
  for (int k = 0; k < 2; ++k)
    for (int mm = 0; mm < 2; ++mm)
      pr.push_back({a, d, c, 0, Mc + (size_t)k * a * c * E, Nc + (size_t)mm * c * d * E,
                    T + (size_t)(2 * k + mm) * a * d * E, nullptr, 1.0, 0});
  zkq_status s = mw_gemm_batched(pr.data(), 4, W, W, W, p_bits, 1, ob.oz_ws, ob.oz_bytes, ob.oz_meta, ob.oz_meta_bytes, st, ob.stage);
  if (s != ZKQ_OK) return s;
  {
    ProfScope ps(PC_MPS, st);
    mps_theta_kernel<W><<<blocks<W>(4 * (size_t)a * d), 256, 0, st>>>(T, m->gate, a, d, M);
    mps_conj_transpose_kernel<W><<<blocks<W>((size_t)R * C), 256, 0, st>>>(M, R, C, MH);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  // rho = M M^H (op(A) = (M^H)^H with A = MH stored C x R, B = MH) or M^H M (A = M stored R x C, B = M)
  MwProd pg = left ? MwProd{R, R, C, 1, MH, MH, Rho, nullptr, 1.0, 0} : MwProd{C, C, R, 1, M, M, Rho, nullptr, 1.0, 0};
  pg.hermitian = 1;
  s = mw_gemm_batched(&pg, 1, W, W, W, p_bits, 1, ob.oz_ws, ob.oz_bytes, ob.oz_meta, ob.oz_meta_bytes, st, ob.stage);
  if (s != ZKQ_OK) return s;
  // eigen-decomposition of rho (descending), refined to W words
  int32_t nn = g; int64_t zero = 0;
  if (svd) {
    // the eigenvectors of rho are M's singular vectors on the Gram side: U (R x g) for M M^H, V (C x g) for
    // M^H M; the FP64 SVD computes them without squaring M's conditioning
    int32_t mr = R, mc = C;
    const int64_t u_off = 0, v_off = 0;
    void **fws, **fmeta; size_t *fws_b, *fmeta_b;
    ctx_fp64_bufs(ctx, &fws, &fws_b, &fmeta, &fmeta_b);
    double* Ux = left ? V64 : b + oSvdX;
    double* Vx = left ? b + oSvdX : V64;
    s = svd_internal(ctx, 1, &mr, &mc, &zero, M, W, b + oSvdS, Ux, &u_off, Vx, &v_off, Info, st, fws, fws_b, fmeta, fmeta_b);
    if (s != ZKQ_OK) return s;
  } else {
    s = eigh_internal(ctx, 1, &nn, &zero, Rho, W, W64, V64, Info, st);
    if (s != ZKQ_OK) return s;
  }
  if (method == ZKQ_PLAIN_RQI)
    s = rqi_refine_internal(ctx, 1, &nn, &zero, Rho, W, W64, V64, W, Wq, Vq, Err, Info + 1, st);
  else
    s = oa_refine(ctx, ob, 1, &nn, &zero, Rho, W, V64, W, Wq, Vq, Err, Info + 1, ctx_oa_max_iter(ctx), method == ZKQ_OA_FP64 ? 0 : 1, st);
  if (s != ZKQ_OK) return s;
  // truncation (host reads the eigenvalues' leading words: the new bond dimension is a host decision)
  std::vector<double> ev((size_t)g * W);
  ZKQ_CUDA_TRY(cudaMemcpyAsync(ev.data(), Wq, ev.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  int32_t hinfo[2] = {0, 0};
  ZKQ_CUDA_TRY(cudaMemcpyAsync(hinfo, Info, sizeof(hinfo), cudaMemcpyDeviceToHost, st));
  ZKQ_CUDA_TRY(cudaStreamSynchronize(st));
  double tot = 0.0;
  for (int i = 0; i < g; ++i) tot += std::max(ev[(size_t)i * W], 0.0);
  int chi = 0;
  const int cap = m->cap[l];
  while (chi < g && chi < cap && chi < m->r_max && ev[(size_t)chi * W] > tau * tot) ++chi;
  if (chi == 0) chi = 1;
  {
    ProfScope ps(PC_MPS, st);
    mps_weight_kernel<W><<<1, 32, 0, st>>>(Wq, chi, g, Norm);
    mps_sigma_kernel<W><<<blocks<W>(chi), 256, 0, st>>>(Wq, chi, Norm, Sig, m->lam[l]);
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  // split back
  if (left) {
    // Z = U^H M  (chi x C): op(A) = U^H with A = U stored R x chi
    MwProd pz{chi, C, R, 1, Vq, M, Y, nullptr, 1.0, 0};
    s = mw_gemm_batched(&pz, 1, W, W, W, p_bits, 1, ob.oz_ws, ob.oz_bytes, ob.oz_meta, ob.oz_meta_bytes, st, ob.stage);
    if (s != ZKQ_OK) return s;
    ProfScope ps(PC_MPS, st);
    mps_split_left_kernel<W><<<blocks<W>(2 * (size_t)a * chi), 256, 0, st>>>(Vq, a, chi, lamL, nullptr, m->gamma[l]);
    mps_split_right_kernel<W><<<blocks<W>(2 * (size_t)chi * d), 256, 0, st>>>(Y, chi, d, 0, lamR, Sig, m->gamma[l + 1]);
  } else {
    // Y = M V (R x chi)
    MwProd py{R, chi, C, 0, M, Vq, Y, nullptr, 1.0, 0};
    s = mw_gemm_batched(&py, 1, W, W, W, p_bits, 1, ob.oz_ws, ob.oz_bytes, ob.oz_meta, ob.oz_meta_bytes, st, ob.stage);
    if (s != ZKQ_OK) return s;
    ProfScope ps(PC_MPS, st);
    mps_split_left_kernel<W><<<blocks<W>(2 * (size_t)a * chi), 256, 0, st>>>(Y, a, chi, lamL, Sig, m->gamma[l]);
    mps_split_right_kernel<W><<<blocks<W>(2 * (size_t)chi * d), 256, 0, st>>>(Vq, chi, d, 1, lamR, nullptr, m->gamma[l + 1]);
  }
  ZKQ_CUDA_TRY(cudaGetLastError());
  m->chi[l] = chi;
  std::vector<double> nrm(2 * W);
  ZKQ_CUDA_TRY(cudaMemcpyAsync(nrm.data(), Norm, nrm.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  ZKQ_CUDA_TRY(cudaStreamSynchronize(st));
  if (new_bond) *new_bond = chi;
  if (discarded) {
    double kept = 0, all = 0;
    for (int k = W - 1; k >= 0; --k) { kept += nrm[k]; all += nrm[W + k]; }
    *discarded = all > 0 ? (all - kept) / all : 0.0;
  }
  return (hinfo[0] == 0 && hinfo[1] == 0) ? ZKQ_OK : ZKQ_ENOCONV;
}

extern "C" zkq_status zkq_mps_footprint(zkq_ctx* ctx, int n_qubits, int r_max, int words, int method,
                                        size_t* state_bytes, size_t* gate_bytes) try {
  if (!ctx || !state_bytes || !gate_bytes || n_qubits < 2 || n_qubits > 4096 || r_max < 1 || r_max > 2048 ||
      (words != 2 && words != 4) || method < 0 || method > 3)
    return ZKQ_EINVAL;
  const std::vector<int> cap = mps_caps(n_qubits, r_max);
  *state_bytes = mps_state_bytes(n_qubits, words, cap);
  // the widest gate update: bond dimensions at capacity on both sides of a middle bond
  size_t worst = 0; int gmax = 1;
  for (int l = 0; l + 1 < n_qubits; ++l) {
    const int a = l == 0 ? 1 : cap[l - 1], c = cap[l], d = l + 1 == n_qubits - 1 ? 1 : cap[l + 1];
    const GateScratch gs = gate_scratch(a, c, d, words, method == ZKQ_SVD_OA);
    worst = std::max(worst, gs.total * sizeof(double));
    gmax = std::max(gmax, std::min(2 * a, 2 * d));
  }
  worst += worst / 4;                                   // the growth slack of the gate buffer
  size_t eig = 0;
  const int rm = method == ZKQ_SVD_OA ? ZKQ_OA_OZAKI : method;
  zkq_status s = zkq_workspace_size(ctx, 1, &gmax, words, words, rm, &eig);
  if (s != ZKQ_OK) return s;
  *gate_bytes = worst + eig;
  return ZKQ_OK;
} catch (...) {
  return api_exception(ctx);
}

extern "C" zkq_status zkq_mps_apply2q(zkq_ctx* ctx, zkq_mps* m, int site, const double* G, double trunc_tau, int method,
                                      int32_t* new_bond, double* discarded_weight, void* stream) try {
  if (!ctx || !m || !G || site < 0 || site + 1 >= m->n || !(trunc_tau >= 0.0) || method < 0 || method > 3 ||
      ctx_device(ctx) != m->device)
    return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (m->W == 2) return apply2q_t<2>(ctx, m, site, G, trunc_tau, method, new_bond, discarded_weight, st);
  return apply2q_t<4>(ctx, m, site, G, trunc_tau, method, new_bond, discarded_weight, st);
} catch (...) {
  return api_exception(ctx);
}
