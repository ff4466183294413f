// Autotuning of the batched Jacobi's cluster width: for each requested order, time the eigensolve of a
// synthetic batch (one problem per SM, so every width runs on the cluster path) at widths 2, 4, 8 and 16,
// and record the fastest in the context's table, which eigh_layout consults from then on.
#include <algorithm>
#include <vector>
#include "internal.cuh"

using namespace zkq;

namespace {
// a Hermitian test matrix per problem: entries from a counter hash in [-1, 1), real diagonal
__device__ __forceinline__ double hash01(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (double)(x >> 11) * 0x1p-52 - 1.0;
}
__global__ void tune_fill_kernel(double* A, int n, int count, int words) {
  const size_t tot = (size_t)count * n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / ((size_t)n * n), w = e % ((size_t)n * n);
    const int i = (int)(w % n), j = (int)(w / n);
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    const uint64_t key = ((uint64_t)b << 40) ^ ((uint64_t)lo << 20) ^ (uint64_t)hi;
    double re = hash01(2 * key), im = i == j ? 0.0 : hash01(2 * key + 1);
    if (i > j) im = -im;
    double* q = A + e * 2 * words;
    for (int k = 0; k < 2 * words; ++k) q[k] = 0.0;
    q[0] = re; q[words] = im;
  }
}
}  // namespace

extern "C" zkq_status zkq_autotune_jacobi(zkq_ctx* ctx, int nsizes, const int32_t* sizes, int a_words, int reps,
                                          int32_t* best) try {
  if (!ctx || nsizes < 1 || !sizes || !best || reps < 1) return ZKQ_EINVAL;
  if (a_words != 1 && a_words != 2 && a_words != 4) return ZKQ_EINVAL;
  for (int i = 0; i < nsizes; ++i) if (sizes[i] <= 80 || sizes[i] > 2048) return ZKQ_EINVAL;   // cluster-path orders
  ZKQ_CUDA_TRY(cudaSetDevice(ctx_device(ctx)));
  zkq_config& cfg = ctx_config_mut(ctx);
  const int saved = cfg.jacobi_cluster;
  const int count = ctx_num_sms(ctx);
  // host memory first: once device buffers exist, only the eigensolve may throw, and it is caught in place
  JacobiTune table;
  table.reserve(nsizes);
  std::vector<int32_t> nv(count);
  std::vector<int64_t> off(count);
  zkq_status s = ZKQ_OK;
  double *A = nullptr, *W = nullptr, *V = nullptr;
  int32_t* info = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  auto cu = [&](cudaError_t e) { if (e != cudaSuccess) { set_last_cuda_error(e); s = ZKQ_ECUDA; } return e == cudaSuccess; };
  if (!cu(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) || !cu(cudaEventCreate(&e0)) || !cu(cudaEventCreate(&e1)))
    goto done;
  for (int si = 0; si < nsizes && s == ZKQ_OK; ++si) {
    const int n = sizes[si];
    const size_t el = (size_t)count * n * n;
    if (!cu(cudaMalloc(&A, el * 2 * a_words * sizeof(double))) || !cu(cudaMalloc(&W, (size_t)count * n * sizeof(double))) ||
        !cu(cudaMalloc(&V, el * 2 * sizeof(double))) || !cu(cudaMalloc(&info, count * sizeof(int32_t)))) {
      s = ZKQ_ENOMEM; break;
    }
    tune_fill_kernel<<<ctx_num_sms(ctx) * 4, 256, 0, st>>>(A, n, count, a_words);
    if (!cu(cudaGetLastError())) break;
    for (int b = 0; b < count; ++b) { nv[b] = n; off[b] = (int64_t)b * n * n; }
    float bestms = 1e30f; int bestc = 0;
    for (int c : {2, 4, 8, 16}) {
      cfg.jacobi_cluster = c;
      float tmin = 1e30f;
      for (int r = 0; r <= reps && s == ZKQ_OK; ++r) {      // the first run warms up
        if (!cu(cudaEventRecord(e0, st))) break;
        try { s = eigh_internal(ctx, count, nv.data(), off.data(), A, a_words, W, V, info, st); }
        catch (...) { s = api_exception(ctx); }
        if (s != ZKQ_OK || !cu(cudaEventRecord(e1, st)) || !cu(cudaEventSynchronize(e1))) break;
        float ms = 0;
        if (!cu(cudaEventElapsedTime(&ms, e0, e1))) break;
        if (r > 0) tmin = std::min(tmin, ms);
      }
      if (s != ZKQ_OK) break;
      if (tmin < bestms) { bestms = tmin; bestc = c; }
    }
    cudaFree(A); cudaFree(W); cudaFree(V); cudaFree(info);
    A = W = V = nullptr; info = nullptr;
    if (s != ZKQ_OK) break;
    best[si] = bestc;
    table.push_back({n, bestc});
  }
done:
  cfg.jacobi_cluster = saved;
  if (A) cudaFree(A);
  if (W) cudaFree(W);
  if (V) cudaFree(V);
  if (info) cudaFree(info);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (s == ZKQ_OK) {
    std::sort(table.begin(), table.end());
    ctx_jacobi_tune(ctx)->swap(table);
  }
  return s;
} catch (...) {
  return api_exception(ctx);
}

// ---------------------------------------------------------------------------------------------------
// Autotuning of the split-product GEMM's tile width: for each requested order n (16..512, the CRT form's
// range K' = 2n <= 1024), time a synthetic batch of n x n x n complex products in `words` words per real
// (enough products to fill the GPU with 128-column tiles) with 256-column and with 128-column tiles on the
// tcgen05 kernel, and keep the faster in the process-wide table that every later split product consults.
#include "ozaki.cuh"

namespace {
__global__ void tune_fill_words_kernel(double* A, size_t elems, int words, uint64_t salt) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < elems; e += (size_t)gridDim.x * blockDim.x) {
    double* q = A + e * 2 * words;
    for (int p = 0; p < 2; ++p) {
      const double h = hash01((e << 1 | p) ^ salt);
      q[p * words] = h;
      double r = h;                                       // lower words: scaled hashes below the leading ulp
      for (int k = 1; k < words; ++k) { r = ldexp(hash01((e << 8 | p << 4 | k) ^ salt), -53 * k); q[p * words + k] = r; }
    }
  }
}
}  // namespace

extern "C" zkq_status zkq_autotune_gemm(zkq_ctx* ctx, int nsizes, const int32_t* sizes, int words, int reps,
                                        int32_t* best) try {
  if (!ctx || nsizes < 1 || !sizes || !best || reps < 1) return ZKQ_EINVAL;
  if (words != 1 && words != 2 && words != 4) return ZKQ_EINVAL;
  for (int i = 0; i < nsizes; ++i) if (sizes[i] < 16 || sizes[i] > 512) return ZKQ_EINVAL;
  if (gemm_kernel_get() != 1) return ZKQ_EINVAL;                 // the width choice is the tcgen05 kernel's
  ZKQ_CUDA_TRY(cudaSetDevice(ctx_device(ctx)));
  const std::vector<std::pair<int, int>> saved = gemm_wide_table_get();
  std::vector<std::pair<int, int>> table;
  table.reserve(nsizes);
  OaBuffers ob = ctx_oa_buffers(ctx);
  zkq_status s = ZKQ_OK;
  double *A = nullptr, *B = nullptr, *C = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  auto cu = [&](cudaError_t e) { if (e != cudaSuccess) { set_last_cuda_error(e); s = ZKQ_ECUDA; } return e == cudaSuccess; };
  if (!cu(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) || !cu(cudaEventCreate(&e0)) || !cu(cudaEventCreate(&e1)))
    goto done;
  for (int si = 0; si < nsizes && s == ZKQ_OK; ++si) {
    const int n = sizes[si];
    const int tiles_per = ((n + 127) / 128) * ((2 * n + 127) / 128);
    const int count = std::max(1, std::min(256, 4 * ctx_num_sms(ctx) / std::max(1, tiles_per)));
    const size_t el = (size_t)count * n * n;
    if (!cu(cudaMalloc(&A, el * 2 * words * sizeof(double))) || !cu(cudaMalloc(&B, el * 2 * words * sizeof(double))) ||
        !cu(cudaMalloc(&C, el * 2 * words * sizeof(double)))) { s = ZKQ_ENOMEM; break; }
    tune_fill_words_kernel<<<ctx_num_sms(ctx) * 4, 256, 0, st>>>(A, el, words, 0x51ULL + n);
    tune_fill_words_kernel<<<ctx_num_sms(ctx) * 4, 256, 0, st>>>(B, el, words, 0xB2ULL + n);
    if (!cu(cudaGetLastError())) break;
    std::vector<MwProd> pr;
    for (int b = 0; b < count; ++b) {
      const size_t o = (size_t)b * n * n * 2 * words;
      pr.push_back({n, n, n, 0, A + o, B + o, C + o, nullptr, 1.0, 0});
    }
    float t_w[2] = {1e30f, 1e30f};
    for (int wide = 1; wide >= 0 && s == ZKQ_OK; --wide) {
      gemm_wide_table_set({{2 * n, wide}});
      for (int r = 0; r <= reps && s == ZKQ_OK; ++r) {            // the first run warms up
        if (!cu(cudaEventRecord(e0, st))) break;
        try {
          s = mw_gemm_batched(pr.data(), count, words, words, words, 53 * words + 6, 1, ob.oz_ws, ob.oz_bytes,
                              ob.oz_meta, ob.oz_meta_bytes, st, ob.stage);
        } catch (...) { s = api_exception(ctx); }
        if (s != ZKQ_OK || !cu(cudaEventRecord(e1, st)) || !cu(cudaEventSynchronize(e1))) break;
        float ms = 0;
        if (!cu(cudaEventElapsedTime(&ms, e0, e1))) break;
        if (r > 0) t_w[wide] = std::min(t_w[wide], ms);
      }
    }
    cudaFree(A); cudaFree(B); cudaFree(C);
    A = B = C = nullptr;
    if (s != ZKQ_OK) break;
    const int w = t_w[1] <= t_w[0] ? 1 : 0;
    best[si] = w ? 256 : 128;
    table.push_back({2 * n, w});
  }
done:
  if (A) cudaFree(A);
  if (B) cudaFree(B);
  if (C) cudaFree(C);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  gemm_wide_table_set(s == ZKQ_OK ? table : saved);
  return s;
} catch (...) {
  return api_exception(ctx);
}
