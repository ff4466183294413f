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
