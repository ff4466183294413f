// FP64 batched eigensolve for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc (or any allocating routine): code running while a CUDA graph is
// being captured elsewhere in the process, hosts that hand the library a fixed memory budget, or
// real-time loops where an allocation may block on a device-wide synchronisation.  This entry point runs
// the same Jacobi kernels as zkq_eigh_batched, but its scratch (batch metadata and the global-memory
// copies of A and V for orders above 80) lives in one file-scope device array of fixed size that every
// GPU loading the library keeps until the process exits.  The caller still owns all inputs and outputs.
#include <mutex>
#include <vector>
#include <algorithm>
#include "common.cuh"
#include "internal.cuh"

using namespace zkq;

// The scratch.  Host code must not pass this name to a kernel (on the host it is only a stand-in for the
// symbol); the device address comes from cudaGetSymbolAddress, taken once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ZKQ_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256] = {};

static zkq_status noalloc_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (dev < 0 || dev >= 256) return ZKQ_EINVAL;
  if (!g_noalloc_addr[dev]) {                 // first call on this device (the device is current)
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) { set_last_cuda_error(e); return ZKQ_ECUDA; }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return ZKQ_OK;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" zkq_status zkq_eigh_batched_noalloc(int batch, const int32_t* n, const int64_t* a_off, const double* A,
                                               int a_words, double* W, double* V, int32_t* info, void* stream) try {
  if (batch < 0 || (batch > 0 && (!n || !a_off || !A || !W || !V || !info))) return ZKQ_EINVAL;
  if (a_words != 1 && a_words != 2 && a_words != 4) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  constexpr int kSmallMax = 80;               // orders held in shared memory (no scratch needed)
  std::vector<int64_t> w_off(batch), ws_off(batch, 0);
  std::vector<int32_t> small, large;
  int64_t acc = 0; int max_small = 0, max_large = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > 4096 || a_off[b] < 0) return ZKQ_EINVAL;
    w_off[b] = acc; acc += n[b];
    if (n[b] <= kSmallMax) { small.push_back(b); max_small = std::max(max_small, n[b]); }
    else { large.push_back(b); max_large = std::max(max_large, n[b]); }
  }
  std::sort(large.begin(), large.end(), [&](int a, int c) { return n[a] > n[c] || (n[a] == n[c] && a < c); });
  std::vector<int32_t> order(small); order.insert(order.end(), large.begin(), large.end());
  // layout inside the fixed scratch: metadata, per-problem A/V copies, reduction slots
  size_t off = 0;
  const size_t o_n = off; off += al256((size_t)batch * 4);
  const size_t o_a = off; off += al256((size_t)batch * 8);
  const size_t o_w = off; off += al256((size_t)batch * 8);
  const size_t o_o = off; off += al256((size_t)batch * 4);
  const size_t o_s = off; off += al256((size_t)batch * 8);
  const size_t o_ws = off;
  size_t ws_bytes = 0;
  for (int b : large) { ws_off[b] = (int64_t)(ws_bytes / sizeof(double)); ws_bytes += al256((size_t)n[b] * n[b] * 4 * sizeof(double)); }
  off += ws_bytes;
  const size_t o_red = off; off += al256((size_t)64 * std::max<size_t>(1, large.size()) * sizeof(double));
  if (off > (size_t)ZKQ_NOALLOC_SCRATCH_BYTES) return ZKQ_ETOOBIG;
  int dev = 0;
  ZKQ_CUDA_TRY(cudaGetDevice(&dev));
  void* base_v = nullptr;
  zkq_status s = noalloc_scratch(dev, &base_v);
  if (s != ZKQ_OK) return s;
  char* base = (char*)base_v;
  cudaStream_t st = (cudaStream_t)stream;
  ZKQ_CUDA_TRY(cudaMemcpyAsync(base + o_n, n, (size_t)batch * 4, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(base + o_a, a_off, (size_t)batch * 8, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(base + o_w, w_off.data(), (size_t)batch * 8, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(base + o_o, order.data(), (size_t)batch * 4, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(base + o_s, ws_off.data(), (size_t)batch * 8, cudaMemcpyHostToDevice, st));
  // every reduction slot is written before it is read; clear them anyway so no value of an earlier call
  // can ever be observed
  ZKQ_CUDA_TRY(cudaMemsetAsync(base + o_red, 0, off - o_red, st));
  int cluster = max_large <= 128 ? 2 : (max_large <= 256 ? 4 : 8);
  JacobiBatch jb{(const int32_t*)(base + o_n), (const int64_t*)(base + o_a), (const int64_t*)(base + o_w),
                 (const int32_t*)(base + o_o), A, W, V, info, (double*)(base + o_ws), (const int64_t*)(base + o_s),
                 (double*)(base + o_red), 40, nullptr, 0};
  return launch_jacobi(jb, a_words, (int)small.size(), (int)large.size(), max_small, max_large, cluster, 0, nullptr, nullptr, 0, st);
} catch (...) {
  return api_exception(nullptr);
}
