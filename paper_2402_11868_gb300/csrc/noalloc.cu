// FP64 batched eigensolve for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc (or any allocating routine): code running while a CUDA graph is
// being captured elsewhere in the process, hosts that hand the library a fixed memory budget, or
// real-time loops where an allocation may block on a device-wide synchronisation.  This entry point runs
// the same Jacobi kernels as zkq_eigh_batched, but its scratch (batch metadata and the global-memory
// copies of A and V for orders above 80) lives in one file-scope device array of fixed size that every
// GPU loading the library keeps until the process exits.  The caller still owns all inputs and outputs.
// The batch layout is the allocating path's (eigh_layout), without the cooperative-grid class: every
// problem above order 80 runs on a thread-block cluster of the built-in width (2 / 4 / 8 CTAs for largest
// orders <= 128 / <= 256 / above).
// The array's device address is looked up once per device and kept for the life of the process; after a
// cudaDeviceReset the module may be loaded at another address, so the entry point must not be used after a
// device reset.
#include <mutex>
#include <vector>
#include <algorithm>
#include "common.cuh"
#include "internal.cuh"
#include "prof.cuh"

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
  cudaStream_t st = (cudaStream_t)stream;
  // The metadata goes up from pageable host memory that is freed when this call returns.  A captured copy
  // would record that host address for every replay, so the call refuses to run inside a stream capture.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  ZKQ_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) return ZKQ_EINVAL;
  // The allocating entry point's layout rules (size classes, order, per-problem A/V copies, reduction
  // slots), with no cooperative grid (num_sms 0) and the built-in cluster width for the largest order.
  EighLayout L;
  zkq_status s = eigh_layout(batch, n, a_off, a_words, 0, 0, &L, nullptr);
  if (s != ZKQ_OK) return s;
  const size_t meta_b = al256(L.meta_bytes()), ws_b = L.ws_bytes();
  if (meta_b + ws_b > (size_t)ZKQ_NOALLOC_SCRATCH_BYTES) return ZKQ_ETOOBIG;
  int dev = 0;
  ZKQ_CUDA_TRY(cudaGetDevice(&dev));
  void* base_v = nullptr;
  s = noalloc_scratch(dev, &base_v);
  if (s != ZKQ_OK) return s;
  char* meta = (char*)base_v;
  char* ws = meta + meta_b;
  std::vector<char> img;
  eigh_meta_image(L, &img);
  ZKQ_CUDA_TRY(cudaMemcpyAsync(meta, img.data(), img.size(), cudaMemcpyHostToDevice, st));
  // every reduction slot is written before it is read; clear them (and the unused barrier words) anyway, so
  // that no value of an earlier call can ever be observed
  ZKQ_CUDA_TRY(cudaMemsetAsync(ws + L.ws_need, 0, ws_b - L.ws_need, st));
  return eigh_launch(L, meta, ws, A, a_words, W, V, info, 40, PC_JACOBI, st);
} catch (...) {
  return api_exception(nullptr);
}
