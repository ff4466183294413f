// Shared definitions for the zkq CUDA library (status codes, device helpers, launch checks).
#pragma once
#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>
#include "../../include/zkq.h"

namespace zkq {

#define ZKQ_CUDA_TRY(expr)                                            \
  do {                                                                \
    cudaError_t _e = (expr);                                          \
    if (_e != cudaSuccess) { ::zkq::set_last_cuda_error(_e); return ZKQ_ECUDA; } \
  } while (0)

void set_last_cuda_error(cudaError_t e);

// Raise a kernel's dynamic shared-memory limit to the device maximum, once per kernel and device.  The
// limit is process-wide state of the kernel, so setting it to the size of each launch would race between
// host threads that launch the same kernel with different sizes (the smaller setting would make the
// larger launch fail); a fixed maximum does not race.
cudaError_t raise_smem_limit(const void* kernel, int slot);
template <auto K>
cudaError_t smem_limit_max() {
  // one slot per kernel instantiation: its address identifies it
  static const int slot = 0;
  return raise_smem_limit(reinterpret_cast<const void*>(K), (int)(reinterpret_cast<uintptr_t>(&slot) & 0x7fffffff));
}

// complex FP64 element helpers (layout: re, im adjacent)
struct c64 { double re, im; };
__device__ __forceinline__ c64 cmul(c64 a, c64 b) { return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)}; }
__device__ __forceinline__ c64 cconj(c64 a) { return {a.re, -a.im}; }

// round-robin (circle) ordering: round r in [0, m-2] of m (even) players; pair k in [0, m/2)
__device__ __forceinline__ void rr_pair(int m, int r, int k, int& p, int& q) {
  int a, b;
  if (k == 0) { a = m - 1; b = r; }
  else { a = (r + k) % (m - 1); b = (r - k + (m - 1)) % (m - 1); }
  p = a < b ? a : b; q = a < b ? b : a;
}

}  // namespace zkq
