// Block-wide reductions of multi-word values (tree in shared memory).
#pragma once
#include "mw.cuh"

namespace zkq {

// sum over all threads of the block; every thread receives the total.  buf: blockDim.x entries.
template <int W>
__device__ cmw<W> block_sum_c(cmw<W> v, cmw<W>* buf) {
  const int tid = threadIdx.x, nth = blockDim.x;
  buf[tid] = v;
  __syncthreads();
  for (int s = 1; s < nth; s <<= 1) {             // pairwise tree: same order on every call
    if ((tid % (2 * s)) == 0 && tid + s < nth) buf[tid] = c_add(buf[tid], buf[tid + s]);
    __syncthreads();
  }
  cmw<W> r = buf[0];
  __syncthreads();
  return r;
}

template <int W>
__device__ mw<W> block_sum_r(mw<W> v, mw<W>* buf) {
  const int tid = threadIdx.x, nth = blockDim.x;
  buf[tid] = v;
  __syncthreads();
  for (int s = 1; s < nth; s <<= 1) {
    if ((tid % (2 * s)) == 0 && tid + s < nth) buf[tid] = mw_add(buf[tid], buf[tid + s]);
    __syncthreads();
  }
  mw<W> r = buf[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max_d(double v, double* buf) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((tid & 31) == 0) buf[tid >> 5] = v;
  __syncthreads();
  double r = buf[0];
  for (int w = 1; w < (nth + 31) / 32; ++w) r = fmax(r, buf[w]);
  __syncthreads();
  return r;
}

}  // namespace zkq
