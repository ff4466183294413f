// Element-wise multi-word arithmetic entry point (diagnostics for the arithmetic of every refinement
// step): the same header code runs on the host (for CPU checks) and in a device kernel.
#include "common.cuh"
#include "mw.cuh"

namespace zkq {

template <int W>
__host__ __device__ void mw_apply(int op, int64_t i, const double* a, const double* b, double* out) {
  if (op <= 4) {
    mw<W> x = mw_load<W, W>(a, i), y = mw_load<W, W>(b, i), r;
    switch (op) {
      case 0: r = mw_add(x, y); break;
      case 1: r = mw_sub(x, y); break;
      case 2: r = mw_mul(x, y); break;
      case 3: r = mw_div(x, y); break;
      default: r = mw_sqrt(x); break;
    }
    mw_store(out, i, r);
  } else {
    cmw<W> x = c_load<W, W>(a, i), y = c_load<W, W>(b, i);
    c_store(out, i, op == 5 ? c_mul(x, y) : c_div(x, y));
  }
}

template <int W>
__global__ void mw_op_kernel(int op, int64_t count, const double* a, const double* b, double* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) mw_apply<W>(op, i, a, b, out);
}

}  // namespace zkq

using namespace zkq;

extern "C" zkq_status zkq_mw_op(int op, int words, int64_t count, const double* a, const double* b, double* out,
                                int on_device, void* stream) {
  if (op < 0 || op > 6 || count < 0 || (count > 0 && (!a || !b || !out))) return ZKQ_EINVAL;
  if (words != 1 && words != 2 && words != 4) return ZKQ_EINVAL;
  if (count == 0) return ZKQ_OK;
  if (!on_device) {
    for (int64_t i = 0; i < count; ++i) {
      if (words == 1) mw_apply<1>(op, i, a, b, out);
      else if (words == 2) mw_apply<2>(op, i, a, b, out);
      else mw_apply<4>(op, i, a, b, out);
    }
    return ZKQ_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned grid = (unsigned)((count + 255) / 256);
  if (words == 1) mw_op_kernel<1><<<grid, 256, 0, st>>>(op, count, a, b, out);
  else if (words == 2) mw_op_kernel<2><<<grid, 256, 0, st>>>(op, count, a, b, out);
  else mw_op_kernel<4><<<grid, 256, 0, st>>>(op, count, a, b, out);
  ZKQ_CUDA_TRY(cudaGetLastError());
  return ZKQ_OK;
}
