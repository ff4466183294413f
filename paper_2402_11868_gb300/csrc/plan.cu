// Fixed-shape batch plans: layout and metadata upload once, then launches only (graph-capturable), and
// a captured CUDA graph per buffer set (see zkq.h).
#include <cstring>
#include <new>
#include <vector>
#include "internal.cuh"
#include "prof.cuh"

using namespace zkq;

struct zkq_plan {
  void* ctx = nullptr;
  int device = 0, a_words = 1, target = 0, max_sweeps = 40, rqi_max_iter = 5;
  EighLayout el;
  RqiLayout rl;
  void* meta = nullptr;       // [eigh metadata | rqi metadata]
  void* ws = nullptr;         // shared by the two stages (they run one after the other on the stream)
  size_t eigh_meta = 0;
  // captured graph and the buffers it was captured for
  cudaGraphExec_t exec = nullptr;
  const void* key[8] = {};
};

namespace {
zkq_status plan_launch(zkq_plan* p, const double* A, double* W, double* V, int32_t* info, double* W_out, double* V_out,
                       double* err, int32_t* rinfo, cudaStream_t st) {
  zkq_status s = eigh_launch(p->el, p->meta, p->ws, A, p->a_words, W, V, info, p->max_sweeps, PC_JACOBI, st);
  if (s != ZKQ_OK || p->target == 0) return s;
  return rqi_launch(p->rl, (char*)p->meta + p->eigh_meta, p->ws, A, p->a_words, W, V, p->target, W_out, V_out, err,
                    rinfo, p->rqi_max_iter, st);
}
bool args_ok(const zkq_plan* p, const double* A, double* W, double* V, int32_t* info, double* W_out, double* V_out,
             double* err, int32_t* rinfo) {
  if (!p || !A || !W || !V || !info) return false;
  return p->target == 0 || (W_out && V_out && err && rinfo);
}
// layout, device buffers and the one-time metadata upload of a plan; on failure the caller frees p
zkq_status plan_build(zkq_plan* p, zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off) {
  ZKQ_CUDA_TRY(cudaSetDevice(p->device));
  zkq_status s = eigh_layout(batch, n, a_off, p->a_words, ctx_config(ctx).jacobi_cluster, ctx_num_sms(ctx), &p->el,
                             ctx_jacobi_tune(ctx));
  if (s != ZKQ_OK) return s;
  if (p->target) {
    s = rqi_layout(batch, n, a_off, p->target, ctx_num_sms(ctx), &p->rl);
    if (s != ZKQ_OK) return s;
  }
  p->eigh_meta = p->el.meta_bytes();
  const size_t meta = p->eigh_meta + (p->target ? p->rl.meta_bytes() : 0);
  const size_t ws = std::max(p->el.ws_bytes(), p->target ? p->rl.ws_bytes() : (size_t)0);
  cudaError_t e = cudaMalloc(&p->meta, meta);
  if (e == cudaSuccess) e = cudaMalloc(&p->ws, std::max<size_t>(ws, 256));
  if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ENOMEM; }
  HostStage hs;                                 // one-time upload, then wait for it
  s = eigh_upload(p->el, p->meta, hs, 0);
  if (s == ZKQ_OK && p->target) s = rqi_upload(p->rl, (char*)p->meta + p->eigh_meta, hs, 0);
  if (s != ZKQ_OK) return s;
  ZKQ_CUDA_TRY(cudaDeviceSynchronize());
  return ZKQ_OK;
}
}  // namespace

extern "C" {

zkq_status zkq_plan_create(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off, int a_words,
                           int target_words, zkq_plan** out) {
  if (!out) return ZKQ_EINVAL;
  *out = nullptr;
  if (!ctx || batch < 1 || !n || !a_off) return ZKQ_EINVAL;
  if (a_words != 1 && a_words != 2 && a_words != 4) return ZKQ_EINVAL;
  if (target_words != 0 && target_words != 2 && target_words != 4) return ZKQ_EINVAL;
  zkq_plan* p = new (std::nothrow) zkq_plan();
  if (!p) return ZKQ_ENOMEM;
  p->ctx = ctx; p->device = ctx_device(ctx); p->a_words = a_words; p->target = target_words;
  p->max_sweeps = ctx_config(ctx).max_sweeps; p->rqi_max_iter = ctx_config(ctx).rqi_max_iter;
  zkq_status s;
  try { s = plan_build(p, ctx, batch, n, a_off); } catch (...) { s = api_exception(nullptr); }
  if (s != ZKQ_OK) { zkq_plan_destroy(p); return s; }
  *out = p;
  return ZKQ_OK;
}

zkq_status zkq_plan_execute(zkq_plan* p, const double* A, double* W, double* V, int32_t* info, double* W_out,
                            double* V_out, double* err_est, int32_t* rinfo, void* stream) {
  if (!args_ok(p, A, W, V, info, W_out, V_out, err_est, rinfo)) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(p->device));
  return plan_launch(p, A, W, V, info, W_out, V_out, err_est, rinfo, (cudaStream_t)stream);
}

zkq_status zkq_plan_execute_graph(zkq_plan* p, const double* A, double* W, double* V, int32_t* info, double* W_out,
                                  double* V_out, double* err_est, int32_t* rinfo, void* stream) {
  if (!args_ok(p, A, W, V, info, W_out, V_out, err_est, rinfo)) return ZKQ_EINVAL;
  if (!stream || profiler().on) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)stream;
  const void* key[8] = {A, W, V, info, W_out, V_out, err_est, rinfo};
  if (!p->exec || std::memcmp(key, p->key, sizeof(key)) != 0) {
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    ZKQ_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    zkq_status s = plan_launch(p, A, W, V, info, W_out, V_out, err_est, rinfo, st);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != ZKQ_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ECUDA; }
    e = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { set_last_cuda_error(e); p->exec = nullptr; return ZKQ_ECUDA; }
    std::memcpy(p->key, key, sizeof(key));
  }
  ZKQ_CUDA_TRY(cudaGraphLaunch(p->exec, st));
  return ZKQ_OK;
}

zkq_status zkq_plan_destroy(zkq_plan* p) {
  if (!p) return ZKQ_OK;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->meta) cudaFree(p->meta);
  if (p->ws) cudaFree(p->ws);
  delete p;
  return ZKQ_OK;
}

}  // extern "C"
