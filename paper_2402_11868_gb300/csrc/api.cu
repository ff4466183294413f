// C ABI of the zkq library: argument checking, batch scheduling metadata, workspace management and
// kernel launches.  Every compute step runs in this library's CUDA kernels.
#include <vector>
#include <algorithm>
#include <cstring>
#include <new>
#include "common.cuh"
#include "mw.cuh"

namespace zkq {

static thread_local int g_last_cuda = 0;
void set_last_cuda_error(cudaError_t e) { g_last_cuda = (int)e; }

struct JacobiBatch { const int32_t* n; const int64_t* a_off; const int64_t* w_off; const int32_t* order;
  const double* A; double* W; double* V; int32_t* info; double* ws; const int64_t* ws_off; double* red; int max_sweeps; };
zkq_status launch_jacobi(const JacobiBatch& jb, int a_words, int n_small, int n_large, int max_small_n,
                         int max_large_n, int cluster, cudaStream_t st);
size_t jacobi_smem_bytes(int n);

struct RqiBatch { const int32_t* n; const int64_t* a_off; const int64_t* w_off; const int32_t* pair_prob;
  const double* A; const double* W; const double* V; double* W_out; double* V_out; double* err; int32_t* info;
  double* ws; int64_t ws_stride; int64_t total_pairs; int max_iter; int* counter; };
zkq_status launch_rqi(const RqiBatch& rb, int W, int WA, int grid, cudaStream_t st);
size_t rqi_slot_doubles(int nmax, int W);

}  // namespace zkq

using namespace zkq;

struct zkq_ctx {
  int device = 0;
  int num_sms = 0;
  zkq_config cfg{};
  void* ws = nullptr;       // scratch workspace (grown on demand)
  size_t ws_bytes = 0;
  void* meta = nullptr;     // per-call metadata (offsets, orders)
  size_t meta_bytes = 0;
};

static zkq_status ensure(void** p, size_t* have, size_t need) {
  if (need <= *have) return ZKQ_OK;
  if (*p) { cudaFree(*p); *p = nullptr; *have = 0; }
  size_t want = std::max(need, (size_t)1 << 20);
  cudaError_t e = cudaMalloc(p, want);
  if (e != cudaSuccess) { set_last_cuda_error(e); *p = nullptr; return ZKQ_ENOMEM; }
  *have = want;
  return ZKQ_OK;
}

static size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

extern "C" {

const char* zkq_status_string(zkq_status s) {
  switch (s) {
    case ZKQ_OK: return "ZKQ_OK";
    case ZKQ_EINVAL: return "ZKQ_EINVAL: invalid argument";
    case ZKQ_ENOMEM: return "ZKQ_ENOMEM: device workspace allocation failed";
    case ZKQ_ENOCONV: return "ZKQ_ENOCONV: no convergence";
    case ZKQ_ETIMEOUT: return "ZKQ_ETIMEOUT: bounded device wait expired";
    case ZKQ_ECUDA: return "ZKQ_ECUDA: CUDA runtime error";
    case ZKQ_EADMIT: return "ZKQ_EADMIT: admission refused";
  }
  return "unknown zkq status";
}

int zkq_last_cuda_error(void) { return g_last_cuda; }

zkq_status zkq_ctx_create(zkq_ctx** ctx, const zkq_config* cfg) {
  if (!ctx) return ZKQ_EINVAL;
  *ctx = nullptr;
  zkq_ctx* c = new (std::nothrow) zkq_ctx();
  if (!c) return ZKQ_ENOMEM;
  if (cfg) c->cfg = *cfg;
  c->device = c->cfg.device;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) { set_last_cuda_error(e); delete c; return ZKQ_ECUDA; }
  if (c->cfg.max_sweeps <= 0) c->cfg.max_sweeps = 40;
  if (c->cfg.rqi_max_iter <= 0) c->cfg.rqi_max_iter = 5;
  if (c->cfg.oa_max_iter <= 0) c->cfg.oa_max_iter = 12;
  *ctx = c;
  return ZKQ_OK;
}

zkq_status zkq_ctx_destroy(zkq_ctx* ctx) {
  if (!ctx) return ZKQ_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->meta) cudaFree(ctx->meta);
  delete ctx;
  return ZKQ_OK;
}

static constexpr int kSmallMax = 80;

zkq_status zkq_eigh_batched(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                            const double* A, int a_words, double* W, double* V, int32_t* info, void* stream) {
  if (!ctx || batch < 0 || (batch > 0 && (!n || !a_off || !A || !W || !V || !info))) return ZKQ_EINVAL;
  if (a_words != 1 && a_words != 2 && a_words != 4) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> w_off(batch), ws_off(batch, 0);
  std::vector<int32_t> small, large;
  int64_t acc = 0; size_t ws_need = 0; int max_small = 0, max_large = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > 4096 || a_off[b] < 0) return ZKQ_EINVAL;
    w_off[b] = acc; acc += n[b];
    if (n[b] <= kSmallMax) { small.push_back(b); max_small = std::max(max_small, n[b]); }
    else { large.push_back(b); max_large = std::max(max_large, n[b]); }
  }
  std::sort(large.begin(), large.end(), [&](int a, int c) { return n[a] > n[c] || (n[a] == n[c] && a < c); });
  for (int b : large) { ws_off[b] = (int64_t)(ws_need / sizeof(double)); ws_need += align_up((size_t)n[b] * n[b] * 4 * sizeof(double)); }
  size_t red_bytes = align_up((size_t)64 * std::max<size_t>(1, large.size()) * sizeof(double));
  std::vector<int32_t> order(small); order.insert(order.end(), large.begin(), large.end());
  // metadata: n, a_off, w_off, order, ws_off
  size_t m_n = align_up(batch * 4), m_a = align_up(batch * 8), m_w = align_up(batch * 8), m_o = align_up(batch * 4), m_s = align_up(batch * 8);
  zkq_status s = ensure(&ctx->meta, &ctx->meta_bytes, m_n + m_a + m_w + m_o + m_s);
  if (s != ZKQ_OK) return s;
  s = ensure(&ctx->ws, &ctx->ws_bytes, ws_need + red_bytes);
  if (s != ZKQ_OK) return s;
  char* mb = (char*)ctx->meta;
  int32_t* d_n = (int32_t*)mb; int64_t* d_a = (int64_t*)(mb + m_n); int64_t* d_w = (int64_t*)(mb + m_n + m_a);
  int32_t* d_o = (int32_t*)(mb + m_n + m_a + m_w); int64_t* d_s = (int64_t*)(mb + m_n + m_a + m_w + m_o);
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_n, n, batch * 4, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_a, a_off, batch * 8, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_w, w_off.data(), batch * 8, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_o, order.data(), batch * 4, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_s, ws_off.data(), batch * 8, cudaMemcpyHostToDevice, st));
  int cluster = ctx->cfg.jacobi_cluster;
  if (cluster <= 0) cluster = max_large <= 128 ? 2 : (max_large <= 256 ? 4 : 8);
  if (cluster > 16) cluster = 16;
  JacobiBatch jb{d_n, d_a, d_w, d_o, A, W, V, info, (double*)ctx->ws, d_s,
                 (double*)((char*)ctx->ws + ws_need), ctx->cfg.max_sweeps};
  return launch_jacobi(jb, a_words, (int)small.size(), (int)large.size(), max_small, max_large, cluster, st);
}

zkq_status zkq_rqi_refine(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                          const double* A, int a_words, const double* W, const double* V,
                          int target_words, int method, double* W_out, double* V_out, double* err_est,
                          int32_t* info, void* stream) {
  if (!ctx || batch < 0 || (batch > 0 && (!n || !a_off || !A || !W || !V || !W_out || !V_out || !err_est || !info)))
    return ZKQ_EINVAL;
  if ((a_words != 1 && a_words != 2 && a_words != 4) || (target_words != 2 && target_words != 4)) return ZKQ_EINVAL;
  if (method != ZKQ_PLAIN_RQI && method != ZKQ_OA_OZAKI) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  if (method == ZKQ_OA_OZAKI) return ZKQ_EINVAL;   // provided by the refinement module when built
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> w_off(batch);
  int64_t total = 0; int nmax = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > 4096 || a_off[b] < 0) return ZKQ_EINVAL;
    w_off[b] = total; total += n[b]; nmax = std::max(nmax, n[b]);
  }
  std::vector<int32_t> pair_prob(total);
  for (int b = 0; b < batch; ++b) for (int i = 0; i < n[b]; ++i) pair_prob[w_off[b] + i] = b;
  size_t m_n = align_up(batch * 4), m_a = align_up(batch * 8), m_w = align_up(batch * 8), m_p = align_up(total * 4), m_c = 256;
  zkq_status s = ensure(&ctx->meta, &ctx->meta_bytes, m_n + m_a + m_w + m_p + m_c);
  if (s != ZKQ_OK) return s;
  int grid = (int)std::min<int64_t>(total, (int64_t)ctx->num_sms);
  size_t slot = rqi_slot_doubles(nmax, target_words);
  s = ensure(&ctx->ws, &ctx->ws_bytes, slot * sizeof(double) * grid);
  if (s != ZKQ_OK) return s;
  char* mb = (char*)ctx->meta;
  int32_t* d_n = (int32_t*)mb; int64_t* d_a = (int64_t*)(mb + m_n); int64_t* d_w = (int64_t*)(mb + m_n + m_a);
  int32_t* d_p = (int32_t*)(mb + m_n + m_a + m_w); int* d_c = (int*)(mb + m_n + m_a + m_w + m_p);
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_n, n, batch * 4, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_a, a_off, batch * 8, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_w, w_off.data(), batch * 8, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemcpyAsync(d_p, pair_prob.data(), total * 4, cudaMemcpyHostToDevice, st));
  ZKQ_CUDA_TRY(cudaMemsetAsync(d_c, 0, sizeof(int), st));
  ZKQ_CUDA_TRY(cudaMemsetAsync(info, 0, batch * sizeof(int32_t), st));
  RqiBatch rb{d_n, d_a, d_w, d_p, A, W, V, W_out, V_out, err_est, info, (double*)ctx->ws, (int64_t)slot, total,
              ctx->cfg.rqi_max_iter, d_c};
  return launch_rqi(rb, target_words, a_words, grid, st);
}

}  // extern "C"
