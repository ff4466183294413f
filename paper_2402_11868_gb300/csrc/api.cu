// C ABI of the zkq library: argument checking, batch scheduling metadata, workspace management and
// kernel launches.  Every compute step runs in this library's CUDA kernels.
#include <vector>
#include <algorithm>
#include <cstring>
#include <new>
#include "common.cuh"
#include "mw.cuh"
#include "prof.cuh"
#include "internal.cuh"

namespace zkq {

Profiler& profiler() { static Profiler p; return p; }
static unsigned long long* g_prof_ctr = nullptr;   // device counters, PC_COUNT entries
unsigned long long* prof_device_counters() { return profiler().on ? g_prof_ctr : nullptr; }

static thread_local int g_last_cuda = 0;
void set_last_cuda_error(cudaError_t e) { g_last_cuda = (int)e; }

}  // namespace zkq
#include "ozaki.cuh"

using namespace zkq;

struct zkq_ctx {
  int device = 0;
  int num_sms = 0;
  zkq_config cfg{};
  void* ws = nullptr;       // scratch workspace (grown on demand)
  size_t ws_bytes = 0;
  void* meta = nullptr;     // per-call metadata (offsets, orders)
  size_t meta_bytes = 0;
  void* oa_ws = nullptr;    // refinement state (X, P, S, R, E, lambda, clusters)
  size_t oa_bytes = 0;
  void* oz_ws = nullptr;    // split-product scratch (digit slices, level sums)
  size_t oz_bytes = 0;
  void* oz_meta = nullptr;
  size_t oz_meta_bytes = 0;
  void* mps_ws = nullptr;   // gate-update scratch (theta, rho, split-back)
  size_t mps_bytes = 0;
  HostStage stage;          // pinned staging of metadata uploads and statistics read-back
};

namespace zkq {
OaBuffers ctx_oa_buffers(void* vctx) {
  zkq_ctx* c = (zkq_ctx*)vctx;
  return OaBuffers{&c->oa_ws, &c->oa_bytes, &c->oz_ws, &c->oz_bytes, &c->oz_meta, &c->oz_meta_bytes, &c->stage};
}
HostStage* ctx_stage(void* vctx) { return &((zkq_ctx*)vctx)->stage; }
int ctx_oa_max_iter(void* vctx) { return ((zkq_ctx*)vctx)->cfg.oa_max_iter; }
void** ctx_mps_ws(void* vctx, size_t** bytes) { zkq_ctx* c = (zkq_ctx*)vctx; *bytes = &c->mps_bytes; return &c->mps_ws; }
}  // namespace zkq

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
    case ZKQ_ETOOBIG: return "ZKQ_ETOOBIG: request exceeds the fixed scratch of the no-allocation entry point";
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
  if (c->cfg.oa_max_iter <= 0) c->cfg.oa_max_iter = 40;
  *ctx = c;
  return ZKQ_OK;
}

zkq_status zkq_ctx_destroy(zkq_ctx* ctx) {
  if (!ctx) return ZKQ_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (void* p : {ctx->ws, ctx->meta, ctx->oa_ws, ctx->oz_ws, ctx->oz_meta, ctx->mps_ws}) if (p) cudaFree(p);
  delete ctx;
  return ZKQ_OK;
}

static constexpr int kSmallMax = 80;

}  // extern "C"

namespace zkq {
zkq_status eigh_internal(void* vctx, int batch, const int32_t* n, const int64_t* a_off, const double* A, int a_words,
                         double* W, double* V, int32_t* info, cudaStream_t st, int prof_class) {
  zkq_ctx* ctx = (zkq_ctx*)vctx;
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
  // few large problems: one at a time on a cooperative grid instead of a cluster each (a cluster of at
  // most 16 CTAs would leave most SMs idle)
  int cluster = ctx->cfg.jacobi_cluster;
  if (cluster <= 0) cluster = max_large <= 128 ? 2 : (max_large <= 256 ? 4 : 8);
  if (cluster > 16) cluster = 16;
  int grid_blocks = 0;
  if (!large.empty() && (int)large.size() * cluster * 2 <= ctx->num_sms) {
    const int per_sm = jacobi_grid_max_blocks(max_large, a_words);
    grid_blocks = std::min(std::min(ctx->num_sms, std::max(8, max_large / 4)), per_sm * ctx->num_sms);
  }
  size_t red_bytes = align_up((size_t)64 * std::max<size_t>(1, large.size()) * sizeof(double));
  red_bytes = std::max(red_bytes, align_up((size_t)(2 * grid_blocks + 64) * sizeof(double)));
  const size_t gb_bytes = align_up(sizeof(GridBar));
  std::vector<int32_t> order(small); order.insert(order.end(), large.begin(), large.end());
  // metadata: n, a_off, w_off, order, ws_off
  size_t m_n = align_up(batch * 4), m_a = align_up(batch * 8), m_w = align_up(batch * 8), m_o = align_up(batch * 4), m_s = align_up(batch * 8);
  zkq_status s = ensure(&ctx->meta, &ctx->meta_bytes, m_n + m_a + m_w + m_o + m_s);
  if (s != ZKQ_OK) return s;
  s = ensure(&ctx->ws, &ctx->ws_bytes, ws_need + red_bytes + gb_bytes);
  if (s != ZKQ_OK) return s;
  char* mb = (char*)ctx->meta;
  int32_t* d_n = (int32_t*)mb; int64_t* d_a = (int64_t*)(mb + m_n); int64_t* d_w = (int64_t*)(mb + m_n + m_a);
  int32_t* d_o = (int32_t*)(mb + m_n + m_a + m_w); int64_t* d_s = (int64_t*)(mb + m_n + m_a + m_w + m_o);
  HostStage& hs = ctx->stage;
  hs.add(d_n, n, batch * 4);
  hs.add(d_a, a_off, batch * 8);
  hs.add(d_w, w_off.data(), batch * 8);
  hs.add(d_o, order.data(), batch * 4);
  hs.add(d_s, ws_off.data(), batch * 8);
  ZKQ_CUDA_TRY(hs.flush(st));
  unsigned long long* ctr = prof_device_counters();
  JacobiBatch jb{d_n, d_a, d_w, d_o, A, W, V, info, (double*)ctx->ws, d_s,
                 (double*)((char*)ctx->ws + ws_need), ctx->cfg.max_sweeps, ctr ? ctr + prof_class : nullptr, prof_class};
  GridBar* gb = (GridBar*)((char*)ctx->ws + ws_need + red_bytes);
  return launch_jacobi(jb, a_words, (int)small.size(), (int)large.size(), max_small, max_large, cluster, grid_blocks,
                       gb, st);
}
zkq_status rqi_refine_internal(void* vctx, int batch, const int32_t* n, const int64_t* a_off, const double* A,
                               int a_words, const double* W, const double* V, int target_words, double* W_out,
                               double* V_out, double* err_est, int32_t* info, cudaStream_t st) {
  zkq_ctx* ctx = (zkq_ctx*)vctx;
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
  HostStage& hs = ctx->stage;
  hs.add(d_n, n, batch * 4);
  hs.add(d_a, a_off, batch * 8);
  hs.add(d_w, w_off.data(), batch * 8);
  hs.add(d_p, pair_prob.data(), total * 4);
  ZKQ_CUDA_TRY(hs.flush(st));
  ZKQ_CUDA_TRY(cudaMemsetAsync(d_c, 0, sizeof(int), st));
  ZKQ_CUDA_TRY(cudaMemsetAsync(info, 0, batch * sizeof(int32_t), st));
  RqiBatch rb{d_n, d_a, d_w, d_p, A, W, V, W_out, V_out, err_est, info, (double*)ctx->ws, (int64_t)slot, total,
              ctx->cfg.rqi_max_iter, d_c};
  return launch_rqi(rb, target_words, a_words, grid, st);
}
}  // namespace zkq

extern "C" {

zkq_status zkq_eigh_batched(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                            const double* A, int a_words, double* W, double* V, int32_t* info, void* stream) {
  if (!ctx || batch < 0 || (batch > 0 && (!n || !a_off || !A || !W || !V || !info))) return ZKQ_EINVAL;
  if (a_words != 1 && a_words != 2 && a_words != 4) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  for (int b = 0; b < batch; ++b) if (n[b] < 1 || n[b] > 4096 || a_off[b] < 0) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));
  return eigh_internal(ctx, batch, n, a_off, A, a_words, W, V, info, (cudaStream_t)stream);
}

zkq_status zkq_rqi_refine(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                          const double* A, int a_words, const double* W, const double* V,
                          int target_words, int method, double* W_out, double* V_out, double* err_est,
                          int32_t* info, void* stream) {
  if (!ctx || batch < 0 || (batch > 0 && (!n || !a_off || !A || !W || !V || !W_out || !V_out || !err_est || !info)))
    return ZKQ_EINVAL;
  if ((a_words != 1 && a_words != 2 && a_words != 4) || (target_words != 2 && target_words != 4)) return ZKQ_EINVAL;
  if (method != ZKQ_PLAIN_RQI && method != ZKQ_OA_OZAKI && method != ZKQ_OA_FP64) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (method != ZKQ_PLAIN_RQI) {
    for (int b = 0; b < batch; ++b) if (n[b] < 1 || n[b] > 2048 || a_off[b] < 0) return ZKQ_EINVAL;
    OaBuffers ob{&ctx->oa_ws, &ctx->oa_bytes, &ctx->oz_ws, &ctx->oz_bytes, &ctx->oz_meta, &ctx->oz_meta_bytes, &ctx->stage};
    return oa_refine(ctx, ob, batch, n, a_off, A, a_words, V, target_words, W_out, V_out, err_est, info,
                     ctx->cfg.oa_max_iter, method == ZKQ_OA_OZAKI ? 1 : 0, st);
  }
  return rqi_refine_internal(ctx, batch, n, a_off, A, a_words, W, V, target_words, W_out, V_out, err_est, info, st);
}

zkq_status zkq_mw_gemm(zkq_ctx* ctx, int count, const int32_t* m, const int32_t* n, const int32_t* k,
                       const int32_t* opA, const double* A, const int64_t* a_off, int wa, const double* B,
                       const int64_t* b_off, int wb, double* C, const int64_t* c_off, int wc, int p_bits, int method,
                       void* stream) {
  if (!ctx || count < 0 || (count > 0 && (!m || !n || !k || !opA || !A || !a_off || !B || !b_off || !C || !c_off)))
    return ZKQ_EINVAL;
  if (method != 0 && method != 1 && method != 2) return ZKQ_EINVAL;
  if (p_bits < 1 || p_bits > 53 * 4 + 40) return ZKQ_EINVAL;
  if (count == 0) return ZKQ_OK;
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));
  std::vector<MwProd> pr(count);
  for (int i = 0; i < count; ++i) {
    if (m[i] < 1 || n[i] < 1 || k[i] < 1 || k[i] > 2048 || (opA[i] != 0 && opA[i] != 1) || a_off[i] < 0 || b_off[i] < 0 || c_off[i] < 0)
      return ZKQ_EINVAL;
    pr[i] = {m[i], n[i], k[i], opA[i], A + a_off[i] * 2 * wa, B + b_off[i] * 2 * wb, C + c_off[i] * 2 * wc, nullptr, 1.0, 0};
  }
  zkq_status s = mw_gemm_batched(pr.data(), count, wa, wb, wc, p_bits, method, &ctx->oz_ws, &ctx->oz_bytes,
                                 &ctx->oz_meta, &ctx->oz_meta_bytes, (cudaStream_t)stream, &ctx->stage);
  return s;
}

zkq_status zkq_set_gemm_kernel(int which) {
  if (which != 0 && which != 1) return ZKQ_EINVAL;
  gemm_kernel_set(which);
  return ZKQ_OK;
}

int zkq_get_gemm_kernel(void) { return gemm_kernel_get(); }

zkq_status zkq_check_device_waits(void) { return gemm_kernel_error() ? ZKQ_ETIMEOUT : ZKQ_OK; }

static const char* kProfNames[PC_COUNT] = {"jacobi", "rqi", "ozaki_scale", "ozaki_slice", "ozaki_gemm",
                                           "ozaki_combine", "oa_elementwise", "mps", "other", "jacobi_cluster"};

int zkq_profile_classes(void) { return PC_COUNT; }

const char* zkq_profile_class_name(int cls) { return (cls >= 0 && cls < PC_COUNT) ? kProfNames[cls] : "invalid"; }

zkq_status zkq_profile_enable(int on) {
  Profiler& p = profiler();
  std::lock_guard<std::mutex> g(p.mu);
  if (on && !g_prof_ctr) {
    cudaError_t e = cudaMalloc(&g_prof_ctr, sizeof(unsigned long long) * PC_COUNT);
    if (e != cudaSuccess) { set_last_cuda_error(e); g_prof_ctr = nullptr; return ZKQ_ENOMEM; }
    cudaMemset(g_prof_ctr, 0, sizeof(unsigned long long) * PC_COUNT);
  }
  p.on = on != 0;
  return ZKQ_OK;
}

zkq_status zkq_profile_read(double* ms, int64_t* launches, double* work, int nclasses) {
  if (!ms || !launches || !work || nclasses < 1) return ZKQ_EINVAL;
  Profiler& p = profiler();
  std::lock_guard<std::mutex> g(p.mu);
  for (int i = 0; i < nclasses; ++i) { ms[i] = 0.0; launches[i] = 0; work[i] = 0.0; }
  for (auto& r : p.recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ECUDA; }
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    if (r.cls < nclasses) { ms[r.cls] += t; launches[r.cls] += 1; work[r.cls] += r.work; }
    p.pool.push_back(r.a); p.pool.push_back(r.b);
  }
  p.recs.clear();
  if (g_prof_ctr) {                              // device-counted work (all recorded launches are complete)
    unsigned long long h[PC_COUNT];
    cudaError_t e = cudaMemcpy(h, g_prof_ctr, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ECUDA; }
    for (int i = 0; i < PC_COUNT && i < nclasses; ++i) work[i] += (double)h[i];
    cudaMemset(g_prof_ctr, 0, sizeof(h));
  }
  return ZKQ_OK;
}

}  // extern "C"
