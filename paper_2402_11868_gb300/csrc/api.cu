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
  JacobiTune jacobi_tune;   // cluster widths measured by zkq_autotune_jacobi (empty: built-in choice)
};

namespace zkq {
OaBuffers ctx_oa_buffers(void* vctx) {
  zkq_ctx* c = (zkq_ctx*)vctx;
  return OaBuffers{&c->oa_ws, &c->oa_bytes, &c->oz_ws, &c->oz_bytes, &c->oz_meta, &c->oz_meta_bytes, &c->stage};
}
HostStage* ctx_stage(void* vctx) { return &((zkq_ctx*)vctx)->stage; }
int ctx_num_sms(void* vctx) { return ((zkq_ctx*)vctx)->num_sms; }
JacobiTune* ctx_jacobi_tune(void* vctx) { return &((zkq_ctx*)vctx)->jacobi_tune; }
int ctx_device(void* vctx) { return ((zkq_ctx*)vctx)->device; }
const zkq_config& ctx_config(void* vctx) { return ((zkq_ctx*)vctx)->cfg; }
zkq_config& ctx_config_mut(void* vctx) { return ((zkq_ctx*)vctx)->cfg; }
int ctx_oa_max_iter(void* vctx) { return ((zkq_ctx*)vctx)->cfg.oa_max_iter; }
void** ctx_mps_ws(void* vctx, size_t** bytes) { zkq_ctx* c = (zkq_ctx*)vctx; *bytes = &c->mps_bytes; return &c->mps_ws; }
void ctx_fp64_bufs(void* vctx, void*** ws, size_t** ws_bytes, void*** meta, size_t** meta_bytes) {
  zkq_ctx* c = (zkq_ctx*)vctx;
  *ws = &c->ws; *ws_bytes = &c->ws_bytes; *meta = &c->meta; *meta_bytes = &c->meta_bytes;
}
zkq_status api_exception(void* vctx) noexcept {
  if (vctx) ((zkq_ctx*)vctx)->stage.discard();
  return ZKQ_ENOMEM;
}
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


}  // extern "C"

namespace zkq {
zkq_status eigh_internal(void* vctx, int batch, const int32_t* n, const int64_t* a_off, const double* A, int a_words,
                         double* W, double* V, int32_t* info, cudaStream_t st, int prof_class) {
  zkq_ctx* ctx = (zkq_ctx*)vctx;
  EighLayout L;
  zkq_status s = eigh_layout(batch, n, a_off, a_words, ctx->cfg.jacobi_cluster, ctx->num_sms, &L, &ctx->jacobi_tune);
  if (s != ZKQ_OK) return s;
  s = ensure(&ctx->meta, &ctx->meta_bytes, L.meta_bytes());
  if (s != ZKQ_OK) return s;
  s = ensure(&ctx->ws, &ctx->ws_bytes, L.ws_bytes());
  if (s != ZKQ_OK) return s;
  s = eigh_upload(L, ctx->meta, ctx->stage, st);
  if (s != ZKQ_OK) return s;
  return eigh_launch(L, ctx->meta, ctx->ws, A, a_words, W, V, info, ctx->cfg.max_sweeps, prof_class, st);
}
zkq_status rqi_refine_internal(void* vctx, int batch, const int32_t* n, const int64_t* a_off, const double* A,
                               int a_words, const double* W, const double* V, int target_words, double* W_out,
                               double* V_out, double* err_est, int32_t* info, cudaStream_t st) {
  zkq_ctx* ctx = (zkq_ctx*)vctx;
  RqiLayout L;
  zkq_status s = rqi_layout(batch, n, a_off, target_words, ctx->num_sms, &L);
  if (s != ZKQ_OK) return s;
  s = ensure(&ctx->meta, &ctx->meta_bytes, L.meta_bytes());
  if (s != ZKQ_OK) return s;
  s = ensure(&ctx->ws, &ctx->ws_bytes, L.ws_bytes());
  if (s != ZKQ_OK) return s;
  s = rqi_upload(L, ctx->meta, ctx->stage, st);
  if (s != ZKQ_OK) return s;
  return rqi_launch(L, ctx->meta, ctx->ws, A, a_words, W, V, target_words, W_out, V_out, err_est, info,
                    ctx->cfg.rqi_max_iter, st);
}
}  // namespace zkq

extern "C" {

zkq_status zkq_eigh_batched(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                            const double* A, int a_words, double* W, double* V, int32_t* info, void* stream) try {
  if (!ctx || batch < 0 || (batch > 0 && (!n || !a_off || !A || !W || !V || !info))) return ZKQ_EINVAL;
  if (a_words != 1 && a_words != 2 && a_words != 4) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  for (int b = 0; b < batch; ++b) if (n[b] < 1 || n[b] > 4096 || a_off[b] < 0) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));
  return eigh_internal(ctx, batch, n, a_off, A, a_words, W, V, info, (cudaStream_t)stream);
} catch (...) {
  return api_exception(ctx);
}

zkq_status zkq_svd_batched(zkq_ctx* ctx, int batch, const int32_t* m, const int32_t* n, const int64_t* a_off,
                           const double* A, int a_words, double* S, double* U, const int64_t* u_off, double* V,
                           const int64_t* v_off, int32_t* info, void* stream) try {
  if (!ctx || batch < 0 || (batch > 0 && (!m || !n || !a_off || !A || !S || !U || !u_off || !V || !v_off || !info)))
    return ZKQ_EINVAL;
  if (a_words != 1 && a_words != 2 && a_words != 4) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  for (int b = 0; b < batch; ++b)
    if (m[b] < 1 || n[b] < 1 || m[b] > 4096 || n[b] > 4096 || a_off[b] < 0 || u_off[b] < 0 || v_off[b] < 0) return ZKQ_EINVAL;
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));
  return svd_internal(ctx, batch, m, n, a_off, A, a_words, S, U, u_off, V, v_off, info, (cudaStream_t)stream,
                      &ctx->ws, &ctx->ws_bytes, &ctx->meta, &ctx->meta_bytes);
} catch (...) {
  return api_exception(ctx);
}

zkq_status zkq_rqi_refine(zkq_ctx* ctx, int batch, const int32_t* n, const int64_t* a_off,
                          const double* A, int a_words, const double* W, const double* V,
                          int target_words, int method, double* W_out, double* V_out, double* err_est,
                          int32_t* info, void* stream) try {
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
} catch (...) {
  return api_exception(ctx);
}

zkq_status zkq_workspace_size(zkq_ctx* ctx, int batch, const int32_t* n, int a_words, int target_words,
                              int method, size_t* bytes) try {
  if (!ctx || !bytes || batch < 0 || (batch > 0 && !n)) return ZKQ_EINVAL;
  *bytes = 0;
  if ((a_words != 1 && a_words != 2 && a_words != 4) || (target_words != 0 && target_words != 2 && target_words != 4))
    return ZKQ_EINVAL;
  if (method != ZKQ_PLAIN_RQI && method != ZKQ_OA_OZAKI && method != ZKQ_OA_FP64) return ZKQ_EINVAL;
  if (batch == 0) return ZKQ_OK;
  const bool oa = target_words != 0 && method != ZKQ_PLAIN_RQI;
  int64_t xe = 0, le = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > (oa ? 2048 : 4096)) return ZKQ_EINVAL;
    xe += (int64_t)n[b] * n[b]; le += n[b];
  }
  ZKQ_CUDA_TRY(cudaSetDevice(ctx->device));          // the layout asks the device for grid occupancy
  const std::vector<int64_t> zero(batch, 0);
  const size_t floor_bytes = (size_t)1 << 20;        // smallest allocation of every workspace buffer
  EighLayout L;
  zkq_status s = eigh_layout(batch, n, zero.data(), a_words, ctx->cfg.jacobi_cluster, ctx->num_sms, &L,
                             &ctx->jacobi_tune);
  if (s != ZKQ_OK) return s;
  size_t meta = std::max(L.meta_bytes(), floor_bytes), ws = std::max(L.ws_bytes(), floor_bytes);
  if (target_words != 0 && method == ZKQ_PLAIN_RQI) {  // the RQI shares the eigensolve's buffers
    RqiLayout R;
    s = rqi_layout(batch, n, zero.data(), target_words, ctx->num_sms, &R);
    if (s != ZKQ_OK) return s;
    meta = std::max(meta, R.meta_bytes());
    ws = std::max(ws, R.ws_bytes());
  }
  size_t total = meta + ws;
  if (oa) {
    total += oa_grow_bytes(oa_state_bytes(batch, xe, le, target_words) +
                           2 * oa_cache_bytes(batch, n, target_words, method == ZKQ_OA_OZAKI ? 1 : 0));
    // split products of one iteration over every problem: P = A X (with R = I - X^H X when A has W words),
    // then S = X^H P (with R otherwise), then X + X E.  Later iterations run subsets of these products.  When the batch mixes K' = 2n above and
    // below 1024, its products take the digit form while any order above 512 is still refining, and the CRT
    // form (with a modulus count set by the largest remaining K') once only orders up to 512 remain, so the
    // bound takes both.  Distinct dummy addresses stand for the distinct matrices of each problem.
    const int pm = method == ZKQ_OA_OZAKI ? 1 : 0, p_bits = 53 * target_words + 6, W = target_words;
    std::vector<double> tag(4 * (size_t)batch);
    auto ptr = [&](int t, int b) { return &tag[(size_t)t * batch + b]; };   // 0 A, 1 X, 2 P, 3 E
    bool above = false, below = false;
    for (int b = 0; b < batch; ++b) (n[b] > 512 ? above : below) = true;
    size_t zw = 0, zm = 0;
    for (int pass = 0; pass < (above && below ? 2 : 1); ++pass) {
      std::vector<MwProd> p1, p2, p3;
      for (int b = 0; b < batch; ++b) {
        if (pass == 1 && n[b] > 512) continue;
        const int k = n[b];
        p1.push_back({k, k, k, 0, ptr(0, b), ptr(1, b), nullptr, nullptr, 1.0, 0});
        p2.push_back({k, k, k, 1, ptr(1, b), ptr(2, b), nullptr, nullptr, 1.0, 0});
        // R = I - X^H X joins the first call when A has the working precision's words (as oa_refine does)
        (a_words == W ? p1 : p2).push_back({k, k, k, 1, ptr(1, b), ptr(1, b), nullptr, nullptr, -1.0, 1});
        p3.push_back({k, k, k, 0, ptr(1, b), ptr(3, b), nullptr, nullptr, 1.0, 0});
      }
      struct Call { const std::vector<MwProd>* p; int wa, wb; };
      const Call calls[3] = {{&p1, a_words, W}, {&p2, W, W}, {&p3, W, 2}};   // E is double-double
      for (const Call& c : calls) {
        size_t w_need = 0, m_need = 0;
        s = mw_gemm_workspace(c.p->data(), (int)c.p->size(), c.wa, c.wb, p_bits, pm, &w_need, &m_need);
        if (s != ZKQ_OK) return s;
        zw = std::max(zw, w_need); zm = std::max(zm, m_need);
      }
    }
    if (zw) total += oz_grow_bytes(zw);                // the FP64-pipe products use no workspace
    total += oz_grow_bytes(zm);
  }
  *bytes = total;
  return ZKQ_OK;
} catch (...) {
  return api_exception(nullptr);
}

zkq_status zkq_ctx_workspace_bytes(const zkq_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return ZKQ_EINVAL;
  *bytes = ctx->ws_bytes + ctx->meta_bytes + ctx->oa_bytes + ctx->oz_bytes + ctx->oz_meta_bytes + ctx->mps_bytes;
  return ZKQ_OK;
}

zkq_status zkq_mw_gemm(zkq_ctx* ctx, int count, const int32_t* m, const int32_t* n, const int32_t* k,
                       const int32_t* opA, const double* A, const int64_t* a_off, int wa, const double* B,
                       const int64_t* b_off, int wb, double* C, const int64_t* c_off, int wc, int p_bits, int method,
                       void* stream) try {
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
} catch (...) {
  return api_exception(ctx);
}

zkq_status zkq_set_gemm_kernel(int which) {
  if (which != 0 && which != 1) return ZKQ_EINVAL;
  gemm_kernel_set(which);
  return ZKQ_OK;
}

int zkq_get_gemm_kernel(void) { return gemm_kernel_get(); }

zkq_status zkq_check_device_waits(void) { return gemm_kernel_error() ? ZKQ_ETIMEOUT : ZKQ_OK; }
zkq_status zkq_set_gemm_tile_width(int width) {
  if (width != 0 && width != 128 && width != 256) return ZKQ_EINVAL;
  if (width == 0) gemm_wide_table_set({});
  else gemm_wide_table_set({{1 << 30, width == 256 ? 1 : 0}});
  return ZKQ_OK;
}
zkq_status zkq_test_grid_barrier_hook(int extra_arrivals, int log2_poll_limit) {
  return set_grid_barrier_hook(extra_arrivals, log2_poll_limit);
}

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

zkq_status zkq_profile_read(double* ms, int64_t* launches, double* work, int nclasses) try {
  if (!ms || !launches || !work || nclasses < 1) return ZKQ_EINVAL;
  Profiler& p = profiler();
  std::lock_guard<std::mutex> g(p.mu);
  for (int i = 0; i < nclasses; ++i) { ms[i] = 0.0; launches[i] = 0; work[i] = 0.0; }
  p.pool.reserve(p.pool.size() + 2 * p.recs.size());   // the loop below cannot throw
  // records read so far return their events to the pool and leave the list, also when a read fails
  size_t done = 0;
  cudaError_t e = cudaSuccess;
  for (; done < p.recs.size(); ++done) {
    const Profiler::Rec& r = p.recs[done];
    e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) break;
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    if (r.cls < nclasses) { ms[r.cls] += t; launches[r.cls] += 1; work[r.cls] += r.work; }
    p.pool.push_back(r.a); p.pool.push_back(r.b);
  }
  p.recs.erase(p.recs.begin(), p.recs.begin() + done);
  if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ECUDA; }
  if (g_prof_ctr) {                              // device-counted work (all recorded launches are complete)
    unsigned long long h[PC_COUNT];
    e = cudaMemcpy(h, g_prof_ctr, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_last_cuda_error(e); return ZKQ_ECUDA; }
    for (int i = 0; i < PC_COUNT && i < nclasses; ++i) work[i] += (double)h[i];
    cudaMemset(g_prof_ctr, 0, sizeof(h));
  }
  return ZKQ_OK;
} catch (...) {
  return api_exception(nullptr);
}

}  // extern "C"
