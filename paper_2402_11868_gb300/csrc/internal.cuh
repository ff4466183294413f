// Declarations shared by the library's translation units: launch descriptors of the batched kernels,
// internal entry points reused across stages, and the pinned host staging ring of a context.
#pragma once
#include <cstdint>
#include <cstddef>
#include <deque>
#include <vector>
#include <utility>
#include <cuda_runtime.h>
#include "common.cuh"

namespace zkq {

// ---- pinned host staging -------------------------------------------------------------------------
// The small per-call uploads (batch metadata, tile and pair lists, CRT constants) and the per-iteration
// statistics read-back go through one pinned ring per context: copies from pageable memory may wait for
// the stream to drain, copies from pinned memory stay asynchronous, so the host prepares the next launch
// while the device works.  A region is handed out again only after the event recorded behind the copy
// that read (or wrote) it has completed.  A context, and so its ring, is used by one host thread at a time.
class HostStage {
 public:
  HostStage() = default;
  HostStage(const HostStage&) = delete;
  HostStage& operator=(const HostStage&) = delete;
  ~HostStage();
  // H2D copy of `bytes` from pageable `src` to device `dst`, ordered on `st`
  cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t st);
  // D2H copy of `bytes` from device `src` to `dst`; waits for `st` (the caller reads the data next)
  cudaError_t download_sync(void* dst, const void* src, size_t bytes, cudaStream_t st);
  // several uploads through one pinned region and one event: add() the pieces (copied at once), then flush()
  void add(void* dst, const void* src, size_t bytes);
  cudaError_t flush(cudaStream_t st);
  // drop the pieces add() collected since the last flush() (a call that failed before sending them)
  void discard() noexcept { pend_.clear(); pieces_.clear(); }
 private:
  struct Span { size_t lo, hi; cudaEvent_t ev; };
  struct Piece { void* dst; size_t off, bytes; };
  char* buf_ = nullptr;
  size_t cap_ = 0, head_ = 0;
  std::deque<Span> inflight_;
  std::vector<cudaEvent_t> free_ev_;
  std::vector<char> pend_;                            // pieces collected by add() before flush()
  std::vector<Piece> pieces_;
  cudaError_t reserve(size_t bytes, size_t* off);
  cudaError_t fence(size_t lo, size_t hi, cudaStream_t st);
};

// ---- FP64 Jacobi ---------------------------------------------------------------------------------
struct JacobiBatch {
  const int32_t* n; const int64_t* a_off; const int64_t* w_off; const int32_t* order;
  const double* A; double* W; double* V; int32_t* info; double* ws; const int64_t* ws_off; double* red;
  int max_sweeps;
  unsigned long long* flops;     // device counter of applied-rotation flops (null: not counted)
  int prof_class;                // profiler class of the launches
};
// grid barrier state of the cooperative Jacobi launch (zeroed before each launch)
struct GridBar { unsigned count; unsigned gen; int abort; int pad; };
// small problems: one CTA each; large problems: a cluster of `cluster` CTAs each, or, when grid_blocks > 0
// (few large problems), a cooperative grid of grid_blocks CTAs split into one group per large problem:
// blocks grp_start[q] .. grp_start[q+1]-1 (device array, n_large + 1 entries), barrier gb[q], reduction
// slots red + q red_stride
zkq_status launch_jacobi(const JacobiBatch& jb, int a_words, int n_small, int n_large, int max_small_n,
                         int max_large_n, int cluster, int grid_blocks, GridBar* gb, const int32_t* grp_start,
                         int red_stride, cudaStream_t st);
size_t jacobi_smem_bytes(int n);
int jacobi_grid_max_blocks(int max_large_n, int a_words);   // co-resident blocks per SM of the grid kernel
// test hook of the cooperative grid barrier on the current device (zkq_test_grid_barrier_hook)
zkq_status set_grid_barrier_hook(int extra_arrivals, int log2_poll_limit);

// ---- plain RQI -----------------------------------------------------------------------------------
struct RqiBatch {
  const int32_t* n; const int64_t* a_off; const int64_t* w_off; const int32_t* pair_prob;
  const double* A; const double* W; const double* V;
  double* W_out; double* V_out; double* err; int32_t* info;
  double* ws; int64_t ws_stride; int64_t total_pairs; int max_iter; int* counter;
};
zkq_status launch_rqi(const RqiBatch& rb, int W, int WA, int grid, cudaStream_t st);
size_t rqi_slot_doubles(int nmax, int W);

// ---- refinement ----------------------------------------------------------------------------------
struct OaBuffers {
  void** ws; size_t* ws_bytes; void** oz_ws; size_t* oz_bytes; void** oz_meta; size_t* oz_meta_bytes;
  HostStage* stage;
};
zkq_status oa_refine(void* ctx, const OaBuffers& buf, int batch, const int32_t* n, const int64_t* a_off,
                     const double* A, int wa, const double* V, int W, double* W_out, double* V_out, double* err,
                     int32_t* info, int max_iter, int prod_method, cudaStream_t st);
// bytes of the refinement state oa_refine lays out (xe = sum n^2, le = sum n, W words per real), and the
// device bytes its buffer holds once grown to `need` bytes from nothing
size_t oa_state_bytes(int batch, int64_t xe, int64_t le, int W);
// bytes of one of the refinement's two plane caches (A; X^H within an iteration), each added to the state
size_t oa_cache_bytes(int batch, const int32_t* n, int W, int prod_method);
size_t oa_grow_bytes(size_t need);

// ---- batch layouts (layout.cu) -----------------------------------------------------------------------
// FP64 eigensolve: device metadata [n | a_off | w_off | order | ws_off | block groups] (meta_bytes) and
// workspace [large-problem copies of A and V | reduction slots | grid barriers] (ws_bytes)
struct EighLayout {
  int batch = 0, n_small = 0, n_large = 0, max_small = 0, max_large = 0, cluster = 2, grid_blocks = 0, red_stride = 0;
  std::vector<int32_t> n, order, grp;
  std::vector<int64_t> a_off, w_off, ws_off;
  size_t ws_need = 0, red_bytes = 0, gb_bytes = 0;
  size_t meta_bytes() const;
  size_t ws_bytes() const;
};
// cluster width of the large problems: cfg_cluster if > 0, else the tuning table's entry for the largest
// order (tune: (order, width) pairs by increasing order, from zkq_autotune_jacobi; the first entry whose
// order is >= the largest order, else the last), else 2 / 4 / 8 for largest orders <= 128 / 256 / above
using JacobiTune = std::vector<std::pair<int, int>>;
zkq_status eigh_layout(int batch, const int32_t* n, const int64_t* a_off, int a_words, int cfg_cluster, int num_sms,
                       EighLayout* L, const JacobiTune* tune = nullptr);
// the metadata as the device holds it (meta_bytes() bytes), for an upload by the caller
void eigh_meta_image(const EighLayout& L, std::vector<char>* img);
zkq_status eigh_upload(const EighLayout& L, void* meta, HostStage& hs, cudaStream_t st);
zkq_status eigh_launch(const EighLayout& L, const void* meta, void* ws, const double* A, int a_words, double* W,
                       double* V, int32_t* info, int max_sweeps, int prof_class, cudaStream_t st);
// plain RQI: device metadata [n | a_off | w_off | eigenpair -> problem | work counter], workspace grid slots
struct RqiLayout {
  int batch = 0, grid = 0;
  int64_t total = 0;
  size_t slot = 0;
  std::vector<int32_t> n, pair_prob;
  std::vector<int64_t> a_off, w_off;
  size_t meta_bytes() const;
  size_t ws_bytes() const;
};
zkq_status rqi_layout(int batch, const int32_t* n, const int64_t* a_off, int target_words, int num_sms, RqiLayout* L);
zkq_status rqi_upload(const RqiLayout& L, void* meta, HostStage& hs, cudaStream_t st);
// also clears the work counter and info (stream-ordered memsets)
zkq_status rqi_launch(const RqiLayout& L, const void* meta, void* ws, const double* A, int a_words, const double* W,
                      const double* V, int target_words, double* W_out, double* V_out, double* err, int32_t* info,
                      int max_iter, cudaStream_t st);

// ---- FP64 one-sided Jacobi SVD (svd.cu) -------------------------------------------------------------
// A_b (m_b x n_b, a_words words per real, element offset a_off[b]) = U diag(S) V^H, thin (k_b = min(m_b, n_b)):
// S at offset sum_{c<b} k_c, U (m_b x k_b complex FP64) at element offset u_off[b], V (n_b x k_b) at v_off[b];
// info[b] 0 converged, > 0 sweep limit.  ws / meta: the caller's growable device buffers.
zkq_status svd_internal(void* ctx, int batch, const int32_t* m, const int32_t* n, const int64_t* a_off, const double* A,
                        int a_words, double* S, double* U, const int64_t* u_off, double* V, const int64_t* v_off,
                        int32_t* info, cudaStream_t st, void** ws, size_t* ws_bytes, void** meta, size_t* meta_bytes);

// ---- context internals ---------------------------------------------------------------------------
// prof_class: profiler class of the launches (0 = PC_JACOBI; the refinement's cluster solves use their own)
zkq_status eigh_internal(void* ctx, int batch, const int32_t* n, const int64_t* a_off, const double* A, int a_words,
                         double* W, double* V, int32_t* info, cudaStream_t st, int prof_class = 0);
zkq_status rqi_refine_internal(void* ctx, int batch, const int32_t* n, const int64_t* a_off, const double* A,
                               int a_words, const double* W, const double* V, int target_words, double* W_out,
                               double* V_out, double* err_est, int32_t* info, cudaStream_t st);
OaBuffers ctx_oa_buffers(void* ctx);
int ctx_oa_max_iter(void* ctx);
void** ctx_mps_ws(void* ctx, size_t** bytes);
// the context's FP64-stage workspace and metadata buffers (shared by the Jacobi, plain RQI and SVD launches)
void ctx_fp64_bufs(void* ctx, void*** ws, size_t** ws_bytes, void*** meta, size_t** meta_bytes);
HostStage* ctx_stage(void* ctx);
JacobiTune* ctx_jacobi_tune(void* ctx);
int ctx_num_sms(void* ctx);
int ctx_device(void* ctx);
const zkq_config& ctx_config(void* ctx);
zkq_config& ctx_config_mut(void* ctx);

// ---- exceptions at the C ABI ----------------------------------------------------------------------
// No exception may cross the C ABI.  Host allocations (std::vector growth, new) can throw std::bad_alloc or
// std::length_error; the entry points that allocate catch every exception and return api_exception(ctx):
// ZKQ_ENOMEM, after dropping the uploads that the failed call collected in the context's staging ring, so
// that no later call sends them (ctx may be null).
zkq_status api_exception(void* ctx) noexcept;

// ---- split-product GEMM kernel choice --------------------------------------------------------------
int gemm_kernel_get();
void gemm_kernel_set(int k);
bool gemm_kernel_error();
// tile-width table of the tcgen05 slice GEMM: (largest K' of a batch, 1 = 256-column tiles, 0 = 128)
void gemm_wide_table_set(const std::vector<std::pair<int, int>>& t);
std::vector<std::pair<int, int>> gemm_wide_table_get();

}  // namespace zkq
