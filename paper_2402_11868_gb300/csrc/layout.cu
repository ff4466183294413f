// Batch layouts of the FP64 eigensolve and the plain RQI refinement: the host-side scheduling metadata
// (size classes, orders, workspace offsets, block groups), its upload, and the launches.  The per-call entry
// points lay out, upload and launch every call; a plan does the first two once and then only launches.
#include <algorithm>
#include <cstring>
#include <vector>
#include "internal.cuh"
#include "prof.cuh"

namespace zkq {

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
static constexpr int kSmallMax = 80;     // orders held in shared memory by one CTA

size_t EighLayout::meta_bytes() const {
  return al(batch * 4) + 3 * al(batch * 8) + al(batch * 4) + al((grp.size() + 1) * 4);
}
size_t EighLayout::ws_bytes() const { return ws_need + red_bytes + gb_bytes; }

zkq_status eigh_layout(int batch, const int32_t* n, const int64_t* a_off, int a_words, int cfg_cluster, int num_sms,
                       EighLayout* L, const JacobiTune* tune) {
  *L = EighLayout{};
  L->batch = batch;
  L->n.assign(n, n + batch);
  L->a_off.assign(a_off, a_off + batch);
  L->w_off.assign(batch, 0);
  L->ws_off.assign(batch, 0);
  std::vector<int32_t> small, large;
  int64_t acc = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > 4096 || a_off[b] < 0) return ZKQ_EINVAL;
    L->w_off[b] = acc; acc += n[b];
    if (n[b] <= kSmallMax) { small.push_back(b); L->max_small = std::max(L->max_small, n[b]); }
    else { large.push_back(b); L->max_large = std::max(L->max_large, n[b]); }
  }
  std::sort(large.begin(), large.end(), [&](int a, int c) { return n[a] > n[c] || (n[a] == n[c] && a < c); });
  // per large problem: A and V (n^2 complex each)
  for (int b : large) {
    L->ws_off[b] = (int64_t)(L->ws_need / sizeof(double));
    L->ws_need += al((size_t)n[b] * n[b] * 4 * sizeof(double));
  }
  L->n_small = (int)small.size(); L->n_large = (int)large.size();
  int cluster = cfg_cluster;
  if (cluster <= 0 && tune && !tune->empty()) {
    cluster = tune->back().second;
    for (const auto& e : *tune) if (e.first >= L->max_large) { cluster = e.second; break; }
  }
  if (cluster <= 0) cluster = L->max_large <= 128 ? 2 : (L->max_large <= 256 ? 4 : 8);
  L->cluster = std::min(cluster, 16);
  // few large problems: a cooperative grid with one block group per problem instead of a cluster each (a
  // cluster of at most 16 CTAs per problem would leave most SMs idle)
  if (!large.empty() && (int)large.size() * L->cluster * 2 <= num_sms) {
    const int cap = jacobi_grid_max_blocks(L->max_large, a_words) * num_sms;   // co-resident blocks
    // about five block updates per thread and round: n^2 / 2048 blocks (2 .. 128) per problem, scaled
    // down by the n^3 work share when the wanted total exceeds what is co-resident
    std::vector<int> want(large.size());
    long tot = 0; double w3 = 0;
    for (size_t q = 0; q < large.size(); ++q) {
      const int nq = n[large[q]];
      want[q] = std::min(128, std::max(2, nq * nq / 2048));
      tot += want[q]; w3 += (double)nq * nq * nq;
    }
    if (tot > cap) {
      tot = 0;
      for (size_t q = 0; q < large.size(); ++q) {
        const double nq = n[large[q]];
        want[q] = std::max(1, std::min(want[q], (int)(cap * nq * nq * nq / w3)));
        tot += want[q];
      }
    }
    if (cap > 0 && tot <= cap) {
      L->grp.resize(large.size() + 1);
      L->grp[0] = 0;
      for (size_t q = 0; q < large.size(); ++q) L->grp[q + 1] = L->grp[q] + want[q];
      L->grid_blocks = L->grp.back();
      L->red_stride = 2 * (*std::max_element(want.begin(), want.end())) + 64;
    }
  }
  L->red_bytes = al((size_t)64 * std::max<size_t>(1, large.size()) * sizeof(double));
  L->red_bytes = std::max(L->red_bytes, al((size_t)L->red_stride * std::max<size_t>(1, large.size()) * sizeof(double)));
  L->gb_bytes = al(sizeof(GridBar) * std::max<size_t>(1, large.size()));
  L->order = small;
  L->order.insert(L->order.end(), large.begin(), large.end());
  return ZKQ_OK;
}

namespace {
struct EighMeta { int32_t* n; int64_t* a_off; int64_t* w_off; int32_t* order; int64_t* ws_off; int32_t* grp; };
EighMeta eigh_meta(const EighLayout& L, const void* meta) {
  char* mb = (char*)meta;
  const size_t m_n = al(L.batch * 4), m_8 = al(L.batch * 8), m_o = al(L.batch * 4);
  EighMeta m;
  m.n = (int32_t*)mb; m.a_off = (int64_t*)(mb + m_n); m.w_off = (int64_t*)(mb + m_n + m_8);
  m.order = (int32_t*)(mb + m_n + 2 * m_8); m.ws_off = (int64_t*)(mb + m_n + 2 * m_8 + m_o);
  m.grp = (int32_t*)(mb + m_n + 3 * m_8 + m_o);
  return m;
}
}  // namespace

void eigh_meta_image(const EighLayout& L, std::vector<char>* img) {
  img->assign(L.meta_bytes(), 0);
  char* base = img->data();
  const EighMeta m = eigh_meta(L, base);        // the device layout, laid over the host image
  std::memcpy(m.n, L.n.data(), L.batch * 4);
  std::memcpy(m.a_off, L.a_off.data(), L.batch * 8);
  std::memcpy(m.w_off, L.w_off.data(), L.batch * 8);
  std::memcpy(m.order, L.order.data(), L.batch * 4);
  std::memcpy(m.ws_off, L.ws_off.data(), L.batch * 8);
  if (!L.grp.empty()) std::memcpy(m.grp, L.grp.data(), L.grp.size() * 4);
}

zkq_status eigh_upload(const EighLayout& L, void* meta, HostStage& hs, cudaStream_t st) {
  std::vector<char> img;
  eigh_meta_image(L, &img);
  hs.add(meta, img.data(), img.size());
  ZKQ_CUDA_TRY(hs.flush(st));
  return ZKQ_OK;
}

zkq_status eigh_launch(const EighLayout& L, const void* meta, void* ws, const double* A, int a_words, double* W,
                       double* V, int32_t* info, int max_sweeps, int prof_class, cudaStream_t st) {
  const EighMeta m = eigh_meta(L, meta);
  unsigned long long* ctr = prof_device_counters();
  JacobiBatch jb{m.n, m.a_off, m.w_off, m.order, A, W, V, info, (double*)ws, m.ws_off,
                 (double*)((char*)ws + L.ws_need), max_sweeps, ctr ? ctr + prof_class : nullptr, prof_class};
  GridBar* gb = (GridBar*)((char*)ws + L.ws_need + L.red_bytes);
  return launch_jacobi(jb, a_words, L.n_small, L.n_large, L.max_small, L.max_large, L.cluster, L.grid_blocks, gb,
                       m.grp, L.red_stride, st);
}

// ---- plain RQI ---------------------------------------------------------------------------------------
size_t RqiLayout::meta_bytes() const { return al(batch * 4) + 2 * al(batch * 8) + al(total * 4) + 256; }
size_t RqiLayout::ws_bytes() const { return slot * sizeof(double) * grid; }

zkq_status rqi_layout(int batch, const int32_t* n, const int64_t* a_off, int target_words, int num_sms, RqiLayout* L) {
  *L = RqiLayout{};
  L->batch = batch;
  L->n.assign(n, n + batch);
  L->a_off.assign(a_off, a_off + batch);
  L->w_off.assign(batch, 0);
  int nmax = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > 4096 || a_off[b] < 0) return ZKQ_EINVAL;
    L->w_off[b] = L->total; L->total += n[b]; nmax = std::max(nmax, n[b]);
  }
  L->pair_prob.resize(L->total);
  for (int b = 0; b < batch; ++b) for (int i = 0; i < n[b]; ++i) L->pair_prob[L->w_off[b] + i] = b;
  L->grid = (int)std::min<int64_t>(L->total, (int64_t)num_sms);
  L->slot = rqi_slot_doubles(nmax, target_words);
  return ZKQ_OK;
}

namespace {
struct RqiMeta { int32_t* n; int64_t* a_off; int64_t* w_off; int32_t* pair_prob; int* counter; };
RqiMeta rqi_meta(const RqiLayout& L, const void* meta) {
  char* mb = (char*)meta;
  const size_t m_n = al(L.batch * 4), m_8 = al(L.batch * 8), m_p = al(L.total * 4);
  return RqiMeta{(int32_t*)mb, (int64_t*)(mb + m_n), (int64_t*)(mb + m_n + m_8), (int32_t*)(mb + m_n + 2 * m_8),
                 (int*)(mb + m_n + 2 * m_8 + m_p)};
}
}  // namespace

zkq_status rqi_upload(const RqiLayout& L, void* meta, HostStage& hs, cudaStream_t st) {
  const RqiMeta m = rqi_meta(L, meta);
  hs.add(m.n, L.n.data(), L.batch * 4);
  hs.add(m.a_off, L.a_off.data(), L.batch * 8);
  hs.add(m.w_off, L.w_off.data(), L.batch * 8);
  hs.add(m.pair_prob, L.pair_prob.data(), L.total * 4);
  ZKQ_CUDA_TRY(hs.flush(st));
  return ZKQ_OK;
}

zkq_status rqi_launch(const RqiLayout& L, const void* meta, void* ws, const double* A, int a_words, const double* W,
                      const double* V, int target_words, double* W_out, double* V_out, double* err, int32_t* info,
                      int max_iter, cudaStream_t st) {
  const RqiMeta m = rqi_meta(L, meta);
  ZKQ_CUDA_TRY(cudaMemsetAsync(m.counter, 0, sizeof(int), st));
  ZKQ_CUDA_TRY(cudaMemsetAsync(info, 0, L.batch * sizeof(int32_t), st));
  RqiBatch rb{m.n, m.a_off, m.w_off, m.pair_prob, A, W, V, W_out, V_out, err, info, (double*)ws, (int64_t)L.slot,
              L.total, max_iter, m.counter};
  return launch_rqi(rb, target_words, a_words, L.grid, st);
}

}  // namespace zkq
