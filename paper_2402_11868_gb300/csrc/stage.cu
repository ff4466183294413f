// Pinned host staging ring (see internal.cuh).
#include <cstring>
#include <algorithm>
#include <mutex>
#include <set>
#include <utility>
#include "internal.cuh"

namespace zkq {

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

HostStage::~HostStage() {
  for (auto& s : inflight_) { cudaEventSynchronize(s.ev); cudaEventDestroy(s.ev); }
  for (auto e : free_ev_) cudaEventDestroy(e);
  if (buf_) cudaFreeHost(buf_);
}

// a region [off, off + bytes) whose earlier users have completed
cudaError_t HostStage::reserve(size_t bytes, size_t* off) {
  const size_t b = al256(std::max<size_t>(bytes, 1));
  if (b > cap_) {                                     // grow: wait for every copy, then reallocate
    for (auto& s : inflight_) { cudaError_t e = cudaEventSynchronize(s.ev); if (e != cudaSuccess) return e; free_ev_.push_back(s.ev); }
    inflight_.clear();
    if (buf_) { cudaFreeHost(buf_); buf_ = nullptr; cap_ = 0; }
    const size_t want = std::max<size_t>(al256(b) * 2, (size_t)16 << 20);
    void* p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, want, cudaHostAllocDefault);
    if (e != cudaSuccess) return e;
    buf_ = (char*)p; cap_ = want; head_ = 0;
  }
  if (head_ + b > cap_) head_ = 0;                    // wrap
  const size_t lo = head_, hi = head_ + b;
  // spans are handed out circularly, so the oldest ones (front) are the ones right after head
  while (!inflight_.empty() && inflight_.front().lo < hi && lo < inflight_.front().hi) {
    cudaError_t e = cudaEventSynchronize(inflight_.front().ev);
    if (e != cudaSuccess) return e;
    free_ev_.push_back(inflight_.front().ev);
    inflight_.pop_front();
  }
  head_ = hi;
  *off = lo;
  return cudaSuccess;
}

cudaError_t HostStage::fence(size_t lo, size_t hi, cudaStream_t st) {
  cudaEvent_t ev;
  if (!free_ev_.empty()) { ev = free_ev_.back(); free_ev_.pop_back(); }
  else { cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming); if (e != cudaSuccess) return e; }
  cudaError_t e = cudaEventRecord(ev, st);
  if (e != cudaSuccess) { free_ev_.push_back(ev); return e; }
  inflight_.push_back({lo, hi, ev});
  return cudaSuccess;
}

cudaError_t HostStage::upload(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  size_t off;
  cudaError_t e = reserve(bytes, &off);
  if (e != cudaSuccess) return e;
  std::memcpy(buf_ + off, src, bytes);
  e = cudaMemcpyAsync(dst, buf_ + off, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return fence(off, off + al256(bytes), st);
}

cudaError_t HostStage::download_sync(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaStreamSynchronize(st);
  size_t off;
  cudaError_t e = reserve(bytes, &off);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(buf_ + off, src, bytes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  std::memcpy(dst, buf_ + off, bytes);
  return fence(off, off + al256(bytes), st);          // already complete; keeps the ring bookkeeping uniform
}

void HostStage::add(void* dst, const void* src, size_t bytes) {
  const size_t off = al256(pend_.size());
  pend_.resize(off + bytes);
  if (bytes) std::memcpy(pend_.data() + off, src, bytes);
  pieces_.push_back({dst, off, bytes});
}

cudaError_t HostStage::flush(cudaStream_t st) {
  if (pieces_.empty()) return cudaSuccess;
  size_t off;
  cudaError_t e = reserve(pend_.size(), &off);
  if (e == cudaSuccess) {
    std::memcpy(buf_ + off, pend_.data(), pend_.size());
    for (const Piece& p : pieces_) {
      if (p.bytes == 0) continue;
      e = cudaMemcpyAsync(p.dst, buf_ + off + p.off, p.bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = fence(off, off + al256(pend_.size()), st);
  }
  pend_.clear();
  pieces_.clear();
  return e;
}

cudaError_t raise_smem_limit(const void* kernel, int slot) {
  static std::mutex mu;
  static std::set<std::pair<int, int>> done;        // (slot, device)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  if (done.count({slot, dev})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes a;
  e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({slot, dev});
  return e;
}

}  // namespace zkq
