// Launch profiler: when enabled, every library kernel launch is bracketed by CUDA events recorded on the
// launching stream, and device time is accumulated per kernel class.  Read after the stream synchronises.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include <mutex>

namespace zkq {

// PC_JACOBI: the FP64 eigensolve of the inputs; PC_JACOBI_CLUSTER: the same kernels on the refinement's
// cluster blocks
enum ProfClass { PC_JACOBI = 0, PC_RQI, PC_OZ_SCALE, PC_OZ_SLICE, PC_OZ_GEMM, PC_OZ_COMBINE, PC_OA, PC_MPS, PC_OTHER,
                 PC_JACOBI_CLUSTER, PC_COUNT };

struct Profiler {
  bool on = false;
  std::mutex mu;
  struct Rec { int cls; cudaEvent_t a, b; double work; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e; cudaEventCreate(&e); return e;
  }
};
Profiler& profiler();
// Device-side algorithmic work counters (one unsigned 64-bit counter per class; flops counted by the
// kernels themselves where the work depends on the data, e.g. the rotations Jacobi applies).  Null when
// profiling is off.
unsigned long long* prof_device_counters();

// RAII bracket around one launch
struct ProfScope {
  int cls; cudaStream_t st; cudaEvent_t a = nullptr; double work;
  // work: algorithmic flops of the launch (0 if not counted)
  ProfScope(int c, cudaStream_t s, double w = 0.0) : cls(c), st(s), work(w) {
    Profiler& p = profiler();
    if (!p.on) return;
    std::lock_guard<std::mutex> g(p.mu);
    a = p.get();
    cudaEventRecord(a, st);
  }
  ~ProfScope() {
    if (!a) return;
    Profiler& p = profiler();
    std::lock_guard<std::mutex> g(p.mu);
    cudaEvent_t b = p.get();
    cudaEventRecord(b, st);
    try {
      p.recs.push_back({cls, a, b, work});
    } catch (...) {                  // out of host memory: the launch goes unrecorded (a destructor may not throw)
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  }
};

}  // namespace zkq
