// The device-resident Vidal MPS handle, shared by the gate updates (mps.cu) and the measurements
// (mps_measure.cu).
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include "../../include/zkq.h"

struct zkq_mps {
  int n, r_max, W, device;
  std::vector<int> chi;            // chi[l], l = 0..n-2 (bond between l and l+1)
  std::vector<int> cap;            // capacity per bond
  std::vector<double*> gamma;      // per site, capacity 2 * cap_{l-1} * cap_l complex elements
  std::vector<double*> lam;        // per bond, capacity cap_l real values
  double* gate = nullptr;          // 4x4 (or 2x2) device copy of the current gate
  // device table: gamma pointers [n], lambda pointers [n] (the last unused), then int32 dims [n + 1]
  // (dims[l] = chi[l-1], 1 at both ends; rewritten by the calls that read it)
  double** d_ptrs = nullptr;
  cudaEvent_t done = nullptr;      // recorded behind the last asynchronous call (apply1q) for destroy
};
