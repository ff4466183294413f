// Ozaki-style error-free split products for multi-word complex matrices (Ozaki, Ogita, Oishi, Rump 2012),
// the dense products A X, X^H X, X^H (A X) and X E of the refinement step.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_fp16.h>
#include "common.cuh"

namespace zkq {

// One product C = base + sgn * op(A) B of multi-word complex matrices (column-major, packed):
//   opA = 0: A is m x k (ld m);  opA = 1: A is stored k x m (ld k) and op(A) = A^H.
//   B is k x n (ld k);  C is m x n (ld m); base (m x n, wc words) may be null, or equal C when C is not
//   an input of the product; base_identity adds the identity instead of a base matrix.
struct MwProd {
  int m, n, k, opA;
  const double* A; const double* B; double* C; const double* base;
  double sgn; int base_identity;
  int hermitian = 0;             // C is Hermitian (m == n): only tiles touching i <= j are computed and the
                                 // lower triangle is written as the conjugate of the upper one
  int keepA = 0;                 // k > 0: op(A) stays the same over several calls; its residue planes are
                                 // kept in the caller's k-th PlaneCache and reused (CRT form)
};

// Residue planes of operands that stay the same over several calls (the refinement's input matrix).  The
// caller lends a device region for the whole sequence of calls; mw_gemm_batched keeps there the op(A)
// planes and row exponents of products marked keepA, keyed by the operand (pointer, orientation, shape)
// and the CRT constants, and later calls reuse them instead of splitting op(A) again.  The contents of a
// cached operand must not change while its entry is in use; clear() forgets every entry.
struct PlaneCache {
  char* buf = nullptr;
  size_t bytes = 0, used = 0;
  struct Entry { const double* A; int opA, m, k, q, r, s; __half* planes; int32_t* exps; };
  std::vector<Entry> entries;
  void clear() { used = 0; entries.clear(); }
};
// bytes one cached operand of m rows and inner dimension k takes with r moduli (planes and exponents)
size_t plane_cache_entry_bytes(int m, int k, int r);
// moduli of the CRT form for inner dimension k at p_out_bits (0 when the digit form applies)
int crt_moduli(int k, int p_out_bits);

// device-side layout of one product inside the Ozaki workspace
struct OzProd {
  int m, n, k, opA;
  int mp, np2, kp;               // padded: rows of op(A), columns of [Re|Im] output, K' = 2k
  const double* A; const double* B; double* C; const double* base; double sgn; int base_identity;
  __half* Ahat;                  // [sA][mp][kp]
  __half* Bhat;                  // [sB][np2][kp]
  int32_t* D;                    // digit form: int32 [S+1][mp][np2] (levels 2..S used);
                                 // CRT form: uint8 residues [3r][mp][np2] (cast), reduced in the GEMM epilogue
  int32_t* eA;                   // row exponents of op(A) (m)
  int32_t* eB;                   // column exponents of B (n)
  int hermitian;
  int sliceA, sliceB;            // 0: the planes are shared with an earlier product of the batch
};

struct OzPair { int16_t t, u; int16_t level; int16_t flags; };   // flags: 1 chunk end, 2 level end

// one output tile: rows 128 ti.., columns 128 tj.. of product `prod`, w x 128 columns wide (w = 1 or 2), over
// the pairs p0 .. p1-1 of the pair list (the tcgen05 kernel's CRT form may split a tile's pairs over several
// CTAs: every pair there is its own level with its own output planes)
struct OzTile { int prod, ti, tj, w, p0, p1; };

struct OzPlan {
  int b;            // digit width (bits)
  int sA, sB, S;    // digit counts and the highest level kept
  int G;            // pairs per exact fp32 chunk
  int npairs;
};

OzPlan ozaki_plan(int max_kprime, int wa, int wb, int p_out_bits);

class HostStage;
// Run a batch of products (all with the same word counts and output precision).  method 1: CRT residue
// products on the tensor cores (digit form when K' > 1024); method 2: digit form; method 0: plain
// multi-word GEMM on the FP64 pipe.  Metadata goes up through `stage` (pinned) when it is given.
zkq_status mw_gemm_batched(const MwProd* prods, int count, int wa, int wb, int wc, int p_out_bits, int method,
                           void** ws, size_t* ws_bytes, void** meta, size_t* meta_bytes, cudaStream_t st,
                           HostStage* stage, PlaneCache* const* caches = nullptr, int ncaches = 0);
// Bytes mw_gemm_batched needs for the batch: its workspace exactly when no PlaneCache serves it (an upper
// bound otherwise), its metadata as an upper bound (host-side only; the operand pointers are compared, never
// read).
zkq_status mw_gemm_workspace(const MwProd* prods, int count, int wa, int wb, int p_out_bits, int method,
                             size_t* ws_need, size_t* meta_need);
// device bytes held once the split-product workspace or metadata has grown to `need` bytes from nothing
size_t oz_grow_bytes(size_t need);

}  // namespace zkq
