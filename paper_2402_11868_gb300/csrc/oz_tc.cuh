// Exact fp16 slice GEMM on the 5th-generation tensor cores (tcgen05.mma kind::f16, fp32 accumulator in
// tensor memory).  Same contract as oz_gemm_kernel: for every tile, a stream of slice pairs (t, u) whose
// exact integer products are accumulated per chunk, flushed to int32 and stored per level.
//
// CTA: 128 threads (4 warps), tile 128 rows x 128 columns, K staged 64 halves (one 128-byte swizzle atom)
// per step in STAGES shared-memory buffers filled with cp.async.  Thread 0 issues four K=16 MMAs per step
// and commits them to the step's mbarrier; at the end of each slice pair the accumulator is read back with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows), converted to int32 and added / stored
// (CRT form: stored as residues modulo the level's modulus, one byte per entry).
// Every mbarrier wait is bounded; on expiry the kernel raises *err and leaves.
#pragma once
#include <cstdint>
#include "ozaki.cuh"

namespace zkq {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 4;

struct OzTile;
struct CrtConst;
size_t oz_tc_smem_bytes();
// d_c: CRT constants (the levels are stored as uint8 residues) or null (int32 levels, digit form)
zkq_status launch_oz_tc(const OzProd* d_p, const OzTile* d_t, int ntiles, const OzPair* d_q, int npairs,
                        const CrtConst* d_c, int* d_err, cudaStream_t st);

}  // namespace zkq
