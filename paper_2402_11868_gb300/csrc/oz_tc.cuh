// Exact fp16 slice GEMM on the 5th-generation tensor cores (tcgen05.mma kind::f16, fp32 accumulator in
// tensor memory).  Same contract as oz_gemm_kernel: for every tile, a stream of slice pairs (t, u) whose
// exact integer products are accumulated per chunk, flushed to int32 and stored per level.
//
// CTA: 7 warps in three roles, tile 128 rows x 128 columns, K staged 64 halves (one 128-byte swizzle
// atom) per step in STAGES shared-memory buffers.  Two producer warps fill the stages with cp.async; one
// lane issues four K=16 MMAs per stage; four epilogue warps read finished accumulators back with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows), convert them to int32 and add / store them
// (CRT form: residues modulo the level's modulus, one byte per entry).  Two accumulators (2 x 128 TMEM
// columns) alternate between accumulation groups, so the epilogue of one group overlaps the MMAs of the
// next.  The roles hand stages and accumulators to one another through mbarriers.
// Every mbarrier wait is bounded; on expiry the kernel raises *err and leaves.
#pragma once
#include <cstdint>
#include "ozaki.cuh"

namespace zkq {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;
// stages per tile width: 6 x 32 KB (128 columns) or 4 x 48 KB (256 columns)
__host__ __device__ constexpr int tc_stages(int bn) { return bn == 256 ? 4 : 6; }

struct CrtConst;
size_t oz_tc_smem_bytes(int bn, int npairs);
// d_c: CRT constants (the levels are stored as uint8 residues; tiles 128 or 256 columns wide) or null
// (int32 levels, digit form; 128-column tiles only).
zkq_status launch_oz_tc(const OzProd* d_p, const OzTile* d_t, int ntiles, const OzPair* d_q, int npairs,
                        const CrtConst* d_c, int* d_err, cudaStream_t st);

}  // namespace zkq
