// tcgen05 slice GEMM (see oz_tc.cuh).
#include "oz_tc.cuh"
#include "common.cuh"
#include "crt.cuh"

namespace zkq {

struct OzTile { int prod, ti, tj; };

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- mbarrier helpers ----
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(tc_smem_u32(b)), "r"(count));
}
// bounded wait for the phase with parity `par`; returns false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par) {
  uint32_t addr = tc_smem_u32(b);
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(addr), "r"(par));
    if (ok) return true;
  }
  return false;
}

// ---- descriptors ----
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
  d |= (uint64_t)2 << 61;                           // swizzle mode: 128B
  return d;
}
// instruction descriptor, kind::f16: D f32, A/B f16, both K-major, N = 128, M = 128
__device__ __forceinline__ uint32_t instr_desc() {
  uint32_t d = 0;
  d |= 1u << 4;                                     // D format f32
  d |= 0u << 7;                                     // A format f16
  d |= 0u << 10;                                    // B format f16
  d |= (uint32_t)(TC_BN >> 3) << 17;                // N >> 3
  d |= (uint32_t)(TC_BM >> 4) << 24;                // M >> 4
  return d;
}

__device__ __forceinline__ void cp_async16_tc(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" :: "r"(dst), "l"(src));
}
// 128-byte swizzle: 16-byte chunk c of row r lives at r*128 + ((c ^ (r & 7)) * 16)
__device__ __forceinline__ int sw128(int row, int chunk) { return row * 128 + ((chunk ^ (row & 7)) << 4); }

__global__ void __launch_bounds__(128, 1) oz_tc_kernel(const OzProd* __restrict__ P, const OzTile* __restrict__ tiles,
                                                       const OzPair* __restrict__ pairs, int npairs,
                                                       const CrtConst* __restrict__ cc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-out for the swizzled stages
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                                         // STAGES x 16 KB
  unsigned char* sB = smem + TC_STAGES * TC_BM * 128;               // STAGES x 16 KB
  __shared__ __align__(8) uint64_t bar_stage[TC_STAGES];
  __shared__ __align__(8) uint64_t bar_acc;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const OzTile tl = tiles[blockIdx.x];
  const OzProd p = P[tl.prod];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = p.kp / TC_BK;
  const int total = npairs * nk;
  const size_t planeA = (size_t)p.mp * p.kp, planeB = (size_t)p.np2 * p.kp;
  const __half* Abase = p.Ahat + (size_t)tl.ti * TC_BM * p.kp;
  const __half* Bbase = p.Bhat + (size_t)tl.tj * TC_BN * p.kp;

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) mbar_init(&bar_stage[s], 1);
    mbar_init(&bar_acc, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :: "r"(tc_smem_u32(&tmem_base)), "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base;

  auto load = [&](int step) {
    if (step < total) {
      const OzPair pr = pairs[step / nk];
      const int kt = step % nk, stage = step % TC_STAGES;
      const __half* a = Abase + (size_t)(pr.t - 1) * planeA + (size_t)kt * TC_BK;
      const __half* b = Bbase + (size_t)(pr.u - 1) * planeB + (size_t)kt * TC_BK;
      const uint32_t da = tc_smem_u32(sA + stage * TC_BM * 128), db = tc_smem_u32(sB + stage * TC_BN * 128);
      for (int c = tid; c < TC_BM * 8; c += 128) {
        int row = c >> 3, ch = c & 7;
        cp_async16_tc(da + sw128(row, ch), a + (size_t)row * p.kp + ch * 8);
        cp_async16_tc(db + sw128(row, ch), b + (size_t)row * p.kp + ch * 8);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  int32_t dacc[TC_BN];
#pragma unroll
  for (int j = 0; j < TC_BN; ++j) dacc[j] = 0;
  uint32_t stage_phase = 0;       // bit s: parity to wait for on bar_stage[s]
  uint32_t acc_phase = 0;
  const uint32_t idesc = instr_desc();
  bool first_of_chunk = true;

  for (int s = 0; s < TC_STAGES - 1; ++s) load(s);

  for (int step = 0; step < total; ++step) {
    const int stage = step % TC_STAGES;
    asm volatile("cp.async.wait_group %0;\n" :: "n"(TC_STAGES - 2));
    asm volatile("fence.proxy.async.shared::cta;\n" ::);     // cp.async writes -> visible to the tensor core
    __syncthreads();
    if (abort_flag) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t a0 = tc_smem_u32(sA + stage * TC_BM * 128), b0 = tc_smem_u32(sB + stage * TC_BN * 128);
#pragma unroll
      for (int k = 0; k < TC_BK / 16; ++k) {
        uint64_t ad = smem_desc(a0 + 32 * k), bd = smem_desc(b0 + 32 * k);
        uint32_t acc = (first_of_chunk && k == 0) ? 0u : 1u;
        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                   :: "r"(tc_smem_u32(&bar_stage[stage])));
    }
    first_of_chunk = false;
    // refill the buffer consumed one step earlier once its MMAs are done
    const int next = step + TC_STAGES - 1;
    if (step >= 1) {
      const int ps = (step - 1) % TC_STAGES;
      if (!mbar_wait(&bar_stage[ps], (stage_phase >> ps) & 1)) { atomicExch(err, 1); abort_flag = 1; }
      stage_phase ^= 1u << ps;
    }
    load(next);
    if (step % nk == nk - 1) {
      const OzPair pr = pairs[step / nk];
      if (pr.flags & 1) {
        if (tid == 0)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                       :: "r"(tc_smem_u32(&bar_acc)));
        if (!mbar_wait(&bar_acc, acc_phase)) { atomicExch(err, 1); abort_flag = 1; }
        acc_phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
#pragma unroll
        for (int cb = 0; cb < TC_BN; cb += 32) {
          uint32_t v[32];
          const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                       "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                       : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                         "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                         "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                         "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                       : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
          for (int j = 0; j < 32; ++j) dacc[cb + j] += __float2int_rn(__uint_as_float(v[j]));
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        first_of_chunk = true;
      }
      if (pr.flags & 2) {
        // row = tile row of this thread (TMEM lane), 128 consecutive columns
        const int r = tl.ti * TC_BM + warp * 32 + lane;
        const size_t off = (size_t)pr.level * p.mp * p.np2 + (size_t)r * p.np2 + (size_t)tl.tj * TC_BN;
        if (cc) {
          // CRT form: residues modulo the level's modulus, one byte each
          const int t = pr.level % cc->r;
          const uint32_t m = (uint32_t)cc->m[t], minv = cc->minv[t];
          uint8_t* D8 = reinterpret_cast<uint8_t*>(p.D) + off;
#pragma unroll
          for (int j = 0; j < TC_BN; j += 16) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              w[q] = crt_mod(dacc[j + 4 * q], m, minv) | (crt_mod(dacc[j + 4 * q + 1], m, minv) << 8) |
                     (crt_mod(dacc[j + 4 * q + 2], m, minv) << 16) | (crt_mod(dacc[j + 4 * q + 3], m, minv) << 24);
            *reinterpret_cast<uint4*>(D8 + j) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        } else {
          int32_t* D = p.D + off;
#pragma unroll
          for (int j = 0; j < TC_BN; j += 4)
            *reinterpret_cast<int4*>(D + j) = make_int4(dacc[j], dacc[j + 1], dacc[j + 2], dacc[j + 3]);
        }
#pragma unroll
        for (int j = 0; j < TC_BN; ++j) dacc[j] = 0;
      }
      __syncthreads();          // the accumulator is free again before the next pair's first MMA
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
  // drain: make sure no MMA is in flight before releasing tensor memory
  if (tid == 0 && total > 0 && !abort_flag) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 :: "r"(tc_smem_u32(&bar_acc)));
  }
  if (total > 0 && !abort_flag) {
    if (!mbar_wait(&bar_acc, acc_phase)) { if (tid == 0) atomicExch(err, 1); }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(TC_BN));
  }
}

size_t oz_tc_smem_bytes() { return (size_t)TC_STAGES * (TC_BM + TC_BN) * 128 + 1024; }

zkq_status launch_oz_tc(const OzProd* d_p, const OzTile* d_t, int ntiles, const OzPair* d_q, int npairs,
                        const CrtConst* d_c, int* d_err, cudaStream_t st) {
  size_t sm = oz_tc_smem_bytes();
  ZKQ_CUDA_TRY(cudaFuncSetAttribute(oz_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  oz_tc_kernel<<<ntiles, 128, sm, st>>>(d_p, d_t, d_q, npairs, d_c, d_err);
  ZKQ_CUDA_TRY(cudaGetLastError());
  return ZKQ_OK;
}

}  // namespace zkq
