// Chinese-remainder form of the split product (Ozaki scheme II: Ozaki, Uchino, Imamura 2024/25).
// Rows of op(A) and columns of B are scaled by powers of two and truncated to q-bit integers A', B';
// the exact integer product C' = A' B' is formed from r products of residue matrices modulo pairwise
// coprime m_i <= 256 (entries |a| <= m_i/2 are exact in fp16, their K-sums are exact in fp32), and C' is
// reconstructed by the CRT:  C' = (sum_i c_i w_i mod M) taken symmetric,  w_i = (M/m_i) ((M/m_i)^-1 mod m_i).
// Pairwise coprime moduli <= 256 multiply to at most lcm(1..256) ~ 2^369, less than a quad-double product
// needs, so each scaled integer is split in halves, A' = A_h 2^s + A_l, and the three products
// A_h B_h, A_h B_l, A_l B_h (each below K 2^(q-2)) are reconstructed by the CRT; A_l B_l is below the
// requested accuracy and dropped.  3 r = 96-99 exact products (r = 32-33) per quad-double product instead
// of ~500 digit pairs.
#pragma once
#include <cstdint>

namespace zkq {

constexpr int CRT_MAXR = 96;     // moduli
constexpr int CRT_L = 9;         // 64-bit limbs of M and of the reconstruction sums (576 bits)
constexpr int CRT_L32 = 18;      // the same in 32-bit limbs

struct CrtConst {
  int r;                         // number of moduli
  int q;                         // bits of the scaled integers A', B' (|A'| < 2^(q-2))
  int s;                         // split: A' = A_h 2^s + A_l, 0 <= A_l < 2^s
  int m[CRT_MAXR];
  uint8_t pw16[CRT_MAXR][20];    // 2^(16 j) mod m_i, j = 0..19
  uint64_t w[CRT_MAXR][CRT_L];   // CRT weights
  uint64_t M[CRT_L];             // product of the moduli
  uint64_t Mhalf[CRT_L];         // floor(M / 2)
  double Md;                     // M as a double (upper bits), for quotient estimates
  int Mexp;                      // M = Md * 2^Mexp with Md in [1, 2)
  uint32_t w32[CRT_MAXR][CRT_L32];   // weights in 32-bit limbs
  uint32_t M32[CRT_L32];
  uint32_t Mhalf32[CRT_L32];
  uint32_t minv[CRT_MAXR];           // floor(2^32 / m_i) + 1: division-free reduction of sums < 2^29
  int l32;                           // 32-bit limbs that hold M with 16 bits of headroom (<= CRT_L32)
  int hdig;                          // 16-bit digits that hold a split half (|A_h|, A_l < 2^(16 hdig))
  int tbits;                         // bits (with sign) of the reconstructed C' = A' B', bounded by K' 2^(2q-4)
  double Mrcp;                       // 1 / Md (quotient estimates by multiplication)
};

// v mod m in [0, m) for |v| < 2^29 without division: minv = floor(2^32 / m) + 1 makes
// umulhi(|v|, minv) equal to floor(|v| / m) or one more
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t crt_mod(int v, uint32_t m, uint32_t minv) {
  const uint32_t a = (uint32_t)(v < 0 ? -v : v);
  int res = (int)(a - __umulhi(a, minv) * m);
  if (res < 0) res += (int)m;
  if (v < 0 && res) res = (int)m - res;
  return (uint32_t)res;
}
#endif

// host-side construction (moduli, weights); max_kprime decides the modulus bound
bool crt_build(int max_kprime, int p_out_bits, CrtConst* out);

}  // namespace zkq
