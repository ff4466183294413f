// Multi-limb integer helpers of the CRT reconstruction (crt_combine_kernel in ozaki.cu), kept in a header
// of their own so that a host build can check them against exact big-integer arithmetic.
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>
#include "mw.cuh"

#if defined(__CUDACC__)
#define CL_D __device__ __forceinline__
#else
#define CL_D inline
#endif

namespace zkq {

// the most significant 32 bits of (hi:lo) << (s mod 32), and the leading zeros of a 32-bit word
CL_D uint32_t cl_funnel_l(uint32_t lo, uint32_t hi, int s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, s);
#else
  s &= 31;
  return (uint32_t)(((((uint64_t)hi << 32) | lo) << s) >> 32);
#endif
}
CL_D int cl_clz(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __clz(x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// a double from its bit pattern
CL_D double cl_bits_double(long long v) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(v);
#else
  double d;
  std::memcpy(&d, &v, sizeof d);
  return d;
#endif
}

// The reconstruction works on signed integers held as 32-bit limbs in registers.  Every limb index is a
// compile-time constant (runtime shifts go through a barrel shifter of predicated limb moves and funnel
// shifts), so no limb array is placed in local memory.

// 2^e as a double for |e| <= 1022 (exponent field), else by ldexp
CL_D double pow2i(int e) {
  return (e >= -1022 && e <= 1023) ? cl_bits_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}
// Y (M limbs) = X << sh, 0 <= sh < 32 M; bits shifted past limb M-1 are dropped
template <int M>
CL_D void limbs_shl(uint32_t* Y, int sh) {
  const int a = sh >> 5, b = sh & 31;
#pragma unroll
  for (int st = 16; st >= 1; st >>= 1) {
    if (st < M && (a & st)) {
#pragma unroll
      for (int k = M - 1; k >= 0; --k) Y[k] = k >= st ? Y[k - st] : 0u;
    }
  }
  if (a >= 32 || (M < 32 && a >= M)) {
#pragma unroll
    for (int k = 0; k < M; ++k) Y[k] = 0u;
  }
#pragma unroll
  for (int k = M - 1; k >= 1; --k) Y[k] = cl_funnel_l(Y[k - 1], Y[k], b);
  Y[0] <<= b;
}
// two's complement negation of M limbs
template <int M>
CL_D void limbs_negate(uint32_t* Y) {
  uint32_t c = 1;
#pragma unroll
  for (int k = 0; k < M; ++k) { const uint32_t v = ~Y[k] + c; c = (c && v == 0) ? 1u : 0u; Y[k] = v; }
}
// the WC leading words of the nearest-double expansion of the signed integer T (M limbs) times 2^scale:
// each word is the nearest double (ties to even) of what the words before it left.  The remainder is kept
// normalised (its top bit at bit 32 M - 1), so the 53 leading bits always sit in the two top limbs.
template <int WC, int M>
CL_D mw<WC> limbs_round_words(uint32_t* T, int scale) {
  mw<WC> out;
  bool ng = (int32_t)T[M - 1] < 0;
  if (ng) limbs_negate<M>(T);
  int shifted = 0;                               // T (normalised) = |C'| 2^shifted
#pragma unroll
  for (int w = 0; w < WC; ++w) {
    int tk = -1; uint32_t top = 0;
#pragma unroll
    for (int k = 0; k < M; ++k) if (T[k] != 0) { tk = k; top = T[k]; }
    if (tk < 0) { out.x[w] = 0.0; continue; }
    const int sh = 32 * M - 1 - (32 * tk + 31 - cl_clz(top));
    limbs_shl<M>(T, sh);
    shifted += sh;
    const uint64_t v = ((uint64_t)T[M - 1] << 32) | T[M - 2];
    uint64_t m = v >> 11;
    bool sticky = (v & 0x3FFull) != 0;
#pragma unroll
    for (int k = 0; k < M - 2; ++k) sticky |= T[k] != 0;
    const bool up = ((v >> 10) & 1) && (sticky || (m & 1));
    m += up ? 1 : 0;                             // m <= 2^53: exact as a double
    const int ev = 32 * M - 53 - shifted + scale;   // weight of m's last bit
    const double d = (ev >= -1022 && ev <= 1023) ? (double)m * pow2i(ev) : ldexp((double)m, ev);
    out.x[w] = ng ? -d : d;
    // remainder: the two top limbs become (v mod 2^11) - (up ? 2^11 : 0), sign-extended; a negative
    // remainder flips the sign of the words that follow
    const int64_t dl = (int64_t)(v & 0x7FFull) - (up ? 2048 : 0);
    T[M - 1] = (uint32_t)((uint64_t)dl >> 32); T[M - 2] = (uint32_t)(uint64_t)dl;
    if (dl < 0) { limbs_negate<M>(T); ng = !ng; }
  }
  return out;
}

}  // namespace zkq
