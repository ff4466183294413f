// Ozaki-style split products of multi-word complex matrices on tensor cores.
//
// Every row of op(A) is scaled by 2^{-e_i} and every column of B by 2^{-f_j} (powers of two, so |x| < 1/4;
// the spare bit keeps the most significant balanced digit strictly inside [-2^{b-1}, 2^{b-1}] after the
// lower digits' rounding carries),
// turned into a fixed-point integer (64-bit limbs, truncating below 2^{-b s}) and split into s balanced
// digits sigma_t in [-2^{b-1}, 2^{b-1}]:  x ~ 2^{e} sum_t sigma_t 2^{-b t}.  Then
//   op(A) B = 2^{e_i + f_j} sum_{t,u} 2^{-b(t+u)} (Ahat_t Bhat_u),
// and every digit product Ahat_t Bhat_u is an integer matrix product that fp16 tensor cores with fp32
// accumulation compute exactly while every partial sum stays below 2^24.  Pairs with t + u > S are
// dropped (their total is below the requested precision).  Pairs of the same level d = t + u are summed
// in chunks of G pairs per fp32 accumulator (G K' 2^{2(b-1)} <= 2^24), each chunk is added exactly into an
// int32 level sum D_d, and D_d (d = 2..S) are recombined exactly as one wide integer
//   I = sum_d D_d 2^{b(S-d)},  value = 2^{e_i + f_j - b S} I,
// rounded once into the output's double words.  Complex products use the real embedding
//   Re C = [Re op(A) | Im op(A)] [Re B ; -Im B],  Im C = [Re op(A) | Im op(A)] [Im B ; Re B]   (K' = 2k).
#include "ozaki.cuh"
#include "oz_tc.cuh"
#include "crt.cuh"
#include "crt_limbs.cuh"
#include "mw.cuh"
#include "prof.cuh"
#include "internal.cuh"
#include <vector>
#include <mutex>
#include <algorithm>
#include <cstring>

namespace zkq {

// ------------------------------------------------------------------------------------------------
// 320-bit two's complement integers in five 64-bit limbs (little endian)
struct Big { uint64_t l[5]; };

__device__ __forceinline__ void big_zero(Big& x) { for (int i = 0; i < 5; ++i) x.l[i] = 0; }
__device__ __forceinline__ bool big_neg(const Big& x) { return (int64_t)x.l[4] < 0; }
__device__ __forceinline__ void big_negate(Big& x) {
  uint64_t c = 1;
  for (int i = 0; i < 5; ++i) { uint64_t v = ~x.l[i] + c; c = (c && v == 0) ? 1 : 0; x.l[i] = v; }
}
// Y <<= sh (0 <= sh < 512; bits past 320 are dropped).  Runtime shifts go through predicated limb moves
// and funnel shifts, so every limb index is a compile-time constant and Big stays in registers.
__device__ __forceinline__ void big_shl(Big& Y, int sh) {
  const int a = sh >> 6, b = sh & 63;
#pragma unroll
  for (int st = 4; st >= 1; st >>= 1) {
    if (a & st) {
#pragma unroll
      for (int k = 4; k >= 0; --k) Y.l[k] = k >= st ? Y.l[k - st] : 0ULL;
    }
  }
  if (b) {
#pragma unroll
    for (int k = 4; k >= 1; --k) Y.l[k] = (Y.l[k] << b) | (Y.l[k - 1] >> (64 - b));
    Y.l[0] <<= b;
  }
}
// arithmetic shift right by 0 <= sh < 320 bits
__device__ __forceinline__ void big_sar_var(Big& Y, int sh) {
  const uint64_t fill = (int64_t)Y.l[4] < 0 ? ~0ULL : 0ULL;
  const int a = sh >> 6, b = sh & 63;
#pragma unroll
  for (int st = 4; st >= 1; st >>= 1) {
    if (a & st) {
#pragma unroll
      for (int k = 0; k < 5; ++k) Y.l[k] = k + st <= 4 ? Y.l[k + st] : fill;
    }
  }
  if (b) {
#pragma unroll
    for (int k = 0; k < 4; ++k) Y.l[k] = (Y.l[k] >> b) | (Y.l[k + 1] << (64 - b));
    Y.l[4] = (uint64_t)((int64_t)Y.l[4] >> b);
  }
}
// x += (neg ? -1 : 1) * m * 2^shift   (0 <= shift < 320; the part of m 2^shift past bit 320 is dropped)
__device__ __forceinline__ void big_add_shifted(Big& x, uint64_t m, int shift, bool neg) {
  if (m == 0 || shift >= 320) return;
  Big wb = {{m, 0, 0, 0, 0}};
  big_shl(wb, shift);
  const uint64_t* w = wb.l;
  if (!neg) {
    uint64_t c = 0;
    for (int i = 0; i < 5; ++i) { uint64_t a = x.l[i], t = a + w[i]; uint64_t c1 = t < a; uint64_t t2 = t + c; c = c1 | (t2 < t); x.l[i] = t2; }
  } else {
    uint64_t br = 0;
    for (int i = 0; i < 5; ++i) { uint64_t a = x.l[i], t = a - w[i]; uint64_t b1 = a < w[i]; uint64_t t2 = t - br; br = b1 | (t < br); x.l[i] = t2; }
  }
}
// x += v * 2^shift for a signed 64-bit v
__device__ __forceinline__ void big_add_signed(Big& x, int64_t v, int shift) {
  if (v >= 0) big_add_shifted(x, (uint64_t)v, shift, false);
  else big_add_shifted(x, (uint64_t)(-v), shift, true);
}
// arithmetic shift right by s (< 64) bits
__device__ __forceinline__ void big_sar(Big& x, int s) {
  for (int i = 0; i < 4; ++i) x.l[i] = (x.l[i] >> s) | (x.l[i + 1] << (64 - s));
  x.l[4] = (uint64_t)((int64_t)x.l[4] >> s);
}
__device__ __forceinline__ int big_top_bit(const Big& x) {
  for (int i = 4; i >= 0; --i) if (x.l[i]) return 64 * i + 63 - __clzll(x.l[i]);
  return -1;
}
__device__ __forceinline__ int big_bit(const Big& x, int i) { return i < 0 ? 0 : (int)((x.l[i >> 6] >> (i & 63)) & 1); }

// decompose a finite double: |x| = m 2^q, m < 2^53
__device__ __forceinline__ void dsplit(double x, uint64_t& m, int& q, bool& neg) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  neg = (b >> 63) != 0;
  int be = (int)((b >> 52) & 0x7FF);
  uint64_t f = b & 0xFFFFFFFFFFFFFULL;
  if (be == 0) { m = f; q = -1074; } else { m = f | (1ULL << 52); q = be - 1075; }
}

// fixed point: X = trunc(x * 2^{fix}) summed word by word (each word truncated toward zero)
template <int K>
__device__ __forceinline__ void to_fixed(const double* w, int fix, bool negate, Big& X) {
  big_zero(X);
  for (int k = 0; k < K; ++k) {
    double v = w[k];
    if (v == 0.0) continue;
    uint64_t m; int q; bool ng; dsplit(v, m, q, ng);
    int sh = q + fix;
    if (sh < 0) { if (-sh >= 64) continue; m >>= -sh; sh = 0; }
    if (sh > 256) continue;              // cannot happen for scaled inputs (|x 2^-e| < 1/4)
    big_add_shifted(X, m, sh, ng != negate);
  }
}

// s balanced base-2^b digits of X (|X| < 2^{b s - 2}); digit t (1-based, most significant first).
// Lower digits lie in (-2^{b-1}, 2^{b-1}]; what remains for the top digit has |.| <= 2^{b-2} + 1.
template <typename F>
__device__ __forceinline__ void digits(Big X, int b, int s, F&& emit) {
  const int64_t half = 1LL << (b - 1), base = 1LL << b;
  for (int t = s; t >= 1; --t) {
    int64_t d = (int64_t)(X.l[0] & (uint64_t)(base - 1));
    if (d > half) d -= base;
    big_add_signed(X, -d, 0);
    big_sar(X, b);
    emit(t, (int)d);
  }
}

// round the signed big integer R to the nearest double times 2^scale, subtract that double from R
__device__ double big_round_off(Big& R, int scale) {
  bool ng = big_neg(R);
  Big M = R; if (ng) big_negate(M);
  int tb = big_top_bit(M);
  if (tb < 0) return 0.0;
  int lo = tb - 52;
  uint64_t m = 0;
  if (lo >= 0) {
    int li = lo >> 6, bs = lo & 63;
    m = M.l[li] >> bs;
    if (bs && li + 1 < 5) m |= M.l[li + 1] << (64 - bs);
    m &= (1ULL << 53) - 1;
    int rnd = big_bit(M, lo - 1);
    bool sticky = false;
    for (int i = 0; i < ((lo - 1) >> 6) && !sticky; ++i) sticky = M.l[i] != 0;
    if (!sticky && lo - 1 > 0) {
      int li2 = (lo - 1) >> 6, b2 = (lo - 1) & 63;
      sticky = (M.l[li2] & ((1ULL << b2) - 1)) != 0;
    }
    if (rnd && (sticky || (m & 1))) m += 1;
  } else {
    m = M.l[0];                          // fewer than 53 significant bits: exact
    lo = 0;
  }
  // R -= sign * m * 2^lo
  big_add_shifted(R, m, lo, !ng);
  double v = ldexp((double)m, lo + scale);
  return ng ? -v : v;
}

// ------------------------------------------------------------------------------------------------
OzPlan ozaki_plan(int max_kprime, int wa, int wb, int p_out_bits) {
  OzPlan p;
  p.b = max_kprime <= 1024 ? 8 : 7;
  int lg = 0; while ((1 << lg) < max_kprime) ++lg;
  // Digits are counted from each row's / column's power-of-two scale, not per element: an entry far below
  // its row maximum has significant bits far below the scale, so the count follows the requested accuracy
  // whatever the number of input words.
  auto need = [&](int words) {
    (void)words;
    int bits = p_out_bits + 3 + lg;
    return (bits + p.b - 1) / p.b + 1;
  };
  p.sA = need(wa);
  p.sB = need(wb);
  p.S = std::min(p.sA + p.sB, (p_out_bits + 2 * (p.b - 1) + lg + 8 + p.b - 1) / p.b + 1);
  long long cap = (1LL << 24) / ((long long)max_kprime << (2 * (p.b - 1)));
  p.G = (int)std::max(1LL, cap);
  p.npairs = 0;
  return p;
}

static std::vector<OzPair> make_pairs(const OzPlan& p) {
  std::vector<OzPair> v;
  for (int d = 2; d <= p.S; ++d) {
    int cnt = 0;
    int first = (int)v.size();
    for (int t = std::max(1, d - p.sB); t <= std::min(p.sA, d - 1); ++t) {
      OzPair q; q.t = (int16_t)t; q.u = (int16_t)(d - t); q.level = (int16_t)d; q.flags = 0;
      v.push_back(q);
      if (++cnt == p.G) { v.back().flags |= 1; cnt = 0; }
    }
    if ((int)v.size() > first) v.back().flags |= 3;
  }
  return v;
}

// ------------------------------------------------------------------------------------------------
// exponents: rows of op(A), columns of B
template <int WA, int WB>
__global__ void oz_scale_kernel(const OzProd* __restrict__ P) {
  const OzProd p = P[blockIdx.y];
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < p.m) {
    if (!p.sliceA) return;
    double mx = 0.0;
    for (int l = 0; l < p.k; ++l) {
      const double* q = p.opA ? p.A + ((size_t)l + (size_t)r * p.k) * 2 * WA : p.A + ((size_t)r + (size_t)l * p.m) * 2 * WA;
      mx = fmax(mx, fmax(fabs(q[0]), fabs(q[WA])));
    }
    p.eA[r] = mx > 0 ? ilogb(mx) + 3 : 0;
  } else if (r < p.m + p.n) {
    if (!p.sliceB) return;
    int j = r - p.m;
    double mx = 0.0;
    for (int l = 0; l < p.k; ++l) {
      const double* q = p.B + ((size_t)l + (size_t)j * p.k) * 2 * WB;
      mx = fmax(mx, fmax(fabs(q[0]), fabs(q[WB])));
    }
    p.eB[j] = mx > 0 ? ilogb(mx) + 3 : 0;
  }
}

template <int WA>
__global__ void oz_slice_A_kernel(const OzProd* __restrict__ P, int b, int sA) {
  const OzProd p = P[blockIdx.y];
  if (!p.sliceA) return;
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)p.mp * p.kp;
  if (e >= tot) return;
  int i = (int)(e / p.kp), lp = (int)(e % p.kp);
  const size_t plane = (size_t)p.mp * p.kp;
  if (i >= p.m || lp >= 2 * p.k) {
    for (int t = 0; t < sA; ++t) p.Ahat[t * plane + e] = __float2half_rn(0.0f);
    return;
  }
  bool im = lp >= p.k;
  int l = im ? lp - p.k : lp;
  const double* q = p.opA ? p.A + ((size_t)l + (size_t)i * p.k) * 2 * WA : p.A + ((size_t)i + (size_t)l * p.m) * 2 * WA;
  bool negate = im && p.opA;             // conj for A^H
  Big X; to_fixed<WA>(q + (im ? WA : 0), b * sA - p.eA[i], negate, X);
  digits(X, b, sA, [&](int t, int d) { p.Ahat[(size_t)(t - 1) * plane + e] = __int2half_rn(d); });
}

template <int WB>
__global__ void oz_slice_B_kernel(const OzProd* __restrict__ P, int b, int sB) {
  const OzProd p = P[blockIdx.y];
  if (!p.sliceB) return;
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)p.np2 * p.kp;
  if (e >= tot) return;
  int jp = (int)(e / p.kp), lp = (int)(e % p.kp);
  const size_t plane = (size_t)p.np2 * p.kp;
  if (jp >= 2 * p.n || lp >= 2 * p.k) {
    for (int t = 0; t < sB; ++t) p.Bhat[t * plane + e] = __float2half_rn(0.0f);
    return;
  }
  bool imcol = jp >= p.n;
  int j = imcol ? jp - p.n : jp;
  bool lower = lp >= p.k;
  int l = lower ? lp - p.k : lp;
  // re column: [Re B; -Im B];  im column: [Im B; Re B]
  bool use_im = imcol ? !lower : lower;
  bool negate = !imcol && lower;
  const double* q = p.B + ((size_t)l + (size_t)j * p.k) * 2 * WB + (use_im ? WB : 0);
  Big X; to_fixed<WB>(q, b * sB - p.eB[j], negate, X);
  digits(X, b, sB, [&](int t, int d) { p.Bhat[(size_t)(t - 1) * plane + e] = __int2half_rn(d); });
}

// ------------------------------------------------------------------------------------------------
// slice GEMM: fp16 x fp16 -> fp32 (exact), mma.sync m16n8k16, CTA tile 128 x 128 x 32, 8 warps (2 x 4)
constexpr int OZ_BM = 128, OZ_BN = 128, OZ_BK = 32, OZ_STAGES = 3;


// slice-GEMM kernel: 0 mma.sync (legacy warp-level path), 1 tcgen05 (tensor memory accumulators)
static int g_gemm_kernel = 1;
// Tile-width table of the tcgen05 slice GEMM (zkq_autotune_gemm): (largest K' of a batch, 1 for 256-column
// tiles / 0 for 128-column tiles), by increasing K'; a batch takes the first entry whose K' is >= its own,
// else the last; empty: 256-column tiles wherever they fit.  Both widths compute the same exact integer
// slice products, so the choice changes no result.  Process-wide, like the kernel choice.
static std::mutex g_wide_mu;
static std::vector<std::pair<int, int>> g_wide_table;
static bool wide_tiles_for(int max_kp) {
  std::lock_guard<std::mutex> g(g_wide_mu);
  if (g_wide_table.empty()) return true;
  for (const auto& e : g_wide_table) if (e.first >= max_kp) return e.second != 0;
  return g_wide_table.back().second != 0;
}
// SM count of the current device (cached per device)
static int device_sm_count() {
  static std::mutex mu;
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> g(mu);
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cache[dev] = v;
  }
  return cache[dev];
}
void gemm_wide_table_set(const std::vector<std::pair<int, int>>& t) {
  std::lock_guard<std::mutex> g(g_wide_mu);
  g_wide_table = t;
  std::sort(g_wide_table.begin(), g_wide_table.end());
}
std::vector<std::pair<int, int>> gemm_wide_table_get() {
  std::lock_guard<std::mutex> g(g_wide_mu);
  return g_wide_table;
}
static int* g_oz_err = nullptr;              // device flag raised by a bounded wait that expired

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" :: "r"(dst), "l"(src));
}
__device__ __forceinline__ int swz(int row, int chunk) { return row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4); }

__global__ void __launch_bounds__(256) oz_gemm_kernel(const OzProd* __restrict__ P, const OzTile* __restrict__ tiles,
                                                      const OzPair* __restrict__ pairs, int npairs, int S,
                                                      const CrtConst* __restrict__ cc) {
  extern __shared__ __align__(128) unsigned char smem[];
  const OzTile tl = tiles[blockIdx.x];
  const OzProd p = P[tl.prod];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;
  const int nk = p.kp / OZ_BK;
  const int total = npairs * nk;
  const size_t planeA = (size_t)p.mp * p.kp, planeB = (size_t)p.np2 * p.kp;
  const __half* Abase = p.Ahat + (size_t)tl.ti * OZ_BM * p.kp;
  const __half* Bbase = p.Bhat + (size_t)tl.tj * OZ_BN * p.kp;
  unsigned char* sA = smem;                                   // STAGES x 8 KB
  unsigned char* sB = smem + OZ_STAGES * OZ_BM * 64;          // STAGES x 8 KB

  auto load = [&](int step, int stage) {
    if (step < total) {
      const OzPair pr = pairs[step / nk];
      const int kt = step % nk;
      const __half* a = Abase + (size_t)(pr.t - 1) * planeA + kt * OZ_BK;
      const __half* bb = Bbase + (size_t)(pr.u - 1) * planeB + kt * OZ_BK;
      for (int c = tid; c < OZ_BM * 4; c += 256) {
        int row = c >> 2, ch = c & 3;
        cp_async16(smem_u32(sA + stage * OZ_BM * 64 + swz(row, ch)), a + (size_t)row * p.kp + ch * 8);
        cp_async16(smem_u32(sB + stage * OZ_BN * 64 + swz(row, ch)), bb + (size_t)row * p.kp + ch * 8);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  float acc[4][4][4];
  int32_t dacc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2)
#pragma unroll
      for (int c = 0; c < 4; ++c) { acc[a][b2][c] = 0.f; dacc[a][b2][c] = 0; }

  for (int s = 0; s < OZ_STAGES - 1; ++s) load(s, s);

  for (int step = 0; step < total; ++step) {
    asm volatile("cp.async.wait_group %0;\n" :: "n"(OZ_STAGES - 2));
    __syncthreads();
    load(step + OZ_STAGES - 1, (step + OZ_STAGES - 1) % OZ_STAGES);
    const int stage = step % OZ_STAGES;
    const unsigned char* As = sA + stage * OZ_BM * 64;
    const unsigned char* Bs = sB + stage * OZ_BN * 64;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        int row = wm * 64 + mi * 16 + (lane & 15);
        int ch = kk * 2 + (lane >> 4);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(af[mi][0]), "=r"(af[mi][1]), "=r"(af[mi][2]), "=r"(af[mi][3])
                     : "r"(smem_u32(As + swz(row, ch))));
      }
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        int row = wn * 32 + nj * 16 + (lane & 7) + ((lane >> 4) << 3);
        int ch = kk * 2 + ((lane >> 3) & 1);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(bf[2 * nj][0]), "=r"(bf[2 * nj][1]), "=r"(bf[2 * nj + 1][0]), "=r"(bf[2 * nj + 1][1])
                     : "r"(smem_u32(Bs + swz(row, ch))));
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                       : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
                       : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bf[ni][0]), "r"(bf[ni][1]));
    }
    if (step % nk == nk - 1) {
      const OzPair pr = pairs[step / nk];
      if (pr.flags & 1) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2)
#pragma unroll
            for (int c = 0; c < 4; ++c) { dacc[a][b2][c] += __float2int_rn(acc[a][b2][c]); acc[a][b2][c] = 0.f; }
      }
      if (pr.flags & 2) {
        const size_t po = (size_t)pr.level * p.mp * p.np2;
        uint32_t m = 0, minv = 0;
        if (cc) { const int t = pr.level % cc->r; m = (uint32_t)cc->m[t]; minv = cc->minv[t]; }
#pragma unroll
        for (int mi = 0; mi < 4; ++mi)
#pragma unroll
          for (int ni = 0; ni < 4; ++ni) {
            int r = tl.ti * OZ_BM + wm * 64 + mi * 16 + (lane >> 2);
            int c = tl.tj * OZ_BN + wn * 32 + ni * 8 + (lane & 3) * 2;
            if (cc) {                            // CRT form: residues, one byte each
              uint8_t* D8 = reinterpret_cast<uint8_t*>(p.D) + po;
              *reinterpret_cast<uchar2*>(D8 + (size_t)r * p.np2 + c) =
                  make_uchar2((uint8_t)crt_mod(dacc[mi][ni][0], m, minv), (uint8_t)crt_mod(dacc[mi][ni][1], m, minv));
              *reinterpret_cast<uchar2*>(D8 + (size_t)(r + 8) * p.np2 + c) =
                  make_uchar2((uint8_t)crt_mod(dacc[mi][ni][2], m, minv), (uint8_t)crt_mod(dacc[mi][ni][3], m, minv));
            } else {
              int32_t* D = p.D + po;
              *reinterpret_cast<int2*>(D + (size_t)r * p.np2 + c) = make_int2(dacc[mi][ni][0], dacc[mi][ni][1]);
              *reinterpret_cast<int2*>(D + (size_t)(r + 8) * p.np2 + c) = make_int2(dacc[mi][ni][2], dacc[mi][ni][3]);
            }
            dacc[mi][ni][0] = dacc[mi][ni][1] = dacc[mi][ni][2] = dacc[mi][ni][3] = 0;
          }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// ------------------------------------------------------------------------------------------------
template <int WC>
__device__ __forceinline__ mw<WC> combine_value(const OzProd& p, int i, int col, int e_sum, int b, int S) {
  Big I; big_zero(I);
  for (int d = 2; d <= S; ++d) {
    int32_t v = p.D[(size_t)d * p.mp * p.np2 + (size_t)i * p.np2 + col];
    big_add_signed(I, (int64_t)v, b * (S - d));
  }
  mw<WC> r;
  for (int k = 0; k < WC; ++k) r.x[k] = big_round_off(I, e_sum - b * S);
  return r;
}

template <int WC>
__global__ void oz_combine_kernel(const OzProd* __restrict__ P, int b, int S) {
  const OzProd p = P[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.m * p.n) return;
  const int j = t % p.n, i = t / p.n;          // columns fastest: the planes are row-major [i][col]
  const size_t e = (size_t)i + (size_t)j * p.m;
  if (p.hermitian && i > j) return;
  int es = p.eA[i] + p.eB[j];
  cmw<WC> v = c_make(combine_value<WC>(p, i, j, es, b, S), combine_value<WC>(p, i, j + p.n, es, b, S));
  if (p.sgn < 0) v = c_make(mw_neg(v.re), mw_neg(v.im));
  if (p.base) v = c_add(v, c_load<WC, WC>(p.base, (size_t)e));
  if (p.base_identity && i == j) v.re = mw_add_d(v.re, 1.0);
  if (p.hermitian && i == j) v.im = mw_zero<WC>();
  c_store(p.C, (size_t)e, v);
  if (p.hermitian && i < j) c_store(p.C, (size_t)j + (size_t)i * p.m, c_conj(v));
}

// ------------------------------------------------------------------------------------------------
// CRT form: residue planes and reconstruction
// Residue planes of the CRT form.  X (q-bit scaled integer of one operand entry) = A_h 2^s + A_l with
// 0 <= A_l < 2^s; the symmetric residues of A_h and A_l modulo every m_i are written as fp16 planes
// [i][rows][kp] and [r + i][rows][kp].  A half below 2^(16 HD) is a sum of HD 16-bit digits d_j, and
// A mod m = sum_j d_j (2^(16 j) mod m) mod m with the digit sum below 2^29.
struct CrtHalves { uint32_t dh[20], dl[20]; bool nh; };

template <int HD>
__device__ __forceinline__ void crt_halves(const Big& X, int s, CrtHalves& o) {
  Big lo = X;                                  // low s bits (two's complement residue, nonnegative)
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    int b0 = 64 * i;
    if (b0 >= s) lo.l[i] = 0;
    else if (b0 + 64 > s) lo.l[i] &= (s - b0 == 64) ? ~0ULL : ((1ULL << (s - b0)) - 1);
  }
  Big hi = X;                                  // floor(X / 2^s): arithmetic shift
  big_sar_var(hi, s);
  o.nh = big_neg(hi);
  if (o.nh) big_negate(hi);
#pragma unroll
  for (int j = 0; j < HD; ++j) {
    o.dh[j] = (uint32_t)((hi.l[j >> 2] >> (16 * (j & 3))) & 0xFFFF);
    o.dl[j] = (uint32_t)((lo.l[j >> 2] >> (16 * (j & 3))) & 0xFFFF);
  }
}

// symmetric residue of sign * (digit sum) modulo m as fp16
__device__ __forceinline__ __half crt_sym(uint32_t sum, bool neg, uint32_t m, uint32_t minv) {
  int res = (int)(sum - __umulhi(sum, minv) * m);
  if (res < 0) res += (int)m;
  if (neg && res) res = (int)m - res;
  if (res > (int)(m >> 1)) res -= (int)m;
  return __int2half_rn(res);
}

// per-modulus constants in shared memory: [m, minv, pw_0 .. pw_{HD-1}] for every modulus
template <int HD>
__device__ __forceinline__ void crt_stage_consts(const CrtConst* __restrict__ cc, uint32_t* sc) {
  const int r = cc->r;
  for (int x = threadIdx.x; x < r * (HD + 2); x += blockDim.x) {
    const int i = x / (HD + 2), k = x % (HD + 2);
    sc[x] = k == 0 ? (uint32_t)cc->m[i] : (k == 1 ? cc->minv[i] : (uint32_t)cc->pw16[i][k - 2]);
  }
  __syncthreads();
}

// residues of two neighbouring entries (e0, e0 + 1 of every plane) from their halves
template <int HD>
__device__ __forceinline__ void crt_emit2(const CrtHalves& a, const CrtHalves& b, int r, const uint32_t* sc,
                                          __half* out, size_t plane, size_t e0) {
  for (int i = 0; i < r; ++i) {
    const uint32_t* c = sc + i * (HD + 2);
    const uint32_t m = c[0], minv = c[1];
    uint32_t ha = 0, la = 0, hb = 0, lb = 0;
#pragma unroll
    for (int j = 0; j < HD; ++j) {
      const uint32_t pw = c[2 + j];
      ha += a.dh[j] * pw; la += a.dl[j] * pw; hb += b.dh[j] * pw; lb += b.dl[j] * pw;
    }
    *reinterpret_cast<__half2*>(out + (size_t)i * plane + e0) =
        __halves2half2(crt_sym(ha, a.nh, m, minv), crt_sym(hb, b.nh, m, minv));
    *reinterpret_cast<__half2*>(out + (size_t)(r + i) * plane + e0) =
        __halves2half2(crt_sym(la, false, m, minv), crt_sym(lb, false, m, minv));
  }
}

// A planes: two neighbouring K' entries of one row of op(A) per thread (kp is even)
template <int WA, int HD>
__global__ void crt_slice_A_kernel(const OzProd* __restrict__ P, const CrtConst* __restrict__ cc) {
  __shared__ uint32_t sc[CRT_MAXR * (HD + 2)];
  const OzProd p = P[blockIdx.y];
  if (!p.sliceA) return;
  crt_stage_consts<HD>(cc, sc);
  const size_t e0 = 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  const size_t tot = (size_t)p.mp * p.kp;
  if (e0 >= tot) return;
  const int i = (int)(e0 / p.kp), lp = (int)(e0 % p.kp);
  const int r = cc->r;
  if (i >= p.m || lp >= 2 * p.k) {
    for (int t = 0; t < 2 * r; ++t) *reinterpret_cast<__half2*>(p.Ahat + t * tot + e0) = __float2half2_rn(0.0f);
    return;
  }
  CrtHalves h[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const bool im = lp + u >= p.k;
    const int l = im ? lp + u - p.k : lp + u;
    const double* q = p.opA ? p.A + ((size_t)l + (size_t)i * p.k) * 2 * WA : p.A + ((size_t)i + (size_t)l * p.m) * 2 * WA;
    Big X; to_fixed<WA>(q + (im ? WA : 0), cc->q - p.eA[i], im && p.opA, X);
    crt_halves<HD>(X, cc->s, h[u]);
  }
  crt_emit2<HD>(h[0], h[1], r, sc, p.Ahat, tot, e0);
}

// B planes: column j' of [Re | Im] output, rows [Re; Im] of K' (real embedding of the complex product)
template <int WB, int HD>
__global__ void __launch_bounds__(256, 4) crt_slice_B_kernel(const OzProd* __restrict__ P, const CrtConst* __restrict__ cc) {
  __shared__ uint32_t sc[CRT_MAXR * (HD + 2)];
  const OzProd p = P[blockIdx.y];
  if (!p.sliceB) return;
  crt_stage_consts<HD>(cc, sc);
  const size_t e0 = 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  const size_t tot = (size_t)p.np2 * p.kp;
  if (e0 >= tot) return;
  const int jp = (int)(e0 / p.kp), lp = (int)(e0 % p.kp);
  const int r = cc->r;
  if (jp >= 2 * p.n || lp >= 2 * p.k) {
    for (int t = 0; t < 2 * r; ++t) *reinterpret_cast<__half2*>(p.Bhat + t * tot + e0) = __float2half2_rn(0.0f);
    return;
  }
  const bool imcol = jp >= p.n;
  const int j = imcol ? jp - p.n : jp;
  CrtHalves h[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const bool lower = lp + u >= p.k;
    const int l = lower ? lp + u - p.k : lp + u;
    const bool use_im = imcol ? !lower : lower;
    const bool negate = !imcol && lower;
    const double* q = p.B + ((size_t)l + (size_t)j * p.k) * 2 * WB + (use_im ? WB : 0);
    Big X; to_fixed<WB>(q, cc->q - p.eB[j], negate, X);
    crt_halves<HD>(X, cc->s, h[u]);
  }
  crt_emit2<HD>(h[0], h[1], r, sc, p.Bhat, tot, e0);
}

// symmetric (sum_i c_i w_i mod M) from residues c_i; 32-bit limbs with 64-bit lazy accumulators (every
// product c w_limb < 2^40, at most 96 of them per limb), one carry pass at the end.
// out: signed two's complement, CRT_L32 + 2 limbs.
// residue(t) yields c_t in [0, m_t).
template <int LW, typename Res>   // LW: 32-bit limbs of M (>= cc->l32); the output has LW + 2 limbs
__device__ __forceinline__ void crt_sum32(Res&& residue, const CrtConst* __restrict__ cc, uint32_t* out) {
  constexpr int L = LW + 2;
  constexpr int CRT_L32 = LW;
  uint64_t acc[CRT_L32];
#pragma unroll
  for (int k = 0; k < CRT_L32; ++k) acc[k] = 0;
  const int r = cc->r;
  for (int t = 0; t < r; ++t) {
    const uint64_t ct = (uint64_t)residue(t);
    const uint32_t* w = cc->w32[t];
#pragma unroll
    for (int k = 0; k < CRT_L32; ++k) acc[k] += ct * w[k];
  }
  uint32_t S[L];
  uint64_t carry = 0;
#pragma unroll
  for (int k = 0; k < CRT_L32; ++k) { uint64_t v = acc[k] + carry; S[k] = (uint32_t)v; carry = v >> 32; }
  S[CRT_L32] = (uint32_t)carry; S[CRT_L32 + 1] = (uint32_t)(carry >> 32);
  // quotient estimate q = floor(S / M) (< 2^15) from the leading bits, exact correction after
  int top = 0; uint32_t s0 = S[0], s1 = 0, s2 = 0;
#pragma unroll
  for (int k = 1; k < L; ++k) if (S[k] != 0) { top = k; s0 = S[k]; s1 = S[k - 1]; s2 = k > 1 ? S[k - 2] : 0u; }
  double sd = (double)s0 + (double)s1 * 0x1p-32 + (double)s2 * 0x1p-64;
  const int qe = 32 * top - cc->Mexp;            // S / M ~ sd Mrcp 2^qe
  double qd = qe < -60 ? 0.0 : (qe > 60 ? 1e30 : sd * cc->Mrcp * pow2i(qe));
  int64_t qq = qd > 1.0 ? (int64_t)fmin(qd, 1e18) : 0;
  // S -= q M (signed 64-bit lazy borrow)
  {
    int64_t b = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) {
      int64_t v = (int64_t)S[k] - (k < CRT_L32 ? (int64_t)((uint64_t)qq * cc->M32[k] & 0xFFFFFFFFULL) : 0) + b;
      int64_t hi = k < CRT_L32 ? (int64_t)(((uint64_t)qq * cc->M32[k]) >> 32) : 0;
      S[k] = (uint32_t)v;
      b = (v >> 32) - hi;                       // arithmetic shift keeps the borrow
    }
  }
  auto neg = [&]() { return (int32_t)S[L - 1] < 0; };
  auto addM = [&](int sgn) {
    int64_t cy = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) {
      int64_t v = (int64_t)S[k] + (k < CRT_L32 ? sgn * (int64_t)cc->M32[k] : 0) + cy;
      S[k] = (uint32_t)v; cy = v >> 32;
    }
  };
  auto cmp = [&](const uint32_t* X) {           // sign of S - X for nonnegative S (the highest differing limb)
    int c = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) {
      const uint32_t x = k < CRT_L32 ? X[k] : 0u;
      if (S[k] != x) c = S[k] > x ? 1 : -1;
    }
    return c;
  };
  auto geq = [&](const uint32_t* X) { return cmp(X) >= 0; };
  for (int it = 0; it < 3 && neg(); ++it) addM(1);
  for (int it = 0; it < 3 && geq(cc->M32); ++it) addM(-1);
  auto gt = [&](const uint32_t* X) { return cmp(X) > 0; };
  if (!neg() && gt(cc->Mhalf32)) addM(-1);      // symmetric representative
#pragma unroll
  for (int k = 0; k < L; ++k) out[k] = S[k];
}

// C' = C_hh 2^(2s) + (C_hl + C_lh) 2^s, value = C' 2^(e_i + f_j - 2q); LT 64-bit limbs hold C' (tbits)
template <int WC, int LW, int LT>
__device__ __forceinline__ mw<WC> crt_value(const OzProd& p, const CrtConst* __restrict__ cc, int i, int col, int es) {
  constexpr int L32 = LW + 2;
  const int r = cc->r, s = cc->s;
  const size_t stride = (size_t)p.mp * p.np2;
  const uint8_t* D8 = reinterpret_cast<const uint8_t*>(p.D) + (size_t)i * p.np2 + col;   // residues in [0, m_t)
  uint32_t hh[L32], sm[L32];
  crt_sum32<LW>([&](int t) { return (int)__ldg(D8 + (size_t)t * stride); }, cc, hh);
  crt_sum32<LW>([&](int t) {
    const int v = (int)__ldg(D8 + (size_t)(r + t) * stride) + (int)__ldg(D8 + (size_t)(2 * r + t) * stride);
    return v >= cc->m[t] ? v - cc->m[t] : v;
  }, cc, sm);
  // C' = hh 2^(2s) + sm 2^s in M = 2 LT 32-bit limbs (two's complement; both shifted values fit, by tbits)
  constexpr int M = 2 * LT;
  uint32_t T[M], U[M];
  const uint32_t fh = (int32_t)hh[L32 - 1] < 0 ? ~0u : 0u, fs = (int32_t)sm[L32 - 1] < 0 ? ~0u : 0u;
#pragma unroll
  for (int k = 0; k < M; ++k) { T[k] = k < L32 ? hh[k] : fh; U[k] = k < L32 ? sm[k] : fs; }
  limbs_shl<M>(T, 2 * s);
  limbs_shl<M>(U, s);
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const uint64_t v = (uint64_t)T[k] + U[k] + c;
    T[k] = (uint32_t)v; c = (uint32_t)(v >> 32);
  }
  return limbs_round_words<WC, M>(T, es - 2 * cc->q);
}

template <int WC, int LW, int LT>
__global__ void __launch_bounds__(128, (LW <= 9 ? 8 : 4)) crt_combine_kernel(const OzProd* __restrict__ P, const CrtConst* __restrict__ cc) {
  const OzProd p = P[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.m * p.n) return;
  const int j = t % p.n, i = t / p.n;          // columns fastest: the planes are row-major [i][col]
  const size_t e = (size_t)i + (size_t)j * p.m;
  if (p.hermitian && i > j) return;            // written by the (j, i) thread
  int es = p.eA[i] + p.eB[j];
  cmw<WC> v = c_make(crt_value<WC, LW, LT>(p, cc, i, j, es), crt_value<WC, LW, LT>(p, cc, i, j + p.n, es));
  if (p.sgn < 0) v = c_make(mw_neg(v.re), mw_neg(v.im));
  if (p.base) v = c_add(v, c_load<WC, WC>(p.base, (size_t)e));
  if (p.base_identity && i == j) v.re = mw_add_d(v.re, 1.0);
  if (p.hermitian && i == j) v.im = mw_zero<WC>();
  c_store(p.C, (size_t)e, v);
  if (p.hermitian && i < j) c_store(p.C, (size_t)j + (size_t)i * p.m, c_conj(v));
}

// ------------------------------------------------------------------------------------------------
// plain multi-word GEMM on the FP64 pipe (one output element per thread)
template <int WA, int WB, int WC>
__global__ void mw_gemm_plain_kernel(const OzProd* __restrict__ P) {
  const OzProd p = P[blockIdx.y];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.m * p.n) return;
  int i = e % p.m, j = e / p.m;
  cmw<WC> s = c_zero<WC>();
  for (int l = 0; l < p.k; ++l) {
    cmw<WC> a = p.opA ? c_conj(c_load<WC, WA>(p.A, (size_t)l + (size_t)i * p.k)) : c_load<WC, WA>(p.A, (size_t)i + (size_t)l * p.m);
    cmw<WC> bb = c_load<WC, WB>(p.B, (size_t)l + (size_t)j * p.k);
    s = c_add(s, c_mul(a, bb));
  }
  if (p.sgn < 0) s = c_make(mw_neg(s.re), mw_neg(s.im));
  if (p.base) s = c_add(s, c_load<WC, WC>(p.base, (size_t)e));
  if (p.base_identity && i == j) s.re = mw_add_d(s.re, 1.0);
  c_store(p.C, (size_t)e, s);
}

// ------------------------------------------------------------------------------------------------
static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static zkq_status grow(void** p, size_t* have, size_t need) {
  if (need <= *have) return ZKQ_OK;
  if (*p) { cudaFree(*p); *p = nullptr; *have = 0; }
  size_t want = std::max(need + need / 4, (size_t)1 << 20);
  cudaError_t e = cudaMalloc(p, want);
  if (e != cudaSuccess) { set_last_cuda_error(e); *p = nullptr; return ZKQ_ENOMEM; }
  *have = want;
  return ZKQ_OK;
}

#define ZKQ_DISPATCH_W(w, F, ...) \
  do { if ((w) == 1) { F<1> __VA_ARGS__; } else if ((w) == 2) { F<2> __VA_ARGS__; } else { F<4> __VA_ARGS__; } } while (0)

size_t plane_cache_entry_bytes(int m, int k, int r) {
  const size_t mp = (size_t)(m + OZ_BM - 1) / OZ_BM * OZ_BM, kp = (size_t)(2 * k + 63) / 64 * 64;
  return al((size_t)2 * r * mp * kp * sizeof(__half)) + al((size_t)m * sizeof(int32_t));
}

int crt_moduli(int k, int p_out_bits) {
  CrtConst cc;
  return crt_build(2 * k, p_out_bits, &cc) ? cc.r : 0;
}

zkq_status mw_gemm_batched(const MwProd* prods, int count, int wa, int wb, int wc, int p_out_bits, int method,
                           void** ws, size_t* ws_bytes, void** meta, size_t* meta_bytes, cudaStream_t st,
                           HostStage* stage, PlaneCache* const* caches, int ncaches) {
  // uploads of the batch description: pinned ring when available, else plain copies
  auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (stage) { stage->add(dst, src, bytes); return cudaSuccess; }
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  auto up_done = [&]() -> cudaError_t { return stage ? stage->flush(st) : cudaSuccess; };
  if (count <= 0) return ZKQ_OK;
  for (int w : {wa, wb, wc}) if (w != 1 && w != 2 && w != 4) return ZKQ_EINVAL;
  std::vector<OzProd> dp(count);
  int max_kp = 0, max_mn = 0;
  for (int i = 0; i < count; ++i) {
    const MwProd& q = prods[i];
    if (q.m < 1 || q.n < 1 || q.k < 1 || 2 * q.k > 4096) return ZKQ_EINVAL;
    OzProd& o = dp[i];
    std::memset(&o, 0, sizeof(o));
    o.m = q.m; o.n = q.n; o.k = q.k; o.opA = q.opA;
    o.A = q.A; o.B = q.B; o.C = q.C; o.base = q.base; o.sgn = q.sgn; o.base_identity = q.base_identity;
    o.hermitian = (q.hermitian && q.m == q.n) ? 1 : 0;
    o.sliceA = o.sliceB = 1;
    o.mp = (q.m + OZ_BM - 1) / OZ_BM * OZ_BM;
    o.np2 = (2 * q.n + OZ_BN - 1) / OZ_BN * OZ_BN;
    o.kp = (2 * q.k + 63) / 64 * 64;            // multiple of both kernels' K step
    max_kp = std::max(max_kp, 2 * q.k);
    max_mn = std::max(max_mn, q.m * q.n);
  }
  if (method == 0) {
    zkq_status s = grow(meta, meta_bytes, al(sizeof(OzProd) * count));
    if (s != ZKQ_OK) return s;
    ZKQ_CUDA_TRY(up(*meta, dp.data(), sizeof(OzProd) * count));
    ZKQ_CUDA_TRY(up_done());
    dim3 grid((max_mn + 127) / 128, count);
    const OzProd* d = (const OzProd*)*meta;
    ProfScope ps(PC_OZ_GEMM, st);
#define ZKQ_PLAIN(A_, B_, C_) if (wa == A_ && wb == B_ && wc == C_) mw_gemm_plain_kernel<A_, B_, C_><<<grid, 128, 0, st>>>(d);
    ZKQ_PLAIN(1,1,1) ZKQ_PLAIN(1,1,2) ZKQ_PLAIN(1,1,4) ZKQ_PLAIN(1,2,2) ZKQ_PLAIN(1,2,4) ZKQ_PLAIN(1,4,4)
    ZKQ_PLAIN(2,1,2) ZKQ_PLAIN(2,2,2) ZKQ_PLAIN(2,4,4) ZKQ_PLAIN(2,1,4) ZKQ_PLAIN(2,2,4) ZKQ_PLAIN(2,4,2)
    ZKQ_PLAIN(4,1,4) ZKQ_PLAIN(4,2,4) ZKQ_PLAIN(4,4,4) ZKQ_PLAIN(4,4,2) ZKQ_PLAIN(4,1,2) ZKQ_PLAIN(4,2,2)
    ZKQ_PLAIN(1,4,2) ZKQ_PLAIN(2,1,1) ZKQ_PLAIN(4,1,1)
#undef ZKQ_PLAIN
    ZKQ_CUDA_TRY(cudaGetLastError());
    return ZKQ_OK;
  }
  // method 1: CRT form (default); method 2: digit-pair form
  CrtConst cc;
  OzPlan plan;
  std::vector<OzPair> pairs;
  bool crt = (method == 1) && crt_build(max_kp, p_out_bits, &cc);   // K' > 1024: digit form
  if (crt) {
    // planes: [0, r) high halves, [r, 2r) low halves; levels: hh i, hl r + i, lh 2r + i
    plan.b = 0; plan.sA = plan.sB = 2 * cc.r; plan.S = 3 * cc.r - 1; plan.G = 1;
    for (int i = 0; i < cc.r; ++i) {
      pairs.push_back({(int16_t)(i + 1), (int16_t)(i + 1), (int16_t)i, (int16_t)3});
      pairs.push_back({(int16_t)(i + 1), (int16_t)(cc.r + i + 1), (int16_t)(cc.r + i), (int16_t)3});
      pairs.push_back({(int16_t)(cc.r + i + 1), (int16_t)(i + 1), (int16_t)(2 * cc.r + i), (int16_t)3});
    }
  } else {
    plan = ozaki_plan(max_kp, wa, wb, p_out_bits);
    pairs = make_pairs(plan);
  }
  plan.npairs = (int)pairs.size();
  // workspace layout
  size_t off = 0;
  std::vector<size_t> oA(count), oB(count), oD(count), oe(count);
  size_t max_mkp = 0, max_nkp = 0;
  // operands shared by several products of the batch (same matrix, same role) are split once
  std::vector<int> srcA(count), srcB(count);
  for (int i = 0; i < count; ++i) {
    srcA[i] = i; srcB[i] = i;
    for (int j = 0; j < i; ++j) {
      const OzProd &a = dp[i], &b = dp[j];
      if (srcA[i] == i && srcA[j] == j && a.A == b.A && a.opA == b.opA && a.m == b.m && a.k == b.k) srcA[i] = j;
      if (srcB[i] == i && srcB[j] == j && a.B == b.B && a.n == b.n && a.k == b.k) srcB[i] = j;
    }
    if (srcA[i] != i) dp[i].sliceA = 0;
    if (srcB[i] != i) dp[i].sliceB = 0;
  }
  // constant operands: planes and exponents from the caller's cache (kept by an earlier call), or split
  // into a new cache entry by this call
  std::vector<__half*> extP(count, nullptr);
  std::vector<int32_t*> extE(count, nullptr);
  if (crt && caches) {
    for (int i = 0; i < count; ++i) {
      if (srcA[i] != i || prods[i].keepA < 1 || prods[i].keepA > ncaches || !caches[prods[i].keepA - 1]) continue;
      PlaneCache* cache = caches[prods[i].keepA - 1];
      const OzProd& o = dp[i];
      bool hit = false;
      for (const PlaneCache::Entry& e : cache->entries)
        if (e.A == o.A && e.opA == o.opA && e.m == o.m && e.k == o.k && e.q == cc.q && e.r == cc.r && e.s == cc.s) {
          extP[i] = e.planes; extE[i] = e.exps; dp[i].sliceA = 0; hit = true;
          break;
        }
      if (hit) continue;
      const size_t need = plane_cache_entry_bytes(o.m, o.k, cc.r);
      if (cache->used + need > cache->bytes) continue;
      __half* planes = (__half*)(cache->buf + cache->used);
      int32_t* exps = (int32_t*)(cache->buf + cache->used + al((size_t)plan.sA * o.mp * o.kp * sizeof(__half)));
      cache->used += need;
      cache->entries.push_back({o.A, o.opA, o.m, o.k, cc.q, cc.r, cc.s, planes, exps});
      extP[i] = planes; extE[i] = exps;             // split into the entry by this call
    }
  }
  for (int i = 0; i < count; ++i) {
    OzProd& o = dp[i];
    oA[i] = off; if (o.sliceA && !extP[i]) off += al((size_t)plan.sA * o.mp * o.kp * sizeof(__half));
    oB[i] = off; if (o.sliceB) off += al((size_t)plan.sB * o.np2 * o.kp * sizeof(__half));
    oD[i] = off; off += al(crt ? (size_t)3 * cc.r * o.mp * o.np2 : (size_t)(plan.S + 1) * o.mp * o.np2 * sizeof(int32_t));
    oe[i] = off; off += al((size_t)(o.m + o.n) * sizeof(int32_t));
    max_mkp = std::max(max_mkp, (size_t)o.mp * o.kp);
    max_nkp = std::max(max_nkp, (size_t)o.np2 * o.kp);
  }
  zkq_status s = grow(ws, ws_bytes, off);
  if (s != ZKQ_OK) return s;
  char* base = (char*)*ws;
  std::vector<OzTile> tiles, wide;                 // wide: 256-column tiles (CRT form on the tcgen05 kernel)
  const bool use_wide = crt && g_gemm_kernel == 1 && wide_tiles_for(max_kp);
  for (int i = 0; i < count; ++i) {
    OzProd& o = dp[i];
    o.Ahat = (__half*)(base + oA[i]); o.Bhat = (__half*)(base + oB[i]);
    o.D = (int32_t*)(base + oD[i]); o.eA = (int32_t*)(base + oe[i]); o.eB = o.eA + o.m;
    if (extP[i]) { o.Ahat = extP[i]; o.eA = extE[i]; }
  }
  for (int i = 0; i < count; ++i) {                // shared operands point at the first product's planes
    OzProd& o = dp[i];
    if (!o.sliceA) { o.Ahat = dp[srcA[i]].Ahat; o.eA = dp[srcA[i]].eA; }
    if (!o.sliceB) { o.Bhat = dp[srcB[i]].Bhat; o.eB = dp[srcB[i]].eB; }
    // a Hermitian output keeps a tile if one of its columns j (re block: j', im block: j' - n) reaches
    // row ti*BM
    auto needed = [&](int ti, int c0, int width) {
      if (!o.hermitian) return true;
      int c1 = std::min(c0 + width, 2 * o.n), jmax = -1;
      if (c0 < o.n) jmax = std::max(jmax, std::min(c1, o.n) - 1);
      if (c1 > o.n) jmax = std::max(jmax, c1 - 1 - o.n);
      return jmax >= ti * OZ_BM;
    };
    for (int ti = 0; ti < o.mp / OZ_BM; ++ti) {
      const int units = o.np2 / OZ_BN;
      for (int tj = 0; tj < units;) {
        if (use_wide && tj + 1 < units) {
          if (needed(ti, tj * OZ_BN, 2 * OZ_BN)) wide.push_back({i, ti, tj, 2, 0, plan.npairs});
          tj += 2;
        } else {
          if (needed(ti, tj * OZ_BN, OZ_BN)) tiles.push_back({i, ti, tj, 1, 0, plan.npairs});
          tj += 1;
        }
      }
    }
  }
  // biggest problems first (their tiles run longest: K' is larger)
  // one list: longest tiles first (K', then width), so the tail of the launch is short tiles
  tiles.insert(tiles.end(), wide.begin(), wide.end());
  // A batch with fewer tiles than two per SM (one large product, as in an MPS gate update) would leave most SMs
  // idle while each tile walks its 3r pairs: on the tcgen05 kernel's CRT form, where every pair is an
  // independent level with its own residue planes, split each tile's pairs over several CTAs (at least six
  // pairs each).
  if (crt && g_gemm_kernel == 1) {
    const int want = 2 * device_sm_count();
    if (!tiles.empty() && (int)tiles.size() < want) {
      const int G = std::min((want + (int)tiles.size() - 1) / (int)tiles.size(), std::max(1, plan.npairs / 6));
      if (G > 1) {
        std::vector<OzTile> split;
        split.reserve(tiles.size() * G);
        for (const OzTile& t : tiles)
          for (int g = 0; g < G; ++g) {
            OzTile u = t;
            u.p0 = (int)((long)plan.npairs * g / G); u.p1 = (int)((long)plan.npairs * (g + 1) / G);
            split.push_back(u);
          }
        tiles.swap(split);
      }
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(), [&](const OzTile& a, const OzTile& c) {
    const long wa_ = (long)dp[a.prod].kp * a.w * (a.p1 - a.p0), wc_ = (long)dp[c.prod].kp * c.w * (c.p1 - c.p0);
    return wa_ > wc_;
  });
  size_t m_p = al(sizeof(OzProd) * count), m_t = al(sizeof(OzTile) * std::max<size_t>(1, tiles.size())), m_q = al(sizeof(OzPair) * pairs.size());
  size_t m_c = crt ? al(sizeof(CrtConst)) : 0;
  s = grow(meta, meta_bytes, m_p + m_t + m_q + m_c);
  if (s != ZKQ_OK) return s;
  char* mb = (char*)*meta;
  OzProd* d_p = (OzProd*)mb; OzTile* d_t = (OzTile*)(mb + m_p); OzPair* d_q = (OzPair*)(mb + m_p + m_t);
  CrtConst* d_c = (CrtConst*)(mb + m_p + m_t + m_q);
  if (crt) ZKQ_CUDA_TRY(up(d_c, &cc, sizeof(CrtConst)));
  ZKQ_CUDA_TRY(up(d_p, dp.data(), sizeof(OzProd) * count));
  ZKQ_CUDA_TRY(up(d_t, tiles.data(), sizeof(OzTile) * tiles.size()));
  ZKQ_CUDA_TRY(up(d_q, pairs.data(), sizeof(OzPair) * pairs.size()));
  ZKQ_CUDA_TRY(up_done());
  int max_rows = 0;
  for (auto& o : dp) max_rows = std::max(max_rows, o.m + o.n);
  {
    dim3 g((max_rows + 127) / 128, count);
    ProfScope ps(PC_OZ_SCALE, st);
#define ZKQ_SC(A_, B_) if (wa == A_ && wb == B_) oz_scale_kernel<A_, B_><<<g, 128, 0, st>>>(d_p);
    ZKQ_SC(1,1) ZKQ_SC(1,2) ZKQ_SC(1,4) ZKQ_SC(2,1) ZKQ_SC(2,2) ZKQ_SC(2,4) ZKQ_SC(4,1) ZKQ_SC(4,2) ZKQ_SC(4,4)
#undef ZKQ_SC
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  {
    dim3 gA((unsigned)((max_mkp + 255) / 256), count), gB((unsigned)((max_nkp + 255) / 256), count);
    ProfScope ps(PC_OZ_SLICE, st);
    if (crt) {
      // two entries per thread; digits per half: 5 (double-double-sized products), 8 (quad-double), 20
      dim3 gA2((unsigned)((max_mkp / 2 + 255) / 256), count), gB2((unsigned)((max_nkp / 2 + 255) / 256), count);
#define ZKQ_CRT_SLICE(HD) \
      if (wa == 1) crt_slice_A_kernel<1, HD><<<gA2, 256, 0, st>>>(d_p, d_c); \
      else if (wa == 2) crt_slice_A_kernel<2, HD><<<gA2, 256, 0, st>>>(d_p, d_c); \
      else crt_slice_A_kernel<4, HD><<<gA2, 256, 0, st>>>(d_p, d_c); \
      if (wb == 1) crt_slice_B_kernel<1, HD><<<gB2, 256, 0, st>>>(d_p, d_c); \
      else if (wb == 2) crt_slice_B_kernel<2, HD><<<gB2, 256, 0, st>>>(d_p, d_c); \
      else crt_slice_B_kernel<4, HD><<<gB2, 256, 0, st>>>(d_p, d_c);
      if (cc.hdig <= 5) { ZKQ_CRT_SLICE(5) } else if (cc.hdig <= 8) { ZKQ_CRT_SLICE(8) } else { ZKQ_CRT_SLICE(20) }
#undef ZKQ_CRT_SLICE
    } else {
      ZKQ_DISPATCH_W(wa, oz_slice_A_kernel, <<<gA, 256, 0, st>>>(d_p, plan.b, plan.sA));
      ZKQ_DISPATCH_W(wb, oz_slice_B_kernel, <<<gB, 256, 0, st>>>(d_p, plan.b, plan.sB));
    }
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  {
    size_t sm = (size_t)OZ_STAGES * (OZ_BM + OZ_BN) * 64;
    if (g_gemm_kernel != 1)
      ZKQ_CUDA_TRY(smem_limit_max<oz_gemm_kernel>());
    double flops = 0.0;                        // algorithmic: every kept digit pair, unpadded sizes
    for (auto& o : dp) flops += 2.0 * plan.npairs * (double)o.m * (2.0 * o.n) * (2.0 * o.k);
    ProfScope ps(PC_OZ_GEMM, st, flops);
    if (g_gemm_kernel == 1) {
      {
        static std::mutex mu;                          // contexts on several host threads share the flag
        std::lock_guard<std::mutex> g(mu);
        if (!g_oz_err) {
          ZKQ_CUDA_TRY(cudaMalloc(&g_oz_err, sizeof(int)));
          ZKQ_CUDA_TRY(cudaMemset(g_oz_err, 0, sizeof(int)));
        }
      }
      zkq_status ls = launch_oz_tc(d_p, d_t, (int)tiles.size(), d_q, plan.npairs, crt ? d_c : nullptr, g_oz_err, st);
      if (ls != ZKQ_OK) return ls;
    } else {
      oz_gemm_kernel<<<(unsigned)tiles.size(), 256, sm, st>>>(d_p, d_t, d_q, plan.npairs, plan.S, crt ? d_c : nullptr);
    }
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  {
    dim3 g((max_mn + 127) / 128, count);
    ProfScope ps(PC_OZ_COMBINE, st);
    if (crt) {
      // limbs sized to M and C': double-double-sized products (M < 2^176, C' < 2^320), quad-double-sized
      // (M < 2^272, C' < 2^512), else the largest
#define ZKQ_CRT_COMB(LW, LT) \
      if (wc == 1) crt_combine_kernel<1, LW, LT><<<g, 128, 0, st>>>(d_p, d_c); \
      else if (wc == 2) crt_combine_kernel<2, LW, LT><<<g, 128, 0, st>>>(d_p, d_c); \
      else crt_combine_kernel<4, LW, LT><<<g, 128, 0, st>>>(d_p, d_c);
      if (cc.l32 <= 6 && cc.tbits <= 5 * 64 - 1) { ZKQ_CRT_COMB(6, 5) }
      else if (cc.l32 <= 9 && cc.tbits <= 8 * 64 - 1) { ZKQ_CRT_COMB(9, 8) }
      else { ZKQ_CRT_COMB(18, CRT_L + 1) }
#undef ZKQ_CRT_COMB
    } else {
      if (wc == 1) oz_combine_kernel<1><<<g, 128, 0, st>>>(d_p, plan.b, plan.S);
      else if (wc == 2) oz_combine_kernel<2><<<g, 128, 0, st>>>(d_p, plan.b, plan.S);
      else oz_combine_kernel<4><<<g, 128, 0, st>>>(d_p, plan.b, plan.S);
    }
    ZKQ_CUDA_TRY(cudaGetLastError());
  }
  return ZKQ_OK;
}

// Bytes that mw_gemm_batched needs for a product batch: the workspace (residue or digit planes of every
// operand it splits, GEMM outputs, exponents) exactly as it lays them out, and an upper bound of the
// metadata (products, at most one tile per 128 x 128 output block plus the split tiles of a small batch,
// pair list, CRT constants).  Operands are
// shared by the same pointer, role and shape test as in mw_gemm_batched; the pointers are only compared.
zkq_status mw_gemm_workspace(const MwProd* prods, int count, int wa, int wb, int p_out_bits, int method,
                             size_t* ws_need, size_t* meta_need) {
  *ws_need = 0; *meta_need = 0;
  if (count <= 0) return ZKQ_OK;
  for (int w : {wa, wb}) if (w != 1 && w != 2 && w != 4) return ZKQ_EINVAL;
  std::vector<int> mp(count), np2(count), kp(count);
  int max_kp = 0;
  for (int i = 0; i < count; ++i) {
    const MwProd& q = prods[i];
    if (q.m < 1 || q.n < 1 || q.k < 1 || 2 * q.k > 4096) return ZKQ_EINVAL;
    mp[i] = (q.m + OZ_BM - 1) / OZ_BM * OZ_BM;
    np2[i] = (2 * q.n + OZ_BN - 1) / OZ_BN * OZ_BN;
    kp[i] = (2 * q.k + 63) / 64 * 64;
    max_kp = std::max(max_kp, 2 * q.k);
  }
  if (method == 0) { *meta_need = al(sizeof(OzProd) * count); return ZKQ_OK; }
  CrtConst cc;
  size_t sA = 0, sB = 0, levels = 0, npairs = 0;
  const bool crt = (method == 1) && crt_build(max_kp, p_out_bits, &cc);
  if (crt) { sA = sB = 2 * cc.r; npairs = 3 * cc.r; }
  else {
    const OzPlan plan = ozaki_plan(max_kp, wa, wb, p_out_bits);
    sA = plan.sA; sB = plan.sB; levels = plan.S + 1; npairs = make_pairs(plan).size();
  }
  size_t off = 0, tiles = 0;
  for (int i = 0; i < count; ++i) {
    const MwProd& a = prods[i];
    bool ownA = true, ownB = true;
    for (int j = 0; j < i; ++j) {              // the first product with the operand splits it
      const MwProd& b = prods[j];
      if (ownA && a.A == b.A && a.opA == b.opA && a.m == b.m && a.k == b.k) ownA = false;
      if (ownB && a.B == b.B && a.n == b.n && a.k == b.k) ownB = false;
    }
    if (ownA) off += al(sA * mp[i] * kp[i] * sizeof(__half));
    if (ownB) off += al(sB * np2[i] * kp[i] * sizeof(__half));
    off += al(crt ? (size_t)3 * cc.r * mp[i] * np2[i] : levels * mp[i] * np2[i] * sizeof(int32_t));
    off += al((size_t)(a.m + a.n) * sizeof(int32_t));
    tiles += (size_t)(mp[i] / OZ_BM) * (np2[i] / OZ_BN);
  }
  *ws_need = off;
  // a batch of few tiles may have its pairs split over up to 2 x SMs more (mw_gemm_batched)
  tiles += crt ? (size_t)2 * device_sm_count() : 0;
  *meta_need = al(sizeof(OzProd) * count) + al(sizeof(OzTile) * std::max<size_t>(1, tiles)) +
               al(sizeof(OzPair) * npairs) + (crt ? al(sizeof(CrtConst)) : 0);
  return ZKQ_OK;
}

// device bytes grow() holds after growing to `need` bytes from nothing
size_t oz_grow_bytes(size_t need) { return std::max(need + need / 4, (size_t)1 << 20); }

int gemm_kernel_get() { return g_gemm_kernel; }
void gemm_kernel_set(int k) { g_gemm_kernel = k; }
// reads and clears the expired-wait flag of the tcgen05 kernel (synchronous)
bool gemm_kernel_error() {
  if (!g_oz_err) return false;
  int h = 0;
  cudaMemcpy(&h, g_oz_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (h) cudaMemset(g_oz_err, 0, sizeof(int));
  return h != 0;
}

}  // namespace zkq
