// Host construction of the CRT constants: moduli, weights w_i = (M/m_i) inv(M/m_i mod m_i), and M.
#include "crt.cuh"
#include <vector>
#include <cmath>
#include <cstring>
#include <algorithm>

namespace zkq {

namespace {
using Limbs = std::vector<uint32_t>;   // little-endian base 2^32 magnitude
void mul_small(Limbs& a, uint32_t m) {
  uint64_t c = 0;
  for (auto& x : a) { uint64_t t = (uint64_t)x * m + c; x = (uint32_t)t; c = t >> 32; }
  if (c) a.push_back((uint32_t)c);
}
uint32_t mod_small(const Limbs& a, uint32_t m) {
  uint64_t r = 0;
  for (size_t i = a.size(); i-- > 0;) r = ((r << 32) | a[i]) % m;
  return (uint32_t)r;
}
Limbs div_small(const Limbs& a, uint32_t m) {   // exact quotient (floor)
  Limbs q(a.size());
  uint64_t r = 0;
  for (size_t i = a.size(); i-- > 0;) { uint64_t cur = (r << 32) | a[i]; q[i] = (uint32_t)(cur / m); r = cur % m; }
  while (q.size() > 1 && q.back() == 0) q.pop_back();
  return q;
}
int inv_mod(int a, int m) {                    // a^-1 mod m (gcd(a, m) = 1)
  int t = 0, nt = 1, r = m, nr = a % m;
  while (nr) { int qq = r / nr; int tmp = t - qq * nt; t = nt; nt = tmp; tmp = r - qq * nr; r = nr; nr = tmp; }
  return t < 0 ? t + m : t;
}
int gcd(int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }
void to32(const Limbs& a, uint32_t* out) {
  for (int i = 0; i < CRT_L32; ++i) out[i] = i < (int)a.size() ? a[i] : 0;
}
void to64(const Limbs& a, uint64_t* out) {
  for (int i = 0; i < CRT_L; ++i) {
    uint64_t lo = (2 * i < (int)a.size()) ? a[2 * i] : 0, hi = (2 * i + 1 < (int)a.size()) ? a[2 * i + 1] : 0;
    out[i] = lo | (hi << 32);
  }
}
}  // namespace

bool crt_build(int max_kprime, int p_out_bits, CrtConst* out) {
  std::memset(out, 0, sizeof(CrtConst));
  int lg = 0; while ((1 << lg) < max_kprime) ++lg;
  // modulus bound: K' (m/2)^2 <= 2^24 keeps every residue product sum exact in fp32
  int mb = 256;
  if ((long long)max_kprime * (mb / 2) * (mb / 2) > (1LL << 24)) return false;   // K' > 1024: digit form
  const int q = p_out_bits + lg + 4;           // |A'|,|B'| < 2^(q-2); truncation error 2^-q of the scale
  const int s = (q - 2 + 1) / 2;               // halves: |A_h| <= 2^(q-2-s), 0 <= A_l < 2^s
  const int hb = std::max(q - 2 - s, s);       // each half below 2^hb
  const double need = 2.0 * hb + lg + 4;       // log2 M > log2(4 K' 2^(2 hb)): C_hl + C_lh, with a margin
  std::vector<int> ms;
  double bits = 0.0;
  for (int c = mb; c >= 3 && bits < need; --c) {
    bool ok = true;
    for (int x : ms) if (gcd(x, c) != 1) { ok = false; break; }
    if (!ok) continue;
    ms.push_back(c);
    bits += std::log2((double)c);
  }
  if (bits < need || (int)ms.size() > CRT_MAXR || bits + 16 > 64.0 * CRT_L - 2) return false;
  out->r = (int)ms.size();
  out->q = q;
  out->s = s;
  Limbs M{1};
  for (int m : ms) mul_small(M, (uint32_t)m);
  to64(M, out->M);
  to32(M, out->M32);
  Limbs half = div_small(M, 2);
  to64(half, out->Mhalf);
  to32(half, out->Mhalf32);
  for (int i = 0; i < out->r; ++i) {
    int m = ms[i];
    out->m[i] = m;
    Limbs Mi = div_small(M, (uint32_t)m);
    int inv = inv_mod((int)mod_small(Mi, (uint32_t)m), m);
    Limbs w = Mi; mul_small(w, (uint32_t)inv);
    to64(w, out->w[i]);
    to32(w, out->w32[i]);
    out->minv[i] = (uint32_t)((1ULL << 32) / (uint64_t)m) + 1;
    uint32_t p = 1 % m;
    for (int j = 0; j < 20; ++j) { out->pw16[i][j] = (uint8_t)p; p = (uint32_t)(((uint64_t)p << 16) % m); }
  }
  out->l32 = (int)std::ceil((bits + 16.0) / 32.0);
  if (out->l32 > CRT_L32) return false;
  out->hdig = (std::max(q - 2 - s, s) + 1 + 15) / 16;
  if (out->hdig > 20) return false;
  out->tbits = 2 * q - 4 + lg + 2;
  if (out->tbits > 64 * (CRT_L + 1) - 1) return false;
  // M as double * 2^exp (from its top 64 bits)
  int top = CRT_L - 1; while (top > 0 && out->M[top] == 0) --top;
  double v = (double)out->M[top] + (top > 0 ? std::ldexp((double)out->M[top - 1], -64) : 0.0);
  int e = 0; double fr = std::frexp(v, &e);   // v = fr 2^e, fr in [0.5,1)
  out->Md = fr * 2.0; out->Mexp = e - 1 + 64 * top;
  out->Mrcp = 1.0 / out->Md;
  return true;
}

}  // namespace zkq
