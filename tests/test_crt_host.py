"""The host construction of the Chinese-remainder constants of the split products (Ozaki scheme II), checked
against number theory with Python integers: pairwise coprime moduli <= 256 whose product M covers the
bits the exact products need, CRT weights w_i that are 1 modulo m_i and 0 modulo every other modulus,
floor(M / 2), the division-free reciprocals floor(2^32 / m) + 1, the powers 2^(16 j) mod m, and the limb
and digit counts.  CPU only: crt_host.cu is plain C++, built here with a small C wrapper."""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_11868_gb300", "csrc")
MAXR, L64, L32 = 96, 9, 18

WRAP = r"""
#include <cstring>
#include "crt.cuh"
extern "C" int crt_info(int kp, int p, int* ints, int* m, unsigned* minv, unsigned* w32, unsigned* M32, unsigned* Mh32,
                        unsigned char* pw16, unsigned long long* w64, unsigned long long* M64, unsigned long long* Mh64,
                        double* d) {
  zkq::CrtConst c;
  if (!zkq::crt_build(kp, p, &c)) return 0;
  ints[0] = c.r; ints[1] = c.q; ints[2] = c.s; ints[3] = c.l32; ints[4] = c.hdig; ints[5] = c.tbits; ints[6] = c.Mexp;
  for (int i = 0; i < c.r; ++i) {
    m[i] = c.m[i]; minv[i] = c.minv[i];
    std::memcpy(w32 + i * zkq::CRT_L32, c.w32[i], sizeof(c.w32[i]));
    std::memcpy(w64 + i * zkq::CRT_L, c.w[i], sizeof(c.w[i]));
    std::memcpy(pw16 + i * 20, c.pw16[i], 20);
  }
  std::memcpy(M32, c.M32, sizeof(c.M32)); std::memcpy(Mh32, c.Mhalf32, sizeof(c.Mhalf32));
  std::memcpy(M64, c.M, sizeof(c.M)); std::memcpy(Mh64, c.Mhalf, sizeof(c.Mhalf));
  d[0] = c.Md; d[1] = c.Mrcp;
  return 1;
}
"""


@pytest.fixture(scope="module")
def crt(tmp_path_factory):
    d = tmp_path_factory.mktemp("crt")
    (d / "wrap.cpp").write_text(WRAP)
    so = d / "crt.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", f"-I{CSRC}", "-x", "c++",
                    os.path.join(CSRC, "crt_host.cu"), "-x", "c++", str(d / "wrap.cpp"), "-o", str(so)],
                   check=True, capture_output=True, text=True)
    L = ctypes.CDLL(str(so))
    L.crt_info.restype = ctypes.c_int

    def info(kp, p):
        ints = (ctypes.c_int * 7)()
        m = (ctypes.c_int * MAXR)(); minv = (ctypes.c_uint * MAXR)()
        w32 = (ctypes.c_uint * (MAXR * L32))(); M32 = (ctypes.c_uint * L32)(); Mh32 = (ctypes.c_uint * L32)()
        pw16 = (ctypes.c_ubyte * (MAXR * 20))()
        w64 = (ctypes.c_ulonglong * (MAXR * L64))(); M64 = (ctypes.c_ulonglong * L64)(); Mh64 = (ctypes.c_ulonglong * L64)()
        dd = (ctypes.c_double * 2)()
        if not L.crt_info(kp, p, ints, m, minv, w32, M32, Mh32, pw16, w64, M64, Mh64, dd):
            return None
        limbs = lambda arr, off, n, bits: sum(int(arr[off + k]) << (bits * k) for k in range(n))
        r = ints[0]
        return dict(r=r, q=ints[1], s=ints[2], l32=ints[3], hdig=ints[4], tbits=ints[5], Mexp=ints[6],
                    m=[m[i] for i in range(r)], minv=[minv[i] for i in range(r)],
                    w32=[limbs(w32, i * L32, L32, 32) for i in range(r)], w64=[limbs(w64, i * L64, L64, 64) for i in range(r)],
                    M32=limbs(M32, 0, L32, 32), M64=limbs(M64, 0, L64, 64), Mh32=limbs(Mh32, 0, L32, 32),
                    Mh64=limbs(Mh64, 0, L64, 64), pw16=[[pw16[i * 20 + j] for j in range(20)] for i in range(r)],
                    Md=dd[0], Mrcp=dd[1])
    return info


@pytest.mark.parametrize("kp", [2, 64, 250, 1024])
@pytest.mark.parametrize("p", [53 + 6, 106 + 6, 212 + 6])
def test_crt_constants_satisfy_their_definitions(crt, kp, p):
    c = crt(kp, p)
    assert c is not None
    m, r = c["m"], c["r"]
    assert r == len(m) and all(3 <= x <= 256 for x in m) and m == sorted(m, reverse=True)
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(m) for b in m[i + 1:])
    M = math.prod(m)
    assert c["M32"] == M and c["M64"] == M and c["Mh32"] == M // 2 and c["Mh64"] == M // 2
    for i in range(r):
        assert c["w32"][i] == c["w64"][i] < M
        for j in range(r):
            assert c["w32"][i] % m[j] == (1 if i == j else 0)
        assert c["minv"][i] == (1 << 32) // m[i] + 1
        assert c["pw16"][i] == [pow(2, 16 * j, m[i]) for j in range(20)]
    # bit budget: q-bit scaled integers split in halves below 2^hb; M covers the two cross products with margin
    lg = max(0, (kp - 1).bit_length())
    q = p + lg + 4
    s = (q - 1) // 2
    hb = max(q - 2 - s, s)
    assert (c["q"], c["s"]) == (q, s)
    assert math.log2(M) >= 2 * hb + lg + 4
    assert math.log2(M // m[-1]) < 2 * hb + lg + 4           # the last (smallest) modulus was needed
    assert M << 16 < 1 << (32 * c["l32"])
    assert 16 * c["hdig"] >= hb + 1
    assert c["tbits"] == 2 * q - 4 + lg + 2
    assert abs(c["Md"] * 2.0 ** c["Mexp"] / M - 1) < 2.0 ** -50 and 1 <= c["Md"] < 2
    assert c["Mrcp"] == 1.0 / c["Md"]


def test_crt_form_stops_above_k_prime_1024_and_counts_moduli(crt):
    """K' (m/2)^2 <= 2^24 keeps every residue product sum exact in fp32, so K' > 1024 has no CRT form; the
    modulus counts at K' = 1024 are those quoted for double-double and quad-double accuracy."""
    assert crt(1025, 218) is None and crt(4096, 112) is None
    assert crt(1024, 112)["r"] == 18 and crt(1024, 218)["r"] == 33
