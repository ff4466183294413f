"""The multi-limb integer helpers of the CRT reconstruction (csrc/crt_limbs.cuh), built on the host with g++
and checked against Python's exact integers and rationals: the barrel shift of a 512-bit two's complement
integer, and the expansion of a signed integer times 2^scale into four words, each the nearest double (ties
to even) of what the words before it left.  The split-product combine kernel rounds its exact products with
these helpers, so a dropped bit, a wrong rounding direction or a sign slip there shows up here."""
from __future__ import annotations

import os
import random
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_11868_gb300", "csrc")
M = 16                                   # 32-bit limbs, as the quad-double reconstruction uses

HARNESS = r"""
#include "crt_limbs.cuh"
#include <cstdio>
int main() {
  int n;
  if (std::scanf("%d", &n) != 1) return 1;
  for (int t = 0; t < n; ++t) {
    uint32_t T[16], U[16];
    int sh, scale;
    for (int k = 0; k < 16; ++k) if (std::scanf("%u", &T[k]) != 1) return 1;
    if (std::scanf("%d %d", &sh, &scale) != 2) return 1;
    for (int k = 0; k < 16; ++k) U[k] = T[k];
    zkq::limbs_shl<16>(U, sh);
    for (int k = 0; k < 16; ++k) std::printf("%u ", U[k]);
    const zkq::mw<4> w = zkq::limbs_round_words<4, 16>(T, scale);
    for (int k = 0; k < 4; ++k) std::printf("%a ", w.x[k]);
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("limbs")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-std=c++17", "-O2", f"-I{CSRC}", str(src), "-o", str(exe)], check=True)
    return exe


def _limbs(x: int) -> list[int]:
    x %= 1 << (32 * M)
    return [(x >> (32 * k)) & 0xFFFFFFFF for k in range(M)]


def _cases(seed: int, count: int):
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        bits = rng.choice([1, 2, 52, 53, 54, 55, 64, 106, 107, 200, 300, 400, 500])
        v = rng.getrandbits(bits)
        r = rng.random()
        if r < 0.15:
            v = (1 << bits) - 1                               # a run of ones: carries through every word
        elif r < 0.3:
            v = (1 << (bits - 1)) | (1 << max(0, bits - 54))  # exactly halfway below the leading 53 bits
        elif r < 0.4:
            v = ((rng.getrandbits(53) | (1 << 52)) << 200) | (1 << 146)   # tie one word further down
        if rng.random() < 0.5:
            v = -v
        out.append((v, rng.randrange(0, 32 * M), rng.randrange(-700, 200)))
    return out


def _run(exe, cases):
    inp = f"{len(cases)}\n" + "\n".join(" ".join(map(str, _limbs(v))) + f" {sh} {sc}" for v, sh, sc in cases)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=60, check=True).stdout
    return out.strip().split("\n")


def test_barrel_shift_matches_python_integers(harness):
    cases = _cases(1, 1500)
    for (v, sh, _), line in zip(cases, _run(harness, cases)):
        got = [int(x) for x in line.split()[:M]]
        assert got == _limbs(v << sh), (v, sh)


def test_rounded_words_are_the_nearest_double_expansion(harness):
    """Each word is float(remaining rational): Python rounds a Fraction to the nearest double, ties to even."""
    cases = _cases(2, 3000)
    for (v, _, scale), line in zip(cases, _run(harness, cases)):
        words = [float.fromhex(x) for x in line.split()[M:]]
        rest = Fraction(v) * Fraction(2) ** scale
        for w in words:
            assert w == float(rest), (v, scale, words)
            rest -= Fraction(w)
        # four words of 53 bits leave at most about 2^-212 of the value
        if v:
            assert abs(rest) <= abs(Fraction(v) * Fraction(2) ** scale) * Fraction(1, 2 ** 200)


def test_zero_and_powers_of_two(harness):
    cases = [(0, 0, 0), (1, 5, 0), (-1, 0, -3), (1 << 300, 0, -300), (-(1 << 511), 0, -511)]
    lines = _run(harness, cases)
    assert [float.fromhex(x) for x in lines[0].split()[M:]] == [0.0] * 4
    assert float.fromhex(lines[1].split()[M]) == 1.0
    assert float.fromhex(lines[2].split()[M]) == -0.125
    assert float.fromhex(lines[3].split()[M]) == 1.0
    assert float.fromhex(lines[4].split()[M]) == -1.0
