"""The multi-word arithmetic checks are not vacuous.  A copy of the double-double / quad-double header
gets one planted slip, the kind a slip in writing out an error-free transformation would make: a dropped
error term, a missing cross product, a skipped correction, a sign.  It is built for the host into a
library of its own, with a small wrapper that applies each operation the way the element-wise entry point
does, and the host arithmetic checks run against it.  At least one check must fail for every slip.  CPU
only; the slips live in the copies, never in the library."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import pytest

from tests.test_abi_cpu import check_host_op

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_11868_gb300", "csrc")

# (name, text as written, text with the slip, (words, op) checks that must notice)
SLIPS = [
    ("TwoSum drops the second operand's error", "e = (a - (s - bb)) + (b - bb);", "e = (a - (s - bb));",
     [(2, 0), (4, 0)]),
    ("TwoProd without its FMA error", "e = MW_FMA(a, b, -p);", "e = 0.0;", [(2, 2), (4, 2)]),
    ("double-double product drops a cross term",
     "  e = MW_FMA(a.x[1], b.x[0], e);\n  p = fast_two_sum(p, e, e);\n  return dd_make(p, e);\n}\nMW_HD dd mw_mul_d",
     "  p = fast_two_sum(p, e, e);\n  return dd_make(p, e);\n}\nMW_HD dd mw_mul_d", [(2, 2)]),
    ("quad-double product drops an order-e^3 term", "+ a.x[3] * b.x[0] + q0", "+ q0", [(4, 2)]),
    ("quad-double sum loses the first carry's error", "s1 = two_sum(s1, t0, t0);                     // level 1",
     "s1 = s1 + t0; t0 = 0.0;                     // level 1",
     [(4, 0)]),
    ("double-double square root without its Newton correction",
     "double d = mw_add(a, mw_neg(ax2)).x[0] * (x * 0.5);", "double d = 0.0 * (x * 0.5) + 0.0 * ax2.x[0];",
     [(2, 4)]),
    ("complex product with the wrong sign of the imaginary parts' product",
     "return c_make(mw_sub(mw_mul(a.re, b.re), mw_mul(a.im, b.im)), mw_add(mw_mul(a.re, b.im), mw_mul(a.im, b.re)));",
     "return c_make(mw_add(mw_mul(a.re, b.re), mw_mul(a.im, b.im)), mw_add(mw_mul(a.re, b.im), mw_mul(a.im, b.re)));",
     [(2, 5), (4, 5)]),
    ("complex quotient with the conjugate on the wrong operand",
     "cmw<W> n = c_mul_conj(b, a);", "cmw<W> n = c_mul_conj(a, b);", [(2, 6), (4, 6)]),
]

# the host half of the element-wise entry point: one operation per element, as mwop.cu applies it
WRAP = """#include "mw.cuh"
using namespace zkq;
template <int W> static void apply(int op, long i, const double* a, const double* b, double* out) {
  if (op <= 4) {
    mw<W> x = mw_load<W, W>(a, i), y = mw_load<W, W>(b, i), r;
    switch (op) {
      case 0: r = mw_add(x, y); break;
      case 1: r = mw_sub(x, y); break;
      case 2: r = mw_mul(x, y); break;
      case 3: r = mw_div(x, y); break;
      default: r = mw_sqrt(x); break;
    }
    mw_store(out, i, r);
  } else {
    cmw<W> x = c_load<W, W>(a, i), y = c_load<W, W>(b, i);
    c_store(out, i, op == 5 ? c_mul(x, y) : c_div(x, y));
  }
}
extern "C" int mw_host_op(int op, int words, long count, const double* a, const double* b, double* out) {
  for (long i = 0; i < count; ++i) {
    if (words == 2) apply<2>(op, i, a, b, out);
    else if (words == 4) apply<4>(op, i, a, b, out);
    else return 1;
  }
  return 0;
}
"""


def build_copy(tmp, old=None, new=None):
    shutil.copy(os.path.join(CSRC, "mw.cuh"), tmp / "mw.cuh")
    if old is not None:
        text = (tmp / "mw.cuh").read_text()
        assert text.count(old) == 1, f"the text to change is not unique in mw.cuh: {old!r}"
        (tmp / "mw.cuh").write_text(text.replace(old, new))
    (tmp / "wrap.cpp").write_text(WRAP)
    out = tmp / "mw_copy.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", f"-I{tmp}",
                    str(tmp / "wrap.cpp"), "-o", str(out)], check=True, capture_output=True, text=True)
    L = ctypes.CDLL(str(out))
    P = ctypes.c_void_p
    L.mw_host_op.restype = ctypes.c_int
    L.mw_host_op.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, P, P, P]

    def mw_op(op, words, count, a, b, out_):
        assert L.mw_host_op(op, words, count, a.ctypes.data, b.ctypes.data, out_.ctypes.data) == 0
    return mw_op


@pytest.mark.parametrize("name,old,new,checks", SLIPS, ids=[s[0] for s in SLIPS])
def test_planted_slip_fails_a_check(tmp_path, name, old, new, checks):
    mw_op = build_copy(tmp_path, old, new)
    failed = []
    for words, op in checks:
        try:
            check_host_op(mw_op, words, op)
        except AssertionError:
            failed.append((words, op))
    assert failed, f"no check noticed the planted slip: {name}"


def test_unchanged_copy_passes_the_checks(tmp_path):
    mw_op = build_copy(tmp_path)
    for words in (2, 4):
        for op in range(7):
            check_host_op(mw_op, words, op)
