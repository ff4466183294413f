"""The multi-word arithmetic checks are not vacuous.  A copy of the double-double / quad-double header
gets one planted slip, the kind a slip in writing out an error-free transformation would make: a dropped
error term, a missing cross product, a skipped correction, a sign.  It is built on the host together with
the element-wise entry point into a library of its own, and the host arithmetic checks run against it.
At least one check must fail for every slip.  CPU only (nvcc builds host code without a GPU); the slips
live in the copies, never in the library."""
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

STUB = """#include <cuda_runtime.h>
namespace zkq { void set_last_cuda_error(cudaError_t) {} }
"""


def build_copy(tmp, old=None, new=None):
    src = tmp / "pkg" / "csrc"
    src.mkdir(parents=True)
    (tmp / "include").mkdir()
    for f in ("mwop.cu", "mw.cuh", "common.cuh"):
        shutil.copy(os.path.join(CSRC, f), src / f)
    shutil.copy(os.path.join(ROOT, "include", "zkq.h"), tmp / "include" / "zkq.h")
    if old is not None:
        text = (src / "mw.cuh").read_text()
        assert text.count(old) == 1, f"the text to change is not unique in mw.cuh: {old!r}"
        (src / "mw.cuh").write_text(text.replace(old, new))
    (src / "stub.cu").write_text(STUB)
    out = tmp / "mw_copy.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC,-ffp-contract=off", "-diag-suppress", "128", str(src / "mwop.cu"),
                    str(src / "stub.cu"), "-o", str(out)], check=True, capture_output=True, text=True)
    L = ctypes.CDLL(str(out))
    P = ctypes.c_void_p
    L.zkq_mw_op.restype = ctypes.c_int
    L.zkq_mw_op.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, P, P, ctypes.c_int, P]

    def mw_op(op, words, count, a, b, out_):
        assert L.zkq_mw_op(op, words, count, a.ctypes.data, b.ctypes.data, out_.ctypes.data, 0, None) == 0
    return mw_op


@pytest.fixture(scope="module")
def nvcc():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")


@pytest.mark.parametrize("name,old,new,checks", SLIPS, ids=[s[0] for s in SLIPS])
def test_planted_slip_fails_a_check(nvcc, tmp_path, name, old, new, checks):
    mw_op = build_copy(tmp_path, old, new)
    failed = []
    for words, op in checks:
        try:
            check_host_op(mw_op, words, op)
        except AssertionError:
            failed.append((words, op))
    assert failed, f"no check noticed the planted slip: {name}"


def test_unchanged_copy_passes_the_checks(nvcc, tmp_path):
    mw_op = build_copy(tmp_path)
    for words in (2, 4):
        for op in range(7):
            check_host_op(mw_op, words, op)
