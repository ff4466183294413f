"""CPU checks of the C ABI library: it loads without a GPU, exports every declared symbol, rejects bad
arguments, and its host-compiled multi-word arithmetic meets the double-double / quad-double error
bounds against the 320-bit oracle."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests._util import fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zkq():
    import paper_2402_11868_gb300 as Z
    Z.build()
    return Z


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "zkq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(zkq_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(zkq):
    syms = declared_symbols()
    assert len(syms) >= 6
    L = ctypes.CDLL(zkq.LIB_PATH)
    for s in syms:
        assert hasattr(L, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", zkq.LIB_PATH], capture_output=True, text=True).stdout
    for s in syms:
        assert re.search(rf"\bT {s}\b", out), s


def test_status_strings(zkq):
    for s in range(7):
        assert zkq.lib().zkq_status_string(s)


def test_invalid_arguments_are_rejected_without_gpu(zkq):
    L = zkq.lib()
    assert L.zkq_ctx_create(None, None) == zkq.ZKQ_EINVAL
    assert L.zkq_eigh_batched(None, 1, None, None, None, 4, None, None, None, None) == zkq.ZKQ_EINVAL
    assert L.zkq_mw_op(9, 4, 1, None, None, None, 0, None) == zkq.ZKQ_EINVAL
    assert L.zkq_mw_op(0, 3, 1, None, None, None, 0, None) == zkq.ZKQ_EINVAL
    h = ctypes.c_void_p()
    assert L.zkq_plan_create(None, 1, None, None, 4, 4, ctypes.byref(h)) == zkq.ZKQ_EINVAL and not h.value
    assert L.zkq_plan_execute(None, None, None, None, None, None, None, None, None, None) == zkq.ZKQ_EINVAL
    assert L.zkq_plan_execute_graph(None, None, None, None, None, None, None, None, None, None) == zkq.ZKQ_EINVAL
    assert L.zkq_plan_destroy(None) == zkq.ZKQ_OK
    assert L.zkq_autotune_jacobi(None, 1, None, 4, 1, None) == zkq.ZKQ_EINVAL
    nb = ctypes.c_size_t(123)
    n1 = (ctypes.c_int32 * 1)(64)
    assert L.zkq_workspace_size(None, 1, n1, 4, 4, 1, ctypes.byref(nb)) == zkq.ZKQ_EINVAL and nb.value == 123
    assert L.zkq_workspace_size(None, 1, n1, 4, 4, 1, None) == zkq.ZKQ_EINVAL
    assert L.zkq_ctx_workspace_bytes(None, ctypes.byref(nb)) == zkq.ZKQ_EINVAL and nb.value == 123


# published relative error bounds (unit roundoff u = 2^-53): double-double add 3u^2 (accurate sum),
# mul ~4u^2 (Joldes-Muller-Popescu 2017); quad-double ops ~2^-208 (Hida-Li-Bailey 2001 report ~2^-209).
BOUND = {2: {0: 2.0**-103, 1: 2.0**-103, 2: 2.0**-102, 3: 2.0**-101, 4: 2.0**-101},
         4: {0: 2.0**-206, 1: 2.0**-206, 2: 2.0**-206, 3: 2.0**-205, 4: 2.0**-205}}


def random_mw(rng, count, words, spread=30):
    x = np.zeros((count, words))
    e = rng.integers(-spread, spread, count)
    x[:, 0] = np.ldexp(rng.standard_normal(count), e)
    for k in range(1, words):
        x[:, k] = x[:, k - 1] * 2.0**-54 * rng.uniform(-1, 1, count)
    return x


def check_host_op(mw_op, words, op):
    """Raise AssertionError unless the multi-word op (run through mw_op(op, words, count, a, b, out) on host
    arrays) meets its error bound on 400 random operands.  Real ops are compared with the oracle against
    the published bounds; complex multiply and divide (ops 5 and 6) with exact rationals, in norm, against
    bounds that follow from the real ones: |error| <= bound |a| |b| for the product and bound |a| / |b| for
    the quotient."""
    rng = np.random.default_rng(100 * words + op)
    count = 400
    if op >= 5:
        a = random_mw(rng, 2 * count, words).reshape(count, 2, words)
        b = random_mw(rng, 2 * count, words).reshape(count, 2, words)
        out = np.zeros_like(a)
        mw_op(op, words, count, a, b, out)
        for i in range(count):
            ar, ai, br, bi = fr(a[i, 0]), fr(a[i, 1]), fr(b[i, 0]), fr(b[i, 1])
            if op == 5:
                want = (ar * br - ai * bi, ar * bi + ai * br)
                scale2 = (ar * ar + ai * ai) * (br * br + bi * bi)
            else:
                d = br * br + bi * bi
                want = ((ar * br + ai * bi) / d, (ai * br - ar * bi) / d)
                scale2 = (ar * ar + ai * ai) / d
            err2 = (fr(out[i, 0]) - want[0]) ** 2 + (fr(out[i, 1]) - want[1]) ** 2
            bound = {2: 2.0**-100, 4: 2.0**-203}[words]
            assert err2 <= Fraction(bound) ** 2 * scale2, (op, i)
        return
    a = random_mw(rng, count, words)
    b = random_mw(rng, count, words)
    if op == 4:
        a = np.abs(a) * np.sign(a[:, :1])
    if op in (0, 1):       # force heavy cancellation for a third of the operands
        k = count // 3
        b[:k, 0] = -a[:k, 0] if op == 0 else a[:k, 0]
    out = np.zeros_like(a)
    mw_op(op, words, count, a, b, out)
    name = {0: "add", 1: "sub", 2: "mul", 3: "div", 4: "sqrt"}[op]
    for i in range(count):
        ref = fr(oracle.scalar(name, a[i], b[i]))
        got = fr(out[i])
        if op in (0, 1):
            # accurate addition: error relative to the exact result (or to the operands after cancellation)
            scale = max(abs(ref), abs(fr(a[i])) * 2.0**-(53 * words - 10))
        else:
            scale = abs(ref)
        assert abs(got - ref) <= BOUND[words][op] * scale, (op, i)


@pytest.mark.parametrize("words", [2, 4])
@pytest.mark.parametrize("op", [0, 1, 2, 3, 4, 5, 6])
def test_host_multiword_ops_within_published_bounds(zkq, words, op):
    check_host_op(lambda *args: zkq.zkq_mw_op(*args, on_device=False), words, op)


def test_empty_batches_return_ok_before_any_device_work(zkq):
    """Empty batches are valid and return ZKQ_OK at once: no CUDA call, no use of the context beyond the
    null check (a zeroed stand-in handle is passed; the machine has no GPU, so any CUDA call would fail)."""
    L = zkq.lib()
    buf = ctypes.create_string_buffer(1 << 16)
    ctx = ctypes.addressof(buf)
    one = (ctypes.c_int32 * 1)(8)
    off = (ctypes.c_int64 * 1)(0)
    assert L.zkq_eigh_batched(ctx, 0, None, None, None, 4, None, None, None, None) == zkq.ZKQ_OK
    assert L.zkq_rqi_refine(ctx, 0, None, None, None, 4, None, None, 4, 1, None, None, None, None, None) == zkq.ZKQ_OK
    assert L.zkq_mw_gemm(ctx, 0, None, None, None, None, None, None, 4, None, None, 4, None, None, 4, 200, 1,
                         None) == zkq.ZKQ_OK
    nb = ctypes.c_size_t(7)
    assert L.zkq_workspace_size(ctx, 0, None, 4, 4, 1, ctypes.byref(nb)) == zkq.ZKQ_OK and nb.value == 0
    assert L.zkq_eigh_batched_noalloc(0, None, None, None, 4, None, None, None, None) == zkq.ZKQ_OK
    assert L.zkq_mw_op(0, 4, 0, None, None, None, 1, None) == zkq.ZKQ_OK
    # argument errors still come first
    assert L.zkq_eigh_batched(ctx, 0, None, None, None, 3, None, None, None, None) == zkq.ZKQ_EINVAL
    assert L.zkq_rqi_refine(ctx, 0, None, None, None, 4, None, None, 3, 1, None, None, None, None, None) == zkq.ZKQ_EINVAL
    assert L.zkq_eigh_batched(ctx, -1, one, off, None, 4, None, None, None, None) == zkq.ZKQ_EINVAL


def test_header_is_plain_c_and_links(zkq, tmp_path):
    """include/zkq.h is a C header (C99, no C++ constructs, every declaration a plain function of
    pointers and sizes): a C program that includes it and takes the address of every declared entry
    point compiles with -Wall -Werror, links against libzkq.so, and calls the entry points that need no
    GPU."""
    syms = declared_symbols()
    body = "\n".join(f"  table[{i}] = (void (*)(void)){s};" for i, s in enumerate(syms))
    src = tmp_path / "c_abi.c"
    src.write_text(f"""#include <stdio.h>
#include <string.h>
#include "zkq.h"
int main(void) {{
  void (*table[{len(syms)}])(void);
{body}
  size_t b = 0;
  if (zkq_workspace_size(NULL, 1, NULL, 4, 4, ZKQ_OA_OZAKI, &b) != ZKQ_EINVAL) return 1;
  if (strncmp(zkq_status_string(ZKQ_OK), "ZKQ_OK", 6) != 0) return 2;
  if (zkq_profile_classes() < 1) return 3;
  printf("%d\\n", (int)(sizeof(table) / sizeof(table[0])));
  return 0;
}}
""")
    exe = tmp_path / "c_abi"
    libdir = os.path.dirname(zkq.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    f"-I{os.path.join(ROOT, 'include')}", str(src), f"-L{libdir}", "-lzkq", f"-Wl,-rpath,{libdir}",
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert int(out.stdout.strip()) == len(syms)


def test_binding_has_every_entry_point_under_its_c_name(zkq):
    """The Python binding offers each declared entry point under the same name (argument marshalling
    only); the GPU-free ones return what the library returns."""
    missing = [s for s in declared_symbols() if not callable(getattr(zkq, s, None))]
    assert not missing, missing
    assert zkq.zkq_status_string(zkq.ZKQ_EINVAL).startswith("ZKQ_EINVAL")
    assert zkq.zkq_profile_classes() >= 1 and zkq.zkq_profile_class_name(0) == "jacobi"
    assert isinstance(zkq.zkq_last_cuda_error(), int)
