"""Property tests of the double-double and quad-double arithmetic (the library's header, compiled for the
host, run through zkq_mw_op) with generated operands (hypothesis): values with up to 53 W + 8 significant
bits at exponents -300..300, rounded to W words, including partners that cancel their leading words and
expansions with wide gaps between words.  Sums, differences, products and quotients meet the published
bounds against exact rational results; square roots square back within twice the bound.  CPU only."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from tests._util import fr
from tests.test_abi_cpu import BOUND

hyp = pytest.importorskip("hypothesis")
st = hyp.strategies


@pytest.fixture(scope="module")
def zkq():
    import paper_2402_11868_gb300 as Z
    Z.build()
    return Z


def _value(words):
    return st.builds(lambda m, e, s: Fraction(s * m) * Fraction(2) ** e,
                     st.integers(1, 2 ** (53 * words + 8)), st.integers(-300, 300), st.sampled_from([-1, 1]))


@pytest.mark.parametrize("words", [2, 4])
def test_multiword_ops_meet_their_bounds_on_generated_operands(zkq, words):
    @hyp.settings(max_examples=600, deadline=None, derandomize=True, suppress_health_check=list(hyp.HealthCheck))
    @hyp.given(x=_value(words), y=_value(words), op=st.sampled_from([0, 1, 2, 3, 4]), cancel=st.booleans())
    def check(x, y, op, cancel):
        if cancel and op in (0, 1):                  # a partner equal to -x (add) or x (sub) up to a small part
            y = (-x if op == 0 else x) + y * Fraction(2) ** -(53 * words // 2)
        a = np.array([W.words_of(abs(x) if op == 4 else x, words)])
        b = np.array([W.words_of(y, words)])
        A, B = fr(a[0]), fr(b[0])
        hyp.assume(not (op == 3 and B == 0))
        out = np.zeros_like(a)
        zkq.zkq_mw_op(op, words, 1, a, b, out, on_device=False)
        got = fr(out[0])
        if op == 4:
            assert abs(got * got - A) <= 2 * Fraction(BOUND[words][4]) * A * Fraction(101, 100)
            return
        exact = {0: A + B, 1: A - B, 2: A * B, 3: A / B if B else 0}[op]
        # accurate addition: the error is relative to the exact result, or to the operands after cancellation
        scale = max(abs(exact), abs(A) * Fraction(2) ** -(53 * words - 10)) if op in (0, 1) else abs(exact)
        assert abs(got - exact) <= Fraction(BOUND[words][op]) * scale

    check()
