"""Property tests of the oracle's 320-bit arithmetic with generated operands (hypothesis): sums, differences,
products and quotients of expansions of up to 4 doubles, at any exponents and with exact cancellations,
equal the exact rational results within 2^-312 relative; square roots square back within 2^-310.
Operands whose words span more than the 318 bits one value holds, and results whose 6-word expansion
would leave the normal double range, are outside what the oracle represents and are skipped.  CPU only."""
from __future__ import annotations

import math
from fractions import Fraction

import pytest

import oracle
from tests._util import fr

hyp = pytest.importorskip("hypothesis")
st = hyp.strategies

DBL = st.floats(allow_nan=False, allow_infinity=False, width=64)
WORDS = st.lists(DBL, min_size=1, max_size=4)
SETTINGS = hyp.settings(max_examples=800, deadline=None, derandomize=True,
                        suppress_health_check=list(hyp.HealthCheck))


def _span_ok(ws):
    nz = [x for x in ws if x != 0]
    if not nz:
        return True
    es = [math.frexp(x)[1] for x in nz]
    return max(es) - min(es) + 53 <= 318


def _in_range(x: Fraction) -> bool:
    return x == 0 or Fraction(1, 2**700) <= abs(x) <= Fraction(2) ** 1000


@SETTINGS
@hyp.given(a=WORDS, b=WORDS, op=st.sampled_from(["add", "sub", "mul", "div"]))
def test_arithmetic_matches_exact_rationals(a, b, op):
    hyp.assume(_span_ok(a) and _span_ok(b))
    A, B = fr(a), fr(b)
    hyp.assume(not (op == "div" and B == 0))
    exact = {"add": A + B, "sub": A - B, "mul": A * B, "div": A / B if B else None}[op]
    hyp.assume(_in_range(exact))
    got = fr(oracle.scalar(op, a, b))
    if exact == 0:
        assert got == 0
    else:
        assert abs(got - exact) <= abs(exact) / 2**312


@hyp.settings(max_examples=400, deadline=None, derandomize=True, suppress_health_check=list(hyp.HealthCheck))
@hyp.given(a=WORDS)
def test_square_root_squares_back(a):
    hyp.assume(_span_ok(a))
    A = fr(a)
    hyp.assume(A > 0 and _in_range(A) and A >= Fraction(1, 2**600))
    s = fr(oracle.scalar("sqrt", a))
    assert abs(s * s - A) <= A / 2**310
