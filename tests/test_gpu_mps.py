"""MPS gate updates (theta contraction, Gram eigensolve, truncation, split back) against the 320-bit
state vector, the footnote's tiny Schmidt coefficient, and norm preservation."""
from __future__ import annotations

from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W
from tests._util import fr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2402_11868_gb300 as Z
    Z.build()
    c = Z.Context(0)
    yield c
    c.close()


def mps_amps(mps):
    chi, g, lam = mps.download()
    return oracle.mps_amplitudes(mps.n, chi, g, lam.reshape(-1, mps.words) if len(lam) else np.zeros((1, mps.words)),
                                 mps.words), chi, lam


@pytest.mark.parametrize("method_name", ["ZKQ_OA_OZAKI", "ZKQ_PLAIN_RQI"])
def test_brickwork_matches_statevector(ctx, method_name):
    import paper_2402_11868_gb300 as Z
    method = getattr(Z, method_name)
    n, depth = 7, 5
    circ = W.brickwork_circuit(17, n, depth, w=4)
    mps = Z.MPS(ctx, n, r_max=64, words=4)
    sv = oracle.Statevector(n)
    for site, G in circ:
        mps.apply2q(site, G, trunc_tau=2.0**-200, method=method)
        sv.apply2(site, G)
    amps, chi, lam = mps_amps(mps)
    ref = sv.amplitudes()
    worst = max(abs(fr(amps[x, p]) - fr(ref[x, p])) for x in range(1 << n) for p in range(2))
    assert worst <= Fraction(1, 2**185), float(worst)
    # every bond's lambda^2 sums to 1 and equals the oracle's Schmidt values at that cut
    off = 0
    for l, c in enumerate(chi):
        vals = [fr(lam[off + b]) for b in range(c)]
        off += c
        assert abs(sum(v * v for v in vals) - 1) <= Fraction(1, 2**195)
        s2 = sv.schmidt2(l + 1)
        for b in range(c):
            assert abs(vals[b] ** 2 - fr(s2[b])) <= Fraction(1, 2**190), (l, b)


def test_single_qubit_gates_and_product_state(ctx):
    import paper_2402_11868_gb300 as Z
    n = 5
    mps = Z.MPS(ctx, n, r_max=8, words=4)
    sv = oracle.Statevector(n)
    for s in range(n):
        U = W.haar_gate(40, s, w=4, dim=2)
        mps.apply1q(s, U)
        sv.apply1(s, U)
    G = W.haar_gate(41, 0, w=4)
    mps.apply2q(1, G, trunc_tau=2.0**-200)
    sv.apply2(1, G)
    amps, _, _ = mps_amps(mps)
    ref = sv.amplitudes()
    worst = max(abs(fr(amps[x, p]) - fr(ref[x, p])) for x in range(1 << n) for p in range(2))
    assert worst <= Fraction(1, 2**190), float(worst)


def _tiny_schmidt_gates(eps: Fraction, w: int):
    """R_y-type rotation with sin^2 = eps on site 0 (entries rounded to w words) and an exact CNOT."""
    getcontext().prec = 120
    a = (Decimal(1) - Decimal(eps.numerator) / Decimal(eps.denominator)).sqrt()
    b = (Decimal(eps.numerator) / Decimal(eps.denominator)).sqrt()
    U = np.zeros((4, 2, w))
    U[0, 0, :] = W.words_of(Fraction(a), w); U[1, 0, :] = W.words_of(-Fraction(b), w)
    U[2, 0, :] = W.words_of(Fraction(b), w); U[3, 0, :] = W.words_of(Fraction(a), w)
    CX = np.zeros((16, 2, w))
    for r, c in ((0, 0), (1, 1), (2, 3), (3, 2)):
        CX[r * 4 + c, 0, 0] = 1.0
    return U, CX


@pytest.mark.parametrize("n", [14, 60, 120, 180])
def test_footnote_tiny_schmidt_coefficient_survives_in_quad_double(ctx, n):
    """The footnote: a Schmidt coefficient sqrt(eps) with eps ~ 2^-(n-1) must be kept.  Quad-double keeps
    it (sum lambda^2 = 1, lambda_1^2 = eps within 2^-200); double-double truncates it (rank inflation /
    loss through limited precision, Section 1)."""
    import paper_2402_11868_gb300 as Z
    eps = Fraction(1, 2 ** (n - 1))
    U, CX = _tiny_schmidt_gates(eps, 4)
    mps = Z.MPS(ctx, n, r_max=4, words=4)
    mps.apply1q(0, U)
    chi_new, disc = mps.apply2q(0, CX, trunc_tau=2.0**-200)
    chi, g, lam = mps.download()
    assert chi_new == 2 and chi[0] == 2
    l0, l1 = fr(lam[0]), fr(lam[1])
    # U is unitary only to its rounding (2^-212): compare with its actual column norm
    a, b = fr(U[0, 0]), fr(U[2, 0])
    tot = a * a + b * b
    assert abs(l1 * l1 - b * b / tot) <= Fraction(1, 2**200)
    assert abs(l0 * l0 + l1 * l1 - 1) <= Fraction(1, 2**200)
    if n >= 60:
        # double-double resolves eigenvalues of rho down to ~2^-96 ||rho||: eps = 2^-59 survives, while
        # eps = 2^-119, 2^-179 fall below its null-space threshold and the bond collapses to rank 1
        U2, CX2 = _tiny_schmidt_gates(eps, 2)
        dd = Z.MPS(ctx, n, r_max=4, words=2)
        dd.apply1q(0, U2)
        chi_dd, _ = dd.apply2q(0, CX2, trunc_tau=2.0**-96)
        assert chi_dd == (2 if eps > Fraction(1, 2**96) else 1)


def test_truncation_renormalises_and_reports_discarded_weight(ctx):
    import paper_2402_11868_gb300 as Z
    n = 6
    circ = W.brickwork_circuit(23, n, 4, w=4)
    mps = Z.MPS(ctx, n, r_max=2, words=4)      # far below the exact rank: truncation on every bond
    for site, G in circ:
        chi, disc = mps.apply2q(site, G, trunc_tau=2.0**-200)
        assert chi <= 2 and 0.0 <= disc < 1.0
    chi, g, lam = mps.download()
    off = 0
    for c in chi:
        vals = [fr(lam[off + b]) for b in range(c)]
        off += c
        assert abs(sum(v * v for v in vals) - 1) <= Fraction(1, 2**195)
