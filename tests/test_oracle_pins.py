"""Pins for the oracle against things other than itself: exact rationals, closed forms, mpmath,
invariants.  CPU only."""
from __future__ import annotations

from decimal import Decimal, getcontext
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._util import (conj_herm_product, dyadic_unitary, exact_words_ok, fr, to_words_matrix, words, cmul,
                         cconj, cadd)

TWO = Fraction(2)


def rel_close(x: Fraction, y: Fraction, bits: int) -> bool:
    scale = max(abs(y), Fraction(1, 2**1000))
    return abs(x - y) <= scale / TWO**bits


# ------------------------------- the 320-bit arithmetic itself ------------------------------------
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_mp_scalar_ops_match_exact_rationals(op):
    rng = np.random.default_rng(11)
    for trial in range(300):
        # random 4-word expansions with assorted exponents (cancellation-prone for add/sub)
        a = [float(x) for x in rng.standard_normal(1)] 
        e = int(rng.integers(-60, 60))
        a = [math.ldexp(float(rng.standard_normal()), e)]
        a += [a[-1] * 2**-55 * float(rng.standard_normal()) for _ in range(3)]
        if trial % 3 == 0:   # near-cancellation partner
            b = [-a[0]] + [math.ldexp(float(rng.standard_normal()), e - 70 - k * 50) for k in range(3)]
        else:
            eb = int(rng.integers(-60, 60))
            b = [math.ldexp(float(rng.standard_normal()), eb)]
            b += [b[-1] * 2**-55 * float(rng.standard_normal()) for _ in range(3)]
        if trial % 5 == 4:   # full-width operands: 6 words span ~318 of the 320 mantissa bits
            a = a[:1] + [a[0] * 2.0**(-53 * k) * (1 + float(rng.uniform(0, 0.5))) for k in range(1, 6)]
            b = b[:1] + [b[0] * 2.0**(-53 * k) * (1 + float(rng.uniform(0, 0.5))) for k in range(1, 6)]
        A, B = fr(a), fr(b)
        got = fr(oracle.scalar(op, a, b))
        exact = {"add": A + B, "sub": A - B, "mul": A * B, "div": A / B if B else None}[op]
        if exact is None:
            continue
        # each operand converts exactly (span < 320 bits); the result is within a few ulps of 2^-320
        assert rel_close(got, exact, 312), (op, trial)


def test_mp_sqrt_matches_integer_sqrt():
    rng = np.random.default_rng(12)
    for _ in range(200):
        e = int(rng.integers(-400, 400))
        a = [math.ldexp(abs(float(rng.standard_normal())) + 1e-3, e)]
        a += [a[0] * 2**-56 * float(rng.standard_normal()) for _ in range(2)]
        A = fr(a)
        s = fr(oracle.scalar("sqrt", a))
        # compare s^2 with A: relative error of s ~ half that of s^2
        assert rel_close(s * s, A, 310)


def test_mp_word_roundtrip_is_exact():
    rng = np.random.default_rng(13)
    for _ in range(200):
        x = Fraction(int(rng.integers(1, 2**62)), 2**int(rng.integers(0, 200))) * (1 + Fraction(1, 2**100))
        w = words(x, 6)
        out = np.zeros(6)
        oracle._load().oracle_rewords(1, np.ascontiguousarray(w).ctypes.data, 6, out.ctypes.data, 6)
        assert fr(out) == fr(w)


# ------------------------------- the eigensolver ---------------------------------------------------
def test_eigh_2x2_closed_form():
    getcontext().prec = 130
    rng = np.random.default_rng(21)
    for _ in range(20):
        a, d = Fraction(float(rng.standard_normal())), Fraction(float(rng.standard_normal()))
        br, bi = Fraction(float(rng.standard_normal())), Fraction(float(rng.standard_normal()))
        M = [[(a, Fraction(0)), (br, bi)], [(br, -bi), (d, Fraction(0))]]
        A = to_words_matrix(M, 2)
        lam, V, _ = oracle.eigh(A, 2)
        mid = (a + d) / 2
        q = ((a - d) / 2) ** 2 + br * br + bi * bi
        rad = (Decimal(q.numerator) / Decimal(q.denominator)).sqrt()
        exp_hi = Decimal(mid.numerator) / Decimal(mid.denominator) + rad
        exp_lo = Decimal(mid.numerator) / Decimal(mid.denominator) - rad
        for got, want in ((lam[0], exp_hi), (lam[1], exp_lo)):
            g = fr(got)
            assert abs(Decimal(g.numerator) / Decimal(g.denominator) - want) <= Decimal(2) ** -300 * (abs(exp_hi) + abs(exp_lo))


@pytest.mark.parametrize("n,seed", [(3, 1), (6, 2), (9, 3), (12, 4)])
def test_eigh_exact_known_spectrum(n, seed):
    """A = U diag(lam) U^H with U exactly unitary (dyadic) and dyadic lam spanning 2^0 .. 2^-230,
    including a negative and an exactly repeated eigenvalue: every eigenvalue to 2^-300 ||A||."""
    U = dyadic_unitary(n, layers=3 * n, seed=seed)
    lam = [Fraction(1)] + [Fraction((-1) ** k * (2 * k + 1), 2 ** (23 * k)) for k in range(1, n)]
    lam[-1] = lam[-2]                                 # exact double eigenvalue
    A = conj_herm_product(U, lam)
    Aw = to_words_matrix(A, 8)
    assert exact_words_ok(A, Aw, 8)
    got, V, _ = oracle.eigh(Aw, n)
    want = sorted(lam, reverse=True)
    for g, w_ in zip(got, want):
        assert abs(fr(g) - w_) <= Fraction(1, 2**300)
    res, orth = oracle.residual(Aw, n, got, V)
    assert res.max() < 2.0**-295 and orth.max() < 2.0**-300


def test_eigh_eigenvectors_of_distinct_spectrum_match_exact_columns():
    n = 6
    U = dyadic_unitary(n, layers=20, seed=9)
    lam = [Fraction(1, 2**(40 * k)) * (1 + Fraction(k, 8)) for k in range(n)]
    A = conj_herm_product(U, lam)
    Aw = to_words_matrix(A, 8)
    assert exact_words_ok(A, Aw, 8)
    got, V, _ = oracle.eigh(Aw, n)
    order = sorted(range(n), key=lambda k: -lam[k])
    for c, k in enumerate(order):
        u = [U[i][k] for i in range(n)]
        v = [(fr(V[i + c * n, 0]), fr(V[i + c * n, 1])) for i in range(n)]
        # phase-align: ph = <u, v>/|<u, v>|, compare |v - ph u|^2 via exact inner products
        ip = (Fraction(0), Fraction(0))
        for i in range(n):
            ip = cadd(ip, cmul(cconj(u[i]), v[i]))
        mag2 = ip[0] ** 2 + ip[1] ** 2
        vv = sum(a * a + b * b for a, b in v)
        # sin^2(angle(u, v)) = 1 - |<u,v>|^2 / (|u|^2 |v|^2), |u| = 1 exactly; Davis-Kahan with the
        # solver's absolute accuracy 2^-300 ||A|| over the gap to the nearest other eigenvalue
        gap = min(abs(lam[k] - lam[j]) for j in range(n) if j != k)
        assert 1 - mag2 / vv <= (Fraction(1, 2**300) / gap) ** 2
        assert abs(vv - 1) <= Fraction(1, 2**310)


def test_eigh_matches_mpmath_eighe():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    for n, seed in ((5, 31), (8, 32)):
        p = W.herm_spectrum(seed, 0, W.spectrum_graded(n, 120), 4)
        M = mpmath.matrix(n, n)
        for i in range(n):
            for j in range(n):
                re = fr(p.A[i + j * n, 0]); im = fr(p.A[i + j * n, 1])
                M[i, j] = mpmath.mpc(mpmath.mpf(re.numerator) / re.denominator, mpmath.mpf(im.numerator) / im.denominator)
        E, Q = mpmath.eighe(M)
        ref = sorted([E[i] for i in range(n)], reverse=True)
        got, V, _ = oracle.eigh(p.A, n)
        for g, r in zip(got, ref):
            gf = fr(g)
            assert abs(mpmath.mpf(gf.numerator) / gf.denominator - r) < mpmath.mpf(2) ** -300


def test_eigh_trace_and_invariants_on_generated_batch_problem():
    lam, lo, pairs, w = W.batch_problem_spec(2, 1, 0, 24)
    p = W.herm_spectrum(1, 0, lam, w, lam_lo=lo, pairs=pairs)
    got, V, sweeps = oracle.eigh(p.A, 24)
    tr = sum(fr(p.A[i + i * 24, 0]) for i in range(24))
    assert abs(sum(fr(g) for g in got) - tr) <= Fraction(1, 2**300)
    res, orth = oracle.residual(p.A, 24, got, V)
    assert res.max() < 2.0**-290 and orth.max() < 2.0**-300
    # the generator keeps the near-degenerate pairs split (relative 2^-60 here) up to the rounding of
    # A to quad-double words (absolute ~n 2^-212 ||A||)
    vals = [fr(g) for g in got]
    for (a, b) in pairs:
        split = vals[a] - vals[b]
        want = Fraction(float(lam[a])) / 2**60
        assert abs(split - want) <= want * Fraction(1, 2**40) + Fraction(24, 2**212)


def test_eigh_rejects_non_hermitian():
    A = np.zeros((4, 2, 1)); A[1, 0, 0] = 1.0  # a_10 = 1, a_01 = 0
    with pytest.raises(RuntimeError):
        oracle.eigh(A, 2)


# ------------------------------- footnote closed form ---------------------------------------------
@pytest.mark.parametrize("n", [2, 10, 60, 120, 180])
def test_eigh_footnote_reduced_matrix_u_is_z(n):
    """Footnote: C^{n-1}-Z on |+..+>|-> leaves the target with eigenvalues 1 - 2^-(n-1) and 2^-(n-1)."""
    p = Fraction(1, 2 ** (n - 1))
    # reduced state of the target: (1 - p)|-><-| + p|+><+| (Z|-> = |+>), with |+-><+-| = 1/2 [[1, +-1], [+-1, 1]]
    rho = [[((1 - p) * Fraction(1, 2) + p * Fraction(1, 2), Fraction(0)), ((1 - p) * Fraction(-1, 2) + p * Fraction(1, 2), Fraction(0))],
           [((1 - p) * Fraction(-1, 2) + p * Fraction(1, 2), Fraction(0)), ((1 - p) * Fraction(1, 2) + p * Fraction(1, 2), Fraction(0))]]
    # embed in a larger exactly-unitary conjugation so the solver does real work
    U = dyadic_unitary(4, layers=10, seed=n)
    blk = [[rho[0][0], rho[0][1], (Fraction(0), Fraction(0)), (Fraction(0), Fraction(0))],
           [rho[1][0], rho[1][1], (Fraction(0), Fraction(0)), (Fraction(0), Fraction(0))],
           [(Fraction(0),) * 2, (Fraction(0),) * 2, (Fraction(1, 4), Fraction(0)), (Fraction(0),) * 2],
           [(Fraction(0),) * 2, (Fraction(0),) * 2, (Fraction(0),) * 2, (Fraction(1, 8), Fraction(0))]]
    A = [[(Fraction(0), Fraction(0))] * 4 for _ in range(4)]
    for i in range(4):
        for j in range(4):
            s = (Fraction(0), Fraction(0))
            for k in range(4):
                for l in range(4):
                    s = cadd(s, cmul(cmul(U[i][k], blk[k][l]), cconj(U[j][l])))
            A[i][j] = s
    Aw = to_words_matrix(A, 8)
    assert exact_words_ok(A, Aw, 8)
    got, _, _ = oracle.eigh(Aw, 4)
    vals = sorted([1 - p, p, Fraction(1, 4), Fraction(1, 8)], reverse=True)
    for g, v in zip(got, vals):
        assert abs(fr(g) - v) <= Fraction(1, 2**300)


# ------------------------------- statevector --------------------------------------------------------
def _exact_pm_state(n):
    """|+>^{n-1}|-> for even n: every amplitude is +-2^(-n/2) exactly."""
    amps = np.zeros((1 << n, 2, 1))
    a = 2.0 ** (-n / 2)
    for x in range(1 << n):
        amps[x, 0, 0] = -a if (x & 1) else a      # target = site n-1 = least significant bit
    return amps


@pytest.mark.parametrize("n", [4, 8, 12])
def test_statevector_footnote_schmidt_values_u_is_z(n):
    sv = oracle.Statevector(n)
    sv.set(_exact_pm_state(n))
    rng = np.random.default_rng(n)
    ctrl = [int(b) for b in rng.integers(0, 2, n)]
    ctrl[-1] = -1
    Z = np.zeros((4, 2, 1)); Z[0, 0, 0] = 1.0; Z[3, 0, 0] = -1.0
    sv.apply_mcu(n - 1, ctrl, Z)
    lam2 = sv.schmidt2(n - 1)      # cut between controls and target: target side (2 values)
    eps = Fraction(1, 2 ** (n - 1))
    assert abs(fr(lam2[0]) - (1 - eps)) <= Fraction(1, 2**300)
    assert abs(fr(lam2[1]) - eps) <= Fraction(1, 2**300)


def test_statevector_footnote_general_u():
    n = 10
    sv = oracle.Statevector(n)
    sv.set(_exact_pm_state(n))
    G = W.haar_gate(77, 0, w=4, dim=2)
    ctrl = [1, 0, 1, 1, 0, 0, 1, 0, 1, -1]
    sv.apply_mcu(n - 1, ctrl, G)
    lam2 = sv.schmidt2(n - 1)
    p = Fraction(1, 2 ** (n - 1))
    u = [(fr(G[0, 0]), fr(G[0, 1])), (fr(G[1, 0]), fr(G[1, 1])), (fr(G[2, 0]), fr(G[2, 1])), (fr(G[3, 0]), fr(G[3, 1]))]
    # |u> = U|->, scaled by sqrt2: (u00 - u01, u10 - u11); |u><u| carries the 1/2
    v0 = (u[0][0] - u[1][0], u[0][1] - u[1][1]); v1 = (u[2][0] - u[3][0], u[2][1] - u[3][1])
    r00 = (1 - p) / 2 + p * (v0[0] ** 2 + v0[1] ** 2) / 2
    r11 = (1 - p) / 2 + p * (v1[0] ** 2 + v1[1] ** 2) / 2
    off = cmul(v0, cconj(v1)); r01 = (-(1 - p) / 2 + p * off[0] / 2, p * off[1] / 2)
    getcontext().prec = 130
    D = lambda f: Decimal(f.numerator) / Decimal(f.denominator)
    tr, det = r00 + r11, r00 * r11 - r01[0] ** 2 - r01[1] ** 2
    rad = (D(tr) ** 2 / 4 - D(det)).sqrt()
    want = (D(tr) / 2 + rad, D(tr) / 2 - rad)
    for g, w_ in zip(lam2, want):
        assert abs(D(fr(g)) - w_) < Decimal(2) ** -300
    # unitary U: closed form 1/2 (1 +- sqrt(1 - 4 p (1-p) (1 - |f|^2))) within U's rounding (2^-200)
    f = cmul((Fraction(1, 2), Fraction(0)), (u[0][0] - u[1][0] - u[2][0] + u[3][0], u[0][1] - u[1][1] - u[2][1] + u[3][1]))
    f2 = f[0] ** 2 + f[1] ** 2
    closed = (1 + (1 - 4 * D(p) * (1 - D(p)) * (1 - D(f2))).sqrt()) / 2
    assert abs(D(fr(lam2[0])) - closed) < Decimal(2) ** -200


def test_statevector_ghz_and_norm_and_reversibility():
    n = 6
    sv = oracle.Statevector(n)
    # exactly unitary dyadic 4x4 gate and its exact inverse
    U = dyadic_unitary(4, layers=7, seed=5)
    G = to_words_matrix([[U[c][r] for r in range(4)] for c in range(4)], 4)   # row-major r*4+c
    Gh = to_words_matrix([[cconj(U[r][c]) for r in range(4)] for c in range(4)], 4)
    amps0 = np.zeros((1 << n, 2, 1)); amps0[0, 0, 0] = 0.5; amps0[5, 1, 0] = -0.5; amps0[17, 0, 0] = 0.5; amps0[40, 0, 0] = 0.5
    sv.set(amps0)
    for s in (0, 2, 4, 1, 3):
        sv.apply2(s, G)
    assert abs(fr(sv.norm2()) - 1) <= Fraction(1, 2**300)
    for s in (3, 1, 4, 2, 0):
        sv.apply2(s, Gh)
    back = sv.amplitudes()
    for x in range(1 << n):
        for part in range(2):
            assert abs(fr(back[x, part]) - Fraction(float(amps0[x, part, 0]))) <= Fraction(1, 2**300)


def test_mps_amplitudes_ghz():
    """GHZ-shaped Vidal MPS with identity-like Gammas and dyadic weights: amplitudes are the products
    of the weights along the two branches."""
    n = 3
    half = 0.5
    chi = [2, 2]
    g0 = np.zeros((2 * 1 * 2, 2, 1)); g0[0 * 2 + 0, 0, 0] = 1; g0[1 * 2 + 1, 0, 0] = 1
    g1 = np.zeros((2 * 2 * 2, 2, 1)); g1[(0 * 2 + 0) * 2 + 0, 0, 0] = 1; g1[(1 * 2 + 1) * 2 + 1, 0, 0] = 1
    g2 = np.zeros((2 * 2 * 1, 2, 1)); g2[(0 * 2 + 0), 0, 0] = 1; g2[(1 * 2 + 1), 0, 0] = 1
    lam = np.array([[1.0], [1.0], [half], [1.0]])
    amps = oracle.mps_amplitudes(n, chi, np.concatenate([g0, g1, g2]), lam, 1)
    for x in range(8):
        # psi(000) = 1 * 1 * 1 * lam1[0] * 1 = 1/2, psi(111) = 1 * 1 * 1 * lam1[1] * 1 = 1
        want = Fraction(1, 2) if x == 0 else (Fraction(1) if x == 7 else Fraction(0))
        assert fr(amps[x, 0]) == want and fr(amps[x, 1]) == 0


def test_matmul_matches_exact_rationals():
    rng = np.random.default_rng(41)
    m, n, k = 3, 4, 5
    A = np.zeros((m * k, 2, 2)); B = np.zeros((k * n, 2, 2))
    for X in (A, B):
        X[:, :, 0] = rng.standard_normal(X.shape[:2])
        X[:, :, 1] = X[:, :, 0] * 2**-60 * rng.standard_normal(X.shape[:2])
    C = oracle.matmul(A, B, m, n, k)
    for i in range(m):
        for j in range(n):
            s = (Fraction(0), Fraction(0))
            for l in range(k):
                s = cadd(s, cmul((fr(A[i + l * m, 0]), fr(A[i + l * m, 1])), (fr(B[l + j * k, 0]), fr(B[l + j * k, 1]))))
            assert abs(fr(C[i + j * m, 0]) - s[0]) <= Fraction(1, 2**300)
            assert abs(fr(C[i + j * m, 1]) - s[1]) <= Fraction(1, 2**300)
    Ch = oracle.matmul(A, A, k, k, m, opA=1)    # A^H A
    for i in range(k):
        for j in range(k):
            s = (Fraction(0), Fraction(0))
            for l in range(m):
                s = cadd(s, cmul(cconj((fr(A[l + i * m, 0]), fr(A[l + i * m, 1]))), (fr(A[l + j * m, 0]), fr(A[l + j * m, 1]))))
            assert abs(fr(Ch[i + j * k, 0]) - s[0]) <= Fraction(1, 2**300)
            assert abs(fr(Ch[i + j * k, 1]) - s[1]) <= Fraction(1, 2**300)


def test_residual_and_orthonormality_match_exact_values():
    """The 320-bit residual ||A v_c - lambda_c v_c||_2 and the orthonormality defect max_d |v_d^H v_c -
    delta_dc| against values known exactly.  The eigenvectors u_k of A = U diag(lam) U^H (U exactly
    unitary) are perturbed in chosen ways:
    * v_2 = u_2 + eps u_3 has residual eps |lam_3 - lam_2| and defect eps against column 3;
    * lambda_0 shifted by delta gives residual delta in column 0;
    * exact pairs give residual and defect 0."""
    n = 5
    U = dyadic_unitary(n, layers=12, seed=17)
    lam = [Fraction(3), Fraction(1, 2), Fraction(-1, 4), Fraction(1, 2**20), Fraction(-5, 2**40)]
    A = conj_herm_product(U, lam)
    eps, delta = Fraction(1, 2**100), Fraction(3, 2**90)
    cols = [[U[i][k] for i in range(n)] for k in range(n)]
    cols[2] = [cadd(cols[2][i], (eps * U[i][3][0], eps * U[i][3][1])) for i in range(n)]
    V = [[cols[k][i] for k in range(n)] for i in range(n)]            # V[i][k]
    lam_given = list(lam)
    lam_given[0] = lam[0] + delta
    Aw, Vw = to_words_matrix(A, 8), to_words_matrix(V, 8)
    assert exact_words_ok(A, Aw, 8) and exact_words_ok(V, Vw, 8)
    lw = np.array([W.words_of(x, 8) for x in lam_given])
    res, orth = oracle.residual(Aw, n, lw, Vw)
    want_res = [float(delta), 0.0, float(eps * abs(lam[3] - lam[2])), 0.0, 0.0]
    want_orth = [0.0, 0.0, float(eps), float(eps), 0.0]
    for c in range(n):
        assert abs(res[c] - want_res[c]) <= 2.0**-280 + 2.0**-60 * want_res[c], (c, res[c], want_res[c])
        assert abs(orth[c] - want_orth[c]) <= 2.0**-280 + 2.0**-60 * want_orth[c], (c, orth[c], want_orth[c])
    # a column subset returns the same values in the requested order
    r2, o2 = oracle.residual(Aw, n, lw, Vw, cols=[3, 2])
    assert r2[0] == res[3] and r2[1] == res[2] and o2[1] == orth[2]


def test_footnote_golden_schmidt_values():
    """tests/golden/footnote_schmidt.txt: the paper's footnote example (Section 1) with U = Z, for the
    control sequences listed there; the squared Schmidt coefficients at the cut between the controls and
    the target are 1 - 2^e and 2^e (the state vector up to n = 12, the two-product Vidal form beyond)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "footnote_schmidt.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert rows
    Z = np.zeros((4, 2, 1)); Z[0, 0, 0] = 1.0; Z[3, 0, 0] = -1.0
    one, zero = Fraction(1), Fraction(0)
    for n_s, pattern, e_s in rows:
        n, e = int(n_s), int(e_s)
        assert len(pattern) == n - 1
        eps = Fraction(2) ** e
        ctrl = [int(c) for c in pattern]             # qubit n-1 .. qubit 1 are sites 0 .. n-2; the target is last
        if n <= 12:
            sv = oracle.Statevector(n)
            sv.set(_exact_pm_state(n))
            sv.apply_mcu(n - 1, ctrl + [-1], Z)
            l0, l1 = (fr(x) for x in sv.schmidt2(n - 1))
            tol = Fraction(1, 2**300)
        else:                                        # |+..+>|-> + |c> (Z - 1)|->, unnormalised, norm^2 2^n
            plus, minus = ((one, zero), (one, zero)), ((one, zero), (-one, zero))
            e_ = lambda b: (((one, zero), (zero, zero)) if b == 0 else ((zero, zero), (one, zero)))
            vecs = [[plus] * (n - 1) + [minus], [e_(b) for b in ctrl] + [((zero, zero), (Fraction(2), zero))]]
            V, C = _two_product_words(vecs, [(one, zero), (one, zero)])
            chi, _, lam = oracle.mps_two_products(V, C)
            tot = Fraction(2) ** n
            l0, l1 = fr(lam[-2]) ** 2 / tot, fr(lam[-1]) ** 2 / tot
            tol = Fraction(1, 2**290)                # Gram products and a 2 x 2 eigensolve per cut
        assert abs(l0 - (1 - eps)) <= tol, (n, pattern)
        assert abs(l1 - eps) <= tol, (n, pattern)


def _site_words(a, b, entry, w=8):
    """(2 a b, 2, w) words of Gamma (s, alpha, beta) row-major from entry(s, alpha, beta) -> (re, im)."""
    out = np.zeros((2 * a * b, 2, w))
    for s in range(2):
        for al in range(a):
            for be in range(b):
                re, im = entry(s, al, be)
                e = (s * a + al) * b + be
                out[e, 0, :] = words(re, w)
                out[e, 1, :] = words(im, w)
                assert fr(out[e, 0]) == re and fr(out[e, 1]) == im
    return out


@pytest.mark.parametrize("a,b,seed", [(3, 5, 2), (4, 4, 5), (2, 3, 8)])
def test_mps_site_defect_exact_isometries(a, b, seed):
    """Weighted isometries built from an exactly unitary complex U (Section 1: the tensors beside a bond are
    orthonormal in the weight of its Schmidt coefficients) have canonical defect exactly 0:
    * left: Gamma^s[alpha][beta] = U[s a + alpha][beta] / lam_alpha, so that the lam^2-weighted Gram of the
      columns is (U^H U) restricted to the first b columns;
    * right: Gamma^s[alpha][beta] = conj(U[s b + beta][alpha]) / lam_beta.
    Dyadic weights other than 1 make a weight taken once instead of squared fail, complex U makes a missing
    conjugate fail, and non-square shapes make swapped indices fail."""
    lamL = [Fraction(1, 2 ** k) for k in range(a)]
    lamR = [Fraction(1, 2 ** (2 * k)) for k in range(b)]
    lw = lambda v: np.array([words(x, 8) for x in v])
    if b <= 2 * a:
        U = dyadic_unitary(2 * a, layers=4 * a, seed=seed)
        g = _site_words(a, b, lambda s, al, be: (U[s * a + al][be][0] / lamL[al], U[s * a + al][be][1] / lamL[al]))
        assert oracle.mps_site_defect(a, b, g, lw(lamL), None, 8, 0) == 0.0
        assert oracle.mps_site_defect(a, b, g, None, None, 8, 0) > 0.1          # weights ignored: not orthonormal
    if a <= 2 * b:
        U = dyadic_unitary(2 * b, layers=4 * b, seed=seed + 1)
        g = _site_words(a, b, lambda s, al, be: (U[s * b + be][al][0] / lamR[be], -U[s * b + be][al][1] / lamR[be]))
        assert oracle.mps_site_defect(a, b, g, None, lw(lamR), 8, 1) == 0.0
        assert oracle.mps_site_defect(a, b, g, None, lw(lamR), 8, 0) > 0.1      # the other side's contraction


def test_mps_site_defect_closed_forms_and_sensitivity():
    """Sites of the GHZ state's Vidal form, Gamma^s[alpha][beta] = c delta_{alpha s} delta_{beta s} (2 x 2),
    whose left Gram is diag(c^2 lam_0^2, c^2 lam_1^2):
    * c = 1 with weights (1, 1/2): defect exactly 3/4;
    * the GHZ state itself, c = sqrt(2) and weights 1/sqrt(2), each rounded to 4 words: the Gram misses I
      only by that rounding (nonzero, below 2^-200).
    A 2^-90 change of one entry of an exact isometry shows up at that size."""
    ghz = lambda c: (lambda s, al, be: (c if (al == s and be == s) else Fraction(0), Fraction(0)))
    lam = np.array([words(Fraction(1), 8), words(Fraction(1, 2), 8)])
    assert oracle.mps_site_defect(2, 2, _site_words(2, 2, ghz(Fraction(1))), lam, None, 8, 0) == 0.75
    r = W.words_of(Fraction(math.isqrt(2 ** 501), 2 ** 250), 4)                # sqrt(2) in 4 words
    inv = np.concatenate([oracle.scalar("div", [1.0], r, 4), np.zeros(4)])        # 1 / sqrt(2) in 4 words
    d = oracle.mps_site_defect(2, 2, _site_words(2, 2, ghz(fr(r))), np.array([inv, inv]), None, 8, 0)
    assert 0.0 < d < 2.0 ** -200
    U = dyadic_unitary(6, layers=12, seed=21)
    base = lambda s, al, be: U[s * 3 + al][be]
    bump = Fraction(1, 2 ** 90)
    g2 = _site_words(3, 4, lambda s, al, be: (base(s, al, be)[0] + (bump if (s, al, be) == (1, 2, 0) else 0),
                                              base(s, al, be)[1]))
    d2 = oracle.mps_site_defect(3, 4, g2, None, None, 8, 0)
    assert 2.0 ** -96 < d2 < 2.0 ** -88


def test_statevector_gates_on_basis_states():
    """Gates applied to basis states give the gate's columns (the definition of a matrix acting on a basis
    vector), with the conventions of the oracle: site 0 is the most significant bit, a two-qubit gate on
    (site, site+1) has row index 2 i + j with i the bit of `site`, a controlled gate acts only where every
    control bit matches.  Complex dyadic gates keep everything exact."""
    n = 4
    U4 = dyadic_unitary(4, layers=6, seed=33)
    U2 = dyadic_unitary(2, layers=3, seed=34)
    # to_words_matrix stores M[i][j] at i + j dim: M[c][r] = U[r][c] puts U row-major at r dim + c
    G = to_words_matrix([[U4[r][c] for r in range(4)] for c in range(4)], 4)
    U = to_words_matrix([[U2[r][c] for r in range(2)] for c in range(2)], 4)
    bit = lambda site: 1 << (n - 1 - site)

    def run(x, op):
        sv = oracle.Statevector(n)
        amps = np.zeros((1 << n, 2, 1)); amps[x, 0, 0] = 1.0
        sv.set(amps)
        op(sv)
        out = sv.amplitudes()
        return {y: (fr(out[y, 0]), fr(out[y, 1])) for y in range(1 << n) if fr(out[y, 0]) or fr(out[y, 1])}

    rest = bit(0) | bit(3)                                   # spectator bits set, to catch stray indices
    for site in range(n - 1):
        for col in range(4):
            k, m = col >> 1, col & 1
            x = (rest & ~(bit(site) | bit(site + 1))) | (bit(site) if k else 0) | (bit(site + 1) if m else 0)
            got = run(x, lambda sv: sv.apply2(site, G))
            base = x & ~(bit(site) | bit(site + 1))
            want = {}
            for r in range(4):
                y = base | (bit(site) if r >> 1 else 0) | (bit(site + 1) if r & 1 else 0)
                if U4[r][col] != (0, 0):
                    want[y] = U4[r][col]
            assert got == want, (site, col)
    for site in range(n):
        for c in range(2):
            x = (rest & ~bit(site)) | (bit(site) if c else 0)
            got = run(x, lambda sv: sv.apply1(site, U))
            want = {((x & ~bit(site)) | (bit(site) if r else 0)): U2[r][c] for r in range(2) if U2[r][c] != (0, 0)}
            assert got == want, (site, c)
    # controlled U on target 2, controls: site 0 must be 1, site 3 must be 0, site 1 free
    ctrl = [1, -1, -1, 0]
    for x in range(1 << n):
        got = run(x, lambda sv: sv.apply_mcu(2, ctrl, U))
        if (x & bit(0)) and not (x & bit(3)):
            c = 1 if x & bit(2) else 0
            want = {((x & ~bit(2)) | (bit(2) if r else 0)): U2[r][c] for r in range(2) if U2[r][c] != (0, 0)}
        else:
            want = {x: (Fraction(1), Fraction(0))}
        assert got == want, x


def _site_views(n, chi, g, lam):
    """(a, b, Gamma words, left weights, right weights) of every site of a packed Vidal MPS."""
    dims = [1] + [int(c) for c in chi] + [1]
    out, go, lo = [], 0, 0
    for l in range(n):
        a, b = dims[l], dims[l + 1]
        left = lam[lo - a:lo] if l > 0 else None
        right = lam[lo:lo + b] if l < n - 1 else None
        out.append((a, b, g[go:go + 2 * a * b], left, right))
        go += 2 * a * b
        if l < n - 1:
            lo += b
    return out


def test_statevector_vidal_form_reproduces_the_state():
    """The oracle's Vidal MPS of an entangled 6-qubit state (exactly unitary dyadic gates on a brickwork of
    bonds): its amplitudes equal the state vector's to 2^-300, every site meets both canonical conditions
    to 2^-290, the squared weights at each bond are the Schmidt values of the state at that cut, and they
    sum to 1.  Three routes (state vector, MPS contraction, Schmidt values) must agree."""
    n = 6
    sv = oracle.Statevector(n)
    U4 = dyadic_unitary(4, layers=7, seed=5)
    G = to_words_matrix([[U4[r][c] for r in range(4)] for c in range(4)], 4)
    for s in (0, 2, 4, 1, 3, 0, 2):
        sv.apply2(s, G)
    chi, g, lam = sv.vidal()
    assert list(chi) == [2, 4, 8, 4, 2]
    amps = oracle.mps_amplitudes(n, chi, g, lam, oracle.WORDS)
    ref = sv.amplitudes()
    for x in range(1 << n):
        for p in range(2):
            assert abs(fr(amps[x, p]) - fr(ref[x, p])) <= Fraction(1, 2**300)
    for a, b, gl, left, right in _site_views(n, chi, g, lam):
        assert oracle.mps_site_defect(a, b, gl, left, None, oracle.WORDS, 0) <= 2.0**-290
        assert oracle.mps_site_defect(a, b, gl, None, right, oracle.WORDS, 1) <= 2.0**-290
    lo = 0
    for l, c in enumerate(chi):
        s2 = sv.schmidt2(l + 1)
        tot = Fraction(0)
        for k in range(c):
            lk2 = fr(lam[lo + k]) ** 2
            tot += lk2
            assert abs(lk2 - fr(s2[k])) <= Fraction(1, 2**290)
        assert abs(tot - 1) <= Fraction(1, 2**290)
        lo += c


def test_statevector_vidal_form_of_ghz_and_product_states():
    """(|0000> + |1111>) / 2, a GHZ state scaled by 1/sqrt(2), has bond dimension 2 and Schmidt weights
    (1/2, 1/2) at every bond; |0000> has bond dimension 1 and weight 1."""
    n = 4
    sv = oracle.Statevector(n)
    amps = np.zeros((1 << n, 2, 1)); amps[0, 0, 0] = 0.5; amps[(1 << n) - 1, 0, 0] = 0.5
    sv.set(amps)
    chi, g, lam = sv.vidal()
    assert list(chi) == [2, 2, 2]
    for k in range(6):
        assert abs(fr(lam[k]) - Fraction(1, 2)) <= Fraction(1, 2**300)
    sv0 = oracle.Statevector(n)
    chi0, g0, lam0 = sv0.vidal()
    assert list(chi0) == [1, 1, 1]
    assert all(fr(lam0[k]) == 1 for k in range(3))


def test_one_qubit_expectation_values_two_ways():
    """One-qubit expectation values: by definition from the state vector, and from the canonical Vidal MPS
    through one tensor and its Schmidt weights (Section 1: the MPS is a nested Schmidt decomposition, so the
    environments of a site reduce to its weights).  They agree to 2^-290 on an entangled complex state for
    Pauli X, Y, Z and a general complex 2x2 operator, Hermitian operators give real values, the identity
    gives the norm 1, and |0..0> and a GHZ state give their closed forms."""
    n = 6
    sv = oracle.Statevector(n)
    U4 = dyadic_unitary(4, layers=7, seed=5)
    G = to_words_matrix([[U4[r][c] for r in range(4)] for c in range(4)], 4)
    for s in (0, 2, 4, 1, 3, 0, 2):
        sv.apply2(s, G)
    chi, g, lam = sv.vidal()
    one, zero, half = Fraction(1), Fraction(0), Fraction(1, 2)
    ops = {"I": [[(one, zero), (zero, zero)], [(zero, zero), (one, zero)]],
           "X": [[(zero, zero), (one, zero)], [(one, zero), (zero, zero)]],
           "Y": [[(zero, zero), (zero, -one)], [(zero, one), (zero, zero)]],
           "Z": [[(one, zero), (zero, zero)], [(zero, zero), (-one, zero)]],
           "M": [[(half, Fraction(3, 4)), (Fraction(-1, 8), zero)], [(zero, Fraction(5, 16)), (Fraction(7, 2), -half)]]}
    words_of = {k: to_words_matrix([[v[r][c] for r in range(2)] for c in range(2)], 2) for k, v in ops.items()}
    for site in range(n):
        for name, O in words_of.items():
            a = sv.expect1(site, O)
            b = oracle.mps_expect1(n, chi, g, lam, oracle.WORDS, site, O)
            for part in range(2):
                assert abs(fr(a[part]) - fr(b[part])) <= Fraction(1, 2**290), (site, name, part)
            if name != "M":
                assert abs(fr(a[1])) <= Fraction(1, 2**300), (site, name)
            if name == "I":
                assert abs(fr(a[0]) - 1) <= Fraction(1, 2**300)
    z = words_of["Z"]
    sv0 = oracle.Statevector(n)
    for site in range(n):
        assert fr(sv0.expect1(site, z)[0]) == 1
    ghz = oracle.Statevector(4)
    amps = np.zeros((16, 2, 1)); amps[0, 0, 0] = 0.5; amps[15, 0, 0] = 0.5
    ghz.set(amps)
    for site in range(4):
        assert fr(ghz.expect1(site, z)[0]) == 0 and fr(ghz.expect1(site, words_of["X"])[0]) == 0
        assert fr(ghz.expect1(site, words_of["I"])[0]) == Fraction(1, 2)


def _cmat(words, rows, cols):
    """Fractions (re, im) M[i][j] of column-major complex words (rows*cols, 2, w)."""
    return [[(fr(words[i + j * rows, 0]), fr(words[i + j * rows, 1])) for j in range(cols)] for i in range(rows)]


@pytest.mark.parametrize("m,n,seed", [(5, 3, 3), (4, 4, 4), (2, 4, 6)])
def test_svd_of_exact_construction(m, n, seed):
    """M = U0 diag(sigma) V0^H with exactly unitary dyadic U0 (m x m), V0 (n x n) and dyadic singular values
    spanning 2^0..2^-120 (zeros beyond rank min(m, n)): the oracle's one-sided Jacobi returns the singular
    values to 2^-300, orthonormal U (on the nonzero values) and V to 2^-300, and M = U diag(sigma) V^H to
    2^-295; sigma^2 equal the eigenvalues of M^H M from the oracle's Hermitian eigensolver."""
    U0 = dyadic_unitary(m, layers=3 * m, seed=seed)
    V0 = dyadic_unitary(n, layers=3 * n, seed=seed + 50)
    r = min(m, n)
    sig = [Fraction(3, 2 ** (40 * k)) * (1 + Fraction(k, 4)) for k in range(r)]
    M = [[(Fraction(0), Fraction(0)) for _ in range(n)] for _ in range(m)]
    for i in range(m):
        for j in range(n):
            acc = (Fraction(0), Fraction(0))
            for k in range(r):
                acc = cadd(acc, cmul(U0[i][k], cmul((sig[k], Fraction(0)), cconj(V0[j][k]))))
            M[i][j] = acc
    Mw = to_words_matrix(M, 8)
    assert exact_words_ok(M, Mw, 8)
    s, U, V = oracle.svd(Mw, m, n)
    want = sorted(sig, reverse=True) + [Fraction(0)] * (n - r)
    for k in range(n):
        assert abs(fr(s[k]) - want[k]) <= Fraction(1, 2**300), k
    Uf, Vf = _cmat(U, m, n), _cmat(V, n, n)
    for c in range(n):
        for d in range(n):
            vv = (Fraction(0), Fraction(0))
            for i in range(n):
                vv = cadd(vv, cmul(cconj(Vf[i][c]), Vf[i][d]))
            assert abs(vv[0] - (1 if c == d else 0)) <= Fraction(1, 2**300) and abs(vv[1]) <= Fraction(1, 2**300)
            if c < r and d < r:
                uu = (Fraction(0), Fraction(0))
                for i in range(m):
                    uu = cadd(uu, cmul(cconj(Uf[i][c]), Uf[i][d]))
                assert abs(uu[0] - (1 if c == d else 0)) <= Fraction(1, 2**300) and abs(uu[1]) <= Fraction(1, 2**300)
    for i in range(m):
        for j in range(n):
            rec = (Fraction(0), Fraction(0))
            for k in range(r):
                rec = cadd(rec, cmul(Uf[i][k], cmul((fr(s[k]), Fraction(0)), cconj(Vf[j][k]))))
            assert abs(rec[0] - M[i][j][0]) <= Fraction(1, 2**295) and abs(rec[1] - M[i][j][1]) <= Fraction(1, 2**295)
    G = oracle.matmul(Mw, Mw, n, n, m, opA=1)          # M^H M
    lam, _, _ = oracle.eigh(G, n)
    for k in range(n):
        assert abs(fr(lam[k]) - fr(s[k]) ** 2) <= Fraction(1, 2**295)


def test_svd_of_rank_one_and_zero_matrices():
    """u v^H has the single singular value |u| |v| (here 3 * 5 / 4 exactly); the zero matrix has none."""
    u = [(Fraction(2), Fraction(1)), (Fraction(0), Fraction(-2)), (Fraction(0), Fraction(0))]      # |u| = 3
    v = [(Fraction(3, 4), Fraction(0)), (Fraction(0), Fraction(1))]                                 # |v| = 5/4
    M = [[cmul(u[i], cconj(v[j])) for j in range(2)] for i in range(3)]
    s, _, _ = oracle.svd(to_words_matrix(M, 4), 3, 2)
    assert abs(fr(s[0]) - Fraction(15, 4)) <= Fraction(1, 2**300) and abs(fr(s[1])) <= Fraction(1, 2**300)
    s0, U0, _ = oracle.svd(np.zeros((6, 2, 1)), 3, 2)
    assert fr(s0[0]) == 0 and fr(s0[1]) == 0 and not U0.any()


def _two_product_words(vecs, coef, w=8):
    """words arrays for oracle.mps_two_products from Fractions: vecs[t][l] = ((re0, im0), (re1, im1))."""
    n = len(vecs[0])
    V = np.zeros((2, n, 2, 2, w)); C = np.zeros((2, 2, w))
    for t in range(2):
        for l in range(n):
            for s in range(2):
                for p in range(2):
                    V[t, l, s, p] = words(vecs[t][l][s][p], w)
        for p in range(2):
            C[t, p] = words(coef[t][p], w)
    return V, C


def test_two_product_vidal_form_matches_the_state_vector():
    """The Vidal MPS of c_0 (x) v^0_l + c_1 (x) v^1_l built from Gram products (no state vector) equals, on
    8 qubits with Gaussian-dyadic local vectors, the oracle's state-vector route: the same Schmidt weights
    to 2^-290 and amplitudes to 2^-290 relative, and every site canonical."""
    rng = np.random.default_rng(8)
    n = 8
    q = lambda: Fraction(int(rng.integers(-64, 65)), 32)
    vecs = [[((q(), q()), (q(), q())) for _ in range(n)] for _ in range(2)]
    coef = [(Fraction(3, 4), Fraction(-1, 8)), (Fraction(5, 16), Fraction(1, 2))]
    V, C = _two_product_words(vecs, coef)
    chi, g, lam = oracle.mps_two_products(V, C)
    assert list(chi) == [2] * (n - 1)
    amps = []
    for x in range(1 << n):
        acc = (Fraction(0), Fraction(0))
        for t in range(2):
            term = coef[t]
            for l in range(n):
                term = cmul(term, vecs[t][l][(x >> (n - 1 - l)) & 1])
            acc = cadd(acc, term)
        amps.append(acc)
    sv = oracle.Statevector(n)
    sv.set(np.array([[words(a[0], 8), words(a[1], 8)] for a in amps]))
    _, _, lam_sv = sv.vidal()
    norm = sum(a * a + b * b for a, b in amps)
    for k in range(len(lam)):
        assert abs(fr(lam[k]) - fr(lam_sv[k])) <= Fraction(1, 2**290) * norm
    got = oracle.mps_amplitudes(n, chi, g, lam, oracle.WORDS)
    for x in range(1 << n):
        for p in range(2):
            assert abs(fr(got[x, p]) - amps[x][p]) <= Fraction(1, 2**290) * norm
    _check_canonical(n, chi, g, lam, norm, range(n))


def _check_canonical(n, chi, g, lam, norm2, sites):
    """Canonical conditions of an MPS of a state with squared norm norm2: both sides orthonormal, except
    that the outer weights are 1, so the right Gram of site 0 and the left Gram of site n-1 are norm2 I."""
    views = _site_views(n, chi, g, lam)
    for l in sites:
        a, b, gl, left, right = views[l]
        d0 = oracle.mps_site_defect(a, b, gl, left, None, oracle.WORDS, 0)
        d1 = oracle.mps_site_defect(a, b, gl, None, right, oracle.WORDS, 1)
        for d, edge in ((d0, l == n - 1), (d1, l == 0)):
            want = abs(float(norm2) - 1) if edge else 0.0
            assert abs(d - want) <= 2.0**-280 * float(norm2), (l, d, want)


@pytest.mark.parametrize("n", [6, 40, 180])
def test_footnote_state_vidal_form_at_large_n(n):
    """The paper's footnote example (Section 1) at qubit counts no state vector reaches: C^{n-1}-Z on
    |+>^{n-1}|-> (unnormalised, |+> = (1, 1), |-> = (1, -1), norm^2 2^n) is
    |+...+>|-> + |c> (Z - 1)|-> = |+...+>|-> + |c>(0, 2), a sum of two product states.  At the cut between the
    controls and the target its squared Schmidt coefficients are 2^n (1 - 2^-(n-1)) and 2^n 2^-(n-1), so the
    normalised ones are 1 - eps and eps with eps = 2^-(n-1), as the footnote states.  Sampled sites are
    canonical, and every bond has rank 2."""
    rng = np.random.default_rng(n)
    ctrl = [int(b) for b in rng.integers(0, 2, n - 1)]
    one, zero = Fraction(1), Fraction(0)
    plus, minus = ((one, zero), (one, zero)), ((one, zero), (-one, zero))
    e = lambda b: (((one, zero), (zero, zero)) if b == 0 else ((zero, zero), (one, zero)))
    vecs = [[plus] * (n - 1) + [minus], [e(b) for b in ctrl] + [((zero, zero), (Fraction(2), zero))]]
    V, C = _two_product_words(vecs, [(one, zero), (one, zero)])
    chi, g, lam = oracle.mps_two_products(V, C)
    assert list(chi) == [2] * (n - 1)
    last = lam[-2:]
    total = Fraction(2) ** n
    eps = Fraction(1, 2 ** (n - 1))
    assert abs(fr(last[0]) ** 2 / total - (1 - eps)) <= Fraction(1, 2**290)
    assert abs(fr(last[1]) ** 2 / total - eps) <= Fraction(1, 2**290)
    _check_canonical(n, chi, g, lam, total, sorted({0, 1, n // 2, n - 2, n - 1}))


@pytest.mark.parametrize("k,seed,general", [(1, 1, False), (2, 2, False), (4, 3, False), (5, 4, True), (6, 5, False)])
def test_footnote_circuit_equals_the_multi_controlled_gate(k, seed, general):
    """The nearest-neighbour circuit of the footnote's C^k-U (workloads.footnote_circuit, for an MPS
    simulation) acts on |+>^k |-> with its ancillas in |0> exactly as the multi-controlled gate itself
    (oracle state vector, apply_mcu): same amplitudes to 2^-300, ancillas back in |0>.  For U = Z the
    Schmidt coefficients at the cut before the target are then the footnote's 1 - 2^-k and 2^-k."""
    rng = np.random.default_rng(seed)
    ctrl = [int(b) for b in rng.integers(0, 2, k)]
    U = None
    if general:
        D = dyadic_unitary(2, layers=3, seed=seed)
        U = [[D[r][c] for c in range(2)] for r in range(2)]
    sites, gates = W.footnote_circuit(ctrl, U)
    assert sites == 2 * k and all(s + (2 if kind == "2q" else 1) <= sites for kind, s, _ in gates)
    pos = [0] + [2 * l - 1 for l in range(1, k)]
    target = 2 * k - 1
    amps = np.zeros((1 << sites, 2, 1))
    for x in range(1 << sites):
        bits = [(x >> (sites - 1 - q)) & 1 for q in range(sites)]
        if any(bits[q] for q in range(sites) if q not in pos and q != target):
            continue                                              # ancillas in |0>
        amps[x, 0, 0] = -1.0 if bits[target] else 1.0             # |+> = (1, 1) on controls, |-> = (1, -1)
    a = oracle.Statevector(sites); a.set(amps)
    for kind, s, G in gates:
        (a.apply2 if kind == "2q" else a.apply1)(s, G)
    b = oracle.Statevector(sites); b.set(amps)
    cl = [-1] * sites
    for l in range(k):
        cl[pos[l]] = ctrl[l]
    Uw = W._mat_words(U if U is not None else [[(1, 0), (0, 0)], [(0, 0), (-1, 0)]], 4)
    b.apply_mcu(target, cl, Uw)
    A, B = a.amplitudes(), b.amplitudes()
    for x in range(1 << sites):
        for p in range(2):
            assert abs(fr(A[x, p]) - fr(B[x, p])) <= Fraction(1, 2**300), (x, p)
    if not general:
        lam2 = a.schmidt2(sites - 1)                              # cut before the target: 2 values
        tot = fr(lam2[0]) + fr(lam2[1])
        eps = Fraction(1, 2 ** k)
        assert abs(fr(lam2[0]) / tot - (1 - eps)) <= Fraction(1, 2**290)
        assert abs(fr(lam2[1]) / tot - eps) <= Fraction(1, 2**290)


def test_footnote_circuit_state_is_the_two_product_vidal_state():
    """After the footnote circuit (k = 5 controls, ancillas back in |0>), the state is
    |+..+>|0..0>|-> + |c>|0..0> (Z - 1)|->, a sum of two product states: the oracle's two-product Vidal MPS of
    it reproduces the state vector's amplitudes to 2^-290, so it can stand in for the state vector at
    the qubit counts the device runs the circuit at."""
    k = 5
    ctrl = [1, 0, 1, 1, 0]
    sites, gates = W.footnote_circuit(ctrl)
    pos = [0] + [2 * l - 1 for l in range(1, k)]
    target = 2 * k - 1
    amps = np.zeros((1 << sites, 2, 1))
    for x in range(1 << sites):
        bits = [(x >> (sites - 1 - q)) & 1 for q in range(sites)]
        if any(bits[q] for q in range(sites) if q not in pos and q != target):
            continue
        amps[x, 0, 0] = -1.0 if bits[target] else 1.0
    sv = oracle.Statevector(sites); sv.set(amps)
    for kind, s, G in gates:
        (sv.apply2 if kind == "2q" else sv.apply1)(s, G)
    one, zero = Fraction(1), Fraction(0)
    e0, e1 = ((one, zero), (zero, zero)), ((zero, zero), (one, zero))
    plus, minus = ((one, zero), (one, zero)), ((one, zero), (-one, zero))
    t0 = [plus if q in pos else (minus if q == target else e0) for q in range(sites)]
    t1 = [(e1 if ctrl[pos.index(q)] else e0) if q in pos else
          (((zero, zero), (Fraction(2), zero)) if q == target else e0) for q in range(sites)]
    V, C = _two_product_words([t0, t1], [(one, zero), (one, zero)])
    chi, g, lam = oracle.mps_two_products(V, C)
    got = oracle.mps_amplitudes(sites, chi, g, lam, oracle.WORDS)
    ref = sv.amplitudes()
    for x in range(1 << sites):
        for p in range(2):
            assert abs(fr(got[x, p]) - fr(ref[x, p])) <= Fraction(1, 2**290) * 2 ** sites


def _entangled_state(n=6):
    sv = oracle.Statevector(n)
    U4 = dyadic_unitary(4, layers=7, seed=5)
    G = to_words_matrix([[U4[r][c] for r in range(4)] for c in range(4)], 4)
    for s in (0, 2, 4, 1, 3):
        sv.apply2(s, G)
    return sv


def test_mps_gate_update_matches_the_state_vector():
    """The oracle's two-site update of a Vidal MPS (theta contraction, one-sided Jacobi SVD of the reshaped
    tensor, split back; Section 2) applied to the Vidal form of an entangled 6-qubit state gives, at every
    bond, the state vector's amplitudes after the same gate to 2^-300, the Schmidt values of the new state
    at that cut, and canonical updated sites; the identity gate leaves the weights as they were."""
    n = 6
    sv = _entangled_state(n)
    chi, g, lam = sv.vidal()
    U4 = dyadic_unitary(4, layers=9, seed=11)
    G = to_words_matrix([[U4[r][c] for r in range(4)] for c in range(4)], 4)
    one, zero = Fraction(1), Fraction(0)
    I4 = to_words_matrix([[(one if r == c else zero, zero) for r in range(4)] for c in range(4)], 4)
    for site in range(n - 1):
        chi2, g2, lam2, disc = oracle.mps_apply2(n, chi, g, lam, oracle.WORDS, site, G)
        assert disc == 0.0
        ref = oracle.Statevector(n); ref.set(sv.amplitudes()); ref.apply2(site, G)
        got = oracle.mps_amplitudes(n, chi2, g2, lam2, oracle.WORDS)
        want = ref.amplitudes()
        for x in range(1 << n):
            for p in range(2):
                assert abs(fr(got[x, p]) - fr(want[x, p])) <= Fraction(1, 2**300), (site, x)
        s2 = ref.schmidt2(site + 1)
        lo = int(sum(chi2[:site]))
        for k in range(int(chi2[site])):
            assert abs(fr(lam2[lo + k]) ** 2 - fr(s2[k])) <= Fraction(1, 2**290)
        _check_canonical(n, chi2, g2, lam2, 1, [site, site + 1])
        chi3, _, lam3, _ = oracle.mps_apply2(n, chi, g, lam, oracle.WORDS, site, I4)
        assert list(chi3) == list(chi)
        for k in range(len(lam)):
            assert abs(fr(lam3[k]) - fr(lam[k])) <= Fraction(1, 2**300)


def test_mps_gate_update_truncation_keeps_the_schmidt_fidelity():
    """Truncating the updated bond to its leading Schmidt value (r_max = 1) reports the discarded weight
    1 - sigma_0^2 / sum sigma^2, renormalises (weight 1, norm 1), and leaves a state whose overlap with the
    exact one is |<psi|psi_1>|^2 = sigma_0^2 / sum sigma^2, the fidelity of a Schmidt truncation."""
    n = 6
    sv = _entangled_state(n)
    chi, g, lam = sv.vidal()
    U4 = dyadic_unitary(4, layers=9, seed=11)
    G = to_words_matrix([[U4[r][c] for r in range(4)] for c in range(4)], 4)
    site = 2
    chi1, g1, lam1, disc = oracle.mps_apply2(n, chi, g, lam, oracle.WORDS, site, G, r_max=1)
    assert chi1[site] == 1 and abs(fr(lam1[int(sum(chi1[:site]))]) - 1) <= Fraction(1, 2**300)
    ref = oracle.Statevector(n); ref.set(sv.amplitudes()); ref.apply2(site, G)
    s2 = ref.schmidt2(site + 1)
    tot = sum(fr(x) for x in s2)
    keep = fr(s2[0]) / tot
    assert abs(Fraction(disc) - (1 - keep)) <= Fraction(1, 2**50)
    got = oracle.mps_amplitudes(n, chi1, g1, lam1, oracle.WORDS)
    want = ref.amplitudes()
    norm = sum(fr(got[x, 0]) ** 2 + fr(got[x, 1]) ** 2 for x in range(1 << n))
    assert abs(norm - 1) <= Fraction(1, 2**290)
    ov = (Fraction(0), Fraction(0))
    for x in range(1 << n):
        ov = cadd(ov, cmul(cconj((fr(want[x, 0]), fr(want[x, 1]))), (fr(got[x, 0]), fr(got[x, 1]))))
    assert abs(ov[0] ** 2 + ov[1] ** 2 - keep) <= Fraction(1, 2**280)


def test_mps_sampling_follows_the_born_rule():
    """Chain-rule sampling from the canonical Vidal MPS of an entangled 6-qubit state: every bit string x is
    returned for uniform numbers inside its inverse-CDF cell (built here from the state vector's |psi_x|^2
    in the same site order), with the probability |psi_x|^2 to 2^-290; and the cells' lengths sum to 1."""
    n = 6
    sv = _entangled_state(n)
    chi, g, lam = sv.vidal()
    amp = sv.amplitudes()
    p = [fr(amp[x, 0]) ** 2 + fr(amp[x, 1]) ** 2 for x in range(1 << n)]
    assert abs(sum(p) - 1) <= Fraction(1, 2**290)

    def marginal(prefix):                                   # sum of p over strings starting with prefix
        k = len(prefix)
        base = sum(b << (n - 1 - i) for i, b in enumerate(prefix))
        return sum(p[base + r] for r in range(1 << (n - k)))

    for x in range(1 << n):
        if p[x] < Fraction(1, 2**200):
            continue
        bits = [(x >> (n - 1 - i)) & 1 for i in range(n)]
        u = []
        for k in range(n):                                  # midpoint of the cell of bit k given the prefix
            m_all, m0 = marginal(bits[:k]), marginal(bits[:k] + [0])
            lo, hi = (Fraction(0), m0 / m_all) if bits[k] == 0 else (m0 / m_all, Fraction(1))
            u.append(float((lo + hi) / 2))
        got, prob = oracle.mps_sample(n, chi, g, lam, oracle.WORDS, u)
        assert list(got) == bits, x
        assert abs(fr(prob) - p[x]) <= Fraction(1, 2**290), x


# ------------------------------- Deutsch-Jozsa-style circuits -----------------------------------------
@pytest.mark.parametrize("kind", ["balanced", "constant"])
def test_dj_circuit_state_and_graph_state_schmidt_values(kind):
    """The Deutsch-Jozsa-style circuit (workloads.dj_circuit, Section 3.1 with a specified function family)
    on the 320-bit state vector: a balanced f leaves input 0 in |1> (so the all-zeros outcome has probability
    0, the algorithm's answer), a constant f returns every input to |0>; the ancilla stays |->.  Before the
    final Hadamards the inputs hold the graph state of the band graph, and every Schmidt value at every cut
    is 2^-r with r the GF(2) rank of oracle.graph_state_schmidt_rank (also after the Hadamards, which are
    local)."""
    n, w = 9, 3
    sites, gates, edges = W.dj_circuit(n, w, kind, seed=5, wds=8)
    assert edges
    sv = oracle.Statevector(n)
    for g_kind, s, G in gates:
        (sv.apply2 if g_kind == "2q" else sv.apply1)(s, G)
    Zop = np.zeros((4, 2, 1)); Zop[0, 0, 0] = 1.0; Zop[3, 0, 0] = -1.0
    for q in range(n - 1):
        z = fr(sv.expect1(q, Zop)[0])
        if kind == "balanced" and q == 0:
            assert abs(z + 1) <= Fraction(1, 2**290)
        elif kind == "constant":
            assert abs(z - 1) <= Fraction(1, 2**290)
    Xop = np.zeros((4, 2, 1)); Xop[1, 0, 0] = Xop[2, 0, 0] = 1.0
    assert abs(fr(sv.expect1(n - 1, Xop)[0]) + 1) <= Fraction(1, 2**290)      # ancilla in |->
    for cut in range(1, n):
        r = oracle.graph_state_schmidt_rank(n - 1, edges, cut) if cut < n - 1 else 0
        if kind == "constant":
            r = 0
        s2 = sv.schmidt2(cut)
        for b in range(s2.shape[0]):
            want = Fraction(1, 2**r) if b < 2**r else Fraction(0)
            assert abs(fr(s2[b]) - want) <= Fraction(1, 2**280), (cut, b, r)


def test_graph_state_schmidt_rank_closed_forms():
    """GF(2) ranks of small cuts: a path has rank 1 at every cut; the complete bipartite cut has rank 1; a
    perfect matching across the cut has rank = its size; no edge across gives 0."""
    path = [(i, i + 1) for i in range(5)]
    assert all(oracle.graph_state_schmidt_rank(6, path, c) == 1 for c in range(1, 6))
    kb = [(i, j) for i in range(3) for j in range(3, 6)]
    assert oracle.graph_state_schmidt_rank(6, kb, 3) == 1
    match = [(0, 5), (1, 4), (2, 3)]
    assert oracle.graph_state_schmidt_rank(6, match, 3) == 3
    assert oracle.graph_state_schmidt_rank(6, [(0, 1), (4, 5)], 3) == 0
