"""Helpers shared by the tests: exact rational views of word expansions, exactly unitary dyadic
matrices (for known-spectrum pins), and tolerance bookkeeping."""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import workloads as W


def fr(words) -> Fraction:
    return sum((Fraction(float(x)) for x in np.asarray(words).ravel()), Fraction(0))


def words(x: Fraction, w: int) -> list[float]:
    return W.words_of(Fraction(x), w)


def cfr(elem) -> tuple[Fraction, Fraction]:
    """(re, im) of one complex element given as (2, w) words."""
    return fr(elem[0]), fr(elem[1])


def to_words_matrix(M, w):
    """M: list of lists of (re, im) Fractions, M[i][j]; returns (n*m, 2, w) column-major words."""
    n, m = len(M), len(M[0])
    out = np.zeros((n * m, 2, w))
    for j in range(m):
        for i in range(n):
            re, im = M[i][j]
            out[i + j * n, 0, :] = W.words_of(re, w)
            out[i + j * n, 1, :] = W.words_of(im, w)
    return out


def exact_words_ok(M, A, w):
    n, m = len(M), len(M[0])
    for j in range(m):
        for i in range(n):
            re, im = M[i][j]
            if fr(A[i + j * n, 0]) != re or fr(A[i + j * n, 1]) != im:
                return False
    return True


# ---- exactly unitary matrices with Gaussian-dyadic entries ----------------------------------------
HALF = Fraction(1, 2)
# 2-level blocks: sqrt(X) = 1/2 [[1+i, 1-i], [1-i, 1+i]], phase diag(1, i), and their products
_SQX = [[(HALF, HALF), (HALF, -HALF)], [(HALF, -HALF), (HALF, HALF)]]


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def cconj(a):
    return (a[0], -a[1])


def dyadic_unitary(n: int, layers: int, seed: int):
    """Exactly unitary n x n matrix: product of `layers` random 2-level sqrt(X) gates with random
    phases in {1, i, -1, -i}.  Entries are Gaussian dyadic rationals."""
    rng = np.random.default_rng(seed)
    U = [[(Fraction(int(i == j)), Fraction(0)) for j in range(n)] for i in range(n)]
    phases = [(Fraction(1), Fraction(0)), (Fraction(0), Fraction(1)), (Fraction(-1), Fraction(0)), (Fraction(0), Fraction(-1))]
    for _ in range(layers):
        p, q = rng.choice(n, size=2, replace=False)
        ph = phases[int(rng.integers(4))]
        # U <- B U with B acting on rows p, q: B = diag(1, ph) * sqrtX
        rp, rq = U[p], U[q]
        newp = [cadd(cmul(_SQX[0][0], rp[j]), cmul(_SQX[0][1], rq[j])) for j in range(n)]
        newq = [cmul(ph, cadd(cmul(_SQX[1][0], rp[j]), cmul(_SQX[1][1], rq[j]))) for j in range(n)]
        U[p], U[q] = newp, newq
    return U


def conj_herm_product(U, lam):
    """A = U diag(lam) U^H exactly (lam: list of Fractions)."""
    n = len(U)
    A = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            s = (Fraction(0), Fraction(0))
            for k in range(n):
                t = cmul(U[i][k], cconj(U[j][k]))
                s = cadd(s, (t[0] * lam[k], t[1] * lam[k]))
            A[i][j] = s
    return A
