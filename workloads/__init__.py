"""Seeded synthetic workloads for the accurate-eigensolve hot path.

This module only *generates inputs*: Hermitian matrices with a prescribed spectrum
(A = U diag(lambda) U^H, U Haar), Haar 4x4 gates and brickwork circuits.  It is shared by the
CUDA path (tests, bench) and by the oracle's tests, and contains none of the eigensolver's or the
multi-word arithmetic's steps.  The heavy part (exact accumulation of U diag(lambda) U^H) lives in
``gen.c`` and is compiled by :func:`build`.

Workload shapes follow the paper's setting (Hermitian diagonalisation of reduced matrices at every
two-qubit gate update, Section 2.1 and 2.2) with synthetic spectra:

* ``config_single128``: one N=128 problem, lambda_k = 2^(-0.3(k-1)), quad-double input.
* ``config_batch``: 256 problems, N uniform in {16, 32, ..., 512}; graded spectrum
  lambda_k = 2^(-G (k-1)/(N-1)) with G = 40 (double-double) or G = 180 (quad-double), plus 8
  near-degenerate pairs.
* brickwork circuits of Haar 4x4 gates for the MPS gate-update path.

Layout of a matrix returned here: float64 array of shape (n*n, 2, w); element (i, j) of the
column-major matrix is row ``i + j*n``; ``[.., 0, :]`` holds the real part's w words (highest first),
``[.., 1, :]`` the imaginary part's.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_gen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile gen.c into an in-tree shared library (plain C, no contraction, portable)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.gen_key.restype = ctypes.c_uint64
            lib.gen_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gen_uniform.restype = None
            lib.gen_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            lib.gen_cgauss.restype = None
            lib.gen_cgauss.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            lib.gen_herm_spectrum.restype = ctypes.c_int
            lib.gen_herm_spectrum.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p]
            _lib = lib
    return _lib


def key(seed: int, stream: int) -> int:
    return int(_load().gen_key(seed & (2**64 - 1), stream & (2**64 - 1)))


def uniform(seed: int, stream: int, count: int, first: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().gen_uniform(key(seed, stream), first, count, out.ctypes.data)
    return out


def cgauss(seed: int, stream: int, count: int) -> np.ndarray:
    """count standard complex Gaussians (E|z|^2 = 1) as complex128."""
    out = np.empty(2 * count, dtype=np.float64)
    _load().gen_cgauss(key(seed, stream), count, out.ctypes.data)
    return out[0::2] + 1j * out[1::2]


def words_of(x: Fraction, w: int) -> list[float]:
    """Successive round-to-nearest expansion of an exact rational into w doubles."""
    out = []
    for _ in range(w):
        d = float(x)
        out.append(d)
        x -= Fraction(d)
    return out


class Problem:
    """One Hermitian eigenproblem with a prescribed spectrum."""

    def __init__(self, n, A, lam, lam_lo, pairs, w):
        self.n, self.A, self.lam, self.lam_lo, self.pairs, self.w = n, A, lam, lam_lo, pairs, w

    @property
    def lam_exact(self):
        return [Fraction(float(a)) + Fraction(float(b)) for a, b in zip(self.lam, self.lam_lo)]


def herm_spectrum(seed: int, stream: int, lam, w: int, lam_lo=None, pairs=(), want_u: bool = False):
    """A = U diag(lam + lam_lo) U^H with U Haar (by seed/stream), rounded to w words per real.

    ``pairs`` lists (a, b) eigen-indices whose eigenvectors are built as u_b = J conj(u_a), which keeps
    the prescribed split lam_a - lam_b exact in the generated matrix.
    """
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    n = lam.shape[0]
    lo = None if lam_lo is None else np.ascontiguousarray(lam_lo, dtype=np.float64)
    pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1, 2))
    A = np.empty((n * n, 2, w), dtype=np.float64)
    U = np.empty(2 * n * n, dtype=np.float64) if want_u else None
    rc = _load().gen_herm_spectrum(key(seed, stream), n, lam.ctypes.data, None if lo is None else lo.ctypes.data,
                                   pr.shape[0], pr.ctypes.data if pr.size else None, w, A.ctypes.data,
                                   None if U is None else U.ctypes.data)
    if rc != 0:
        raise ValueError(f"gen_herm_spectrum failed ({rc})")
    p = Problem(n, A, lam, np.zeros(n) if lo is None else lo, [tuple(x) for x in pr], w)
    if want_u:
        p.U = (U[0::2] + 1j * U[1::2]).reshape(n, n).T  # U[i, k]
    return p


def _pow2_frac(num: int, den: int) -> float:
    """2^(num/den) rounded to double, computed in decimal so the bits do not depend on the C library."""
    getcontext().prec = 60
    return float(Decimal(2) ** (Decimal(num) / Decimal(den)))


def spectrum_single128(n: int = 128) -> np.ndarray:
    """lambda_k = 2^(-0.3 (k-1)), k = 1..n."""
    return np.array([_pow2_frac(-3 * k, 10) for k in range(n)])


def spectrum_graded(n: int, grade: int) -> np.ndarray:
    """lambda_k = 2^(-grade (k-1)/(n-1)), k = 1..n."""
    if n == 1:
        return np.array([1.0])
    return np.array([_pow2_frac(-grade * k, n - 1) for k in range(n)])


def config_single128(seed: int = 0, w: int = 4) -> Problem:
    """Single 128x128 problem, lambda_k = 2^(-0.3(k-1)), Haar U, quad-double input."""
    return herm_spectrum(seed, 0, spectrum_single128(128), w)


def batch_sizes(seed: int, count: int = 256, step: int = 16, smax: int = 512) -> list[int]:
    u = uniform(seed, 1 << 40, count)
    nsz = smax // step
    return [int(step * (1 + min(nsz - 1, int(x * nsz)))) for x in u]


def pair_indices(seed: int, idx: int, n: int, npairs: int = 8) -> list[tuple[int, int]]:
    """npairs non-overlapping adjacent (k, k+1) eigen-index pairs (0-based), drawn by seed.

    The exact-split construction needs an even order, so odd orders get no pairs."""
    if n % 2:
        return []
    # visit the candidate starts k = 0..n-2 in a seeded random order and keep non-overlapping ones
    u = uniform(seed, (2 << 40) + idx, max(n - 1, 1))
    order = sorted(range(n - 1), key=lambda k: (u[k], k))
    taken, out = set(), []
    for k in order:
        if len(out) == npairs:
            break
        if k in taken or (k + 1) in taken:
            continue
        taken.update((k, k + 1)); out.append((k, k + 1))
    return sorted(out)


def batch_problem_spec(cfg: int, seed: int, idx: int, n: int):
    """(lam, lam_lo, pairs, w) for problem idx of the 256-problem batch.

    cfg 1: grade 40, absolute pair split 2^-60, double-double input.
    cfg 2: grade 180, relative pair split lambda_k * 2^-60 (an absolute 2^-60 split would cross zero
    below 2^-60), quad-double input.
    """
    grade, w = (40, 2) if cfg == 1 else (180, 4)
    lam = spectrum_graded(n, grade)
    lo = np.zeros(n)
    pairs = pair_indices(seed, idx, n)
    for (a, b) in pairs:
        split = Fraction(1, 2**60) if cfg == 1 else Fraction(float(lam[a])) / 2**60
        v = Fraction(float(lam[a])) - split
        hi = float(v)
        lam[b], lo[b] = hi, float(v - Fraction(hi))
    return lam, lo, pairs, w


def config_batch(cfg: int, seed: int = 1, count: int = 256, sizes=None, threads: int | None = None,
                 indices=None) -> list[Problem]:
    """The uneven batch (cfg 1: double-double, grade 40; cfg 2: quad-double, grade 180)."""
    sizes = batch_sizes(seed, count) if sizes is None else list(sizes)
    indices = range(len(sizes)) if indices is None else indices

    def one(i):
        n = sizes[i]
        lam, lo, pairs, w = batch_problem_spec(cfg, seed, i, n)
        return herm_spectrum(seed, i, lam, w, lam_lo=lo, pairs=pairs)

    idx = list(indices)
    with ThreadPoolExecutor(max_workers=threads or min(32, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, idx))


# ----------------------------------------------------------------------------------------------------
# gates and circuits
def haar_gate(seed: int, index: int, w: int = 4, dim: int = 4):
    """Haar dim x dim unitary (Gram-Schmidt of a complex Gaussian in 80-digit decimal), as exact
    Fractions (re, im) rounded to w words: returns float64 array (dim*dim, 2, w), row-major (r*dim + c)."""
    z = cgauss(seed, (3 << 40) + index, dim * dim).reshape(dim, dim)   # z[r, c]
    getcontext().prec = 80
    cols = []
    for c in range(dim):
        v = [[Decimal(float(z[r, c].real)), Decimal(float(z[r, c].imag))] for r in range(dim)]
        for _ in range(2):
            for u in cols:
                pr = sum(u[r][0] * v[r][0] + u[r][1] * v[r][1] for r in range(dim))
                pi = sum(u[r][0] * v[r][1] - u[r][1] * v[r][0] for r in range(dim))
                for r in range(dim):
                    v[r][0] -= pr * u[r][0] - pi * u[r][1]
                    v[r][1] -= pr * u[r][1] + pi * u[r][0]
        nrm = sum(a * a + b * b for a, b in v).sqrt()
        cols.append([[a / nrm, b / nrm] for a, b in v])
    G = np.empty((dim * dim, 2, w))
    for r in range(dim):
        for c in range(dim):
            G[r * dim + c, 0, :] = words_of(Fraction(cols[c][r][0]), w)
            G[r * dim + c, 1, :] = words_of(Fraction(cols[c][r][1]), w)
    return G


def brickwork(n_qubits: int, depth: int):
    """Gate sites of a nearest-neighbour brickwork: layer t acts on (s, s+1) for s = t%2, t%2+2, ..."""
    sites = []
    for t in range(depth):
        sites.extend(range(t % 2, n_qubits - 1, 2))
    return sites


def brickwork_circuit(seed: int, n_qubits: int, depth: int, w: int = 4):
    """[(site, G)] with a fresh Haar gate per position, in seed order."""
    return [(s, haar_gate(seed, i, w)) for i, s in enumerate(brickwork(n_qubits, depth))]


# ----------------------------------------------------------------------------------------------------
# the footnote circuit: C^k-U on nearest-neighbour qubits with a ladder of ancillas
def _mat_words(M, w):
    """Row-major (dim*dim, 2, w) words of a square matrix of (re, im) Fractions."""
    dim = len(M)
    out = np.zeros((dim * dim, 2, w))
    for r in range(dim):
        for c in range(dim):
            out[r * dim + c, 0, :] = words_of(Fraction(M[r][c][0]), w)
            out[r * dim + c, 1, :] = words_of(Fraction(M[r][c][1]), w)
    return out


def _controlled(V):
    """4x4 controlled-V with the control on the first qubit of the pair (row index 2 i + j)."""
    z, o = (Fraction(0), Fraction(0)), (Fraction(1), Fraction(0))
    return [[o, z, z, z], [z, o, z, z], [z, z, V[0][0], V[0][1]], [z, z, V[1][0], V[1][1]]]


def footnote_circuit(ctrl, U=None, w: int = 4):
    """The multi-controlled gate of the paper's footnote example (Section 1), C^k-U with control pattern
    ctrl (k = len(ctrl) bits) and a target, as one- and two-qubit gates on neighbouring qubits only, for an
    MPS simulation.  Layout: control 0 at site 0, control l at site 2l - 1, ancilla l (starting in |0>)
    at site 2l, the target at site 2k - 1; 2k sites in all.  The ancillas hold the running AND of the
    controls through a ladder of Toffoli gates (Barenco et al. 1995: controlled-sqrt(X), CNOT, controlled-
    sqrt(X)^H, CNOT, controlled-sqrt(X), the last one between non-neighbours carried by two SWAPs), the last
    ancilla controls U on the target, and the ladder is undone.  Controls whose pattern bit is 0 are
    conjugated by X.  U: 2x2 of (re, im) Fractions, default Z.  All entries are dyadic, so the circuit is
    exact in binary.  Returns (sites, gates) with gates a list of ("1q" | "2q", site, words)."""
    k = len(ctrl)
    assert k >= 1
    z, o, h = Fraction(0), Fraction(1), Fraction(1, 2)
    if U is None:
        U = [[(o, z), (z, z)], [(z, z), (-o, z)]]
    X = [[(z, z), (o, z)], [(o, z), (z, z)]]
    SX = [[(h, h), (h, -h)], [(h, -h), (h, h)]]                      # sqrt(X)
    SXH = [[(h, -h), (h, h)], [(h, h), (h, -h)]]                     # its conjugate transpose
    Z0, O1 = (z, z), (o, z)
    CNOT = [[O1, Z0, Z0, Z0], [Z0, O1, Z0, Z0], [Z0, Z0, Z0, O1], [Z0, Z0, O1, Z0]]
    SWAP = [[O1, Z0, Z0, Z0], [Z0, Z0, O1, Z0], [Z0, O1, Z0, Z0], [Z0, Z0, Z0, O1]]
    g = lambda M: _mat_words(M, w)
    cv, cvh, cx, sw = g(_controlled(SX)), g(_controlled(SXH)), g(CNOT), g(SWAP)
    pos = [0] + [2 * l - 1 for l in range(1, k)]
    target = 2 * k - 1

    def toffoli(q):                                   # controls at q, q + 1; target q + 2
        return [("2q", q + 1, cv), ("2q", q, cx), ("2q", q + 1, cvh), ("2q", q, cx),
                ("2q", q, sw), ("2q", q + 1, cv), ("2q", q, sw)]

    flips = [("1q", pos[l], g(X)) for l in range(k) if ctrl[l] == 0]
    ladder = []
    for l in range(1, k):                             # ancilla l = (control 0 and ... and control l)
        ladder += toffoli(0 if l == 1 else 2 * l - 2)
    last = 0 if k == 1 else 2 * k - 2                 # the qubit that controls U, next to the target
    gates = flips + ladder + [("2q", last, g(_controlled(U)))] + ladder[::-1] + flips
    return 2 * k, gates


# ----------------------------------------------------------------------------------------------------
# Deutsch-Jozsa-style circuits (Section 3.1; the paper's function structure is not given, so a family is
# specified here): inputs on sites 0..n-2, the ancilla on site n-1.  The oracle is a phase oracle
# (-1)^f(x), equivalent to x, y -> x, y + f(x) with the ancilla in |->.
#   balanced: f(x) = x_0 + sum over edges (i, j) of x_i x_j (mod 2), no edge at input 0 -- balanced because
#             x_0 flips f, and after the final Hadamards input 0 is |1>, so the all-zeros outcome never occurs;
#   constant: the edge phases applied twice (f = 0), entangling in between.
# The edges form a band graph: each pair (i, j) with 1 <= j - i <= w is an edge with probability 1/2 (by
# seed).  Between the two layers of Hadamards the inputs hold a graph state, whose Schmidt coefficients at a
# cut are all equal, 2^(-r/2) with r the GF(2) rank of the cut's edge matrix, so the band width bounds the
# bond dimension (2^w) and with it the size of the matrices the gate updates diagonalise.
def dj_edges(n_inputs: int, w: int, seed: int):
    """Band-graph edges (i, j), 1 <= i < j <= i + w, on inputs 1..n_inputs-1, chosen by seed (input 0 carries
    the balancing term x_0 and no edge)."""
    u = uniform(seed, (7 << 40) + n_inputs * 64 + w, n_inputs * w)
    edges = []
    for i in range(1, n_inputs):
        for d in range(1, w + 1):
            if i + d < n_inputs and u[i * w + d - 1] < 0.5:
                edges.append((i, i + d))
    return edges


def dj_circuit(n: int, w: int, kind: str = "balanced", seed: int = 0, wds: int = 4):
    """(sites, gates, edges) of the Deutsch-Jozsa-style circuit on n sites (n - 1 inputs, ancilla last):
    X on the ancilla, H on every site, the phase oracle, H on the inputs.  A CZ on inputs i < j is carried to
    neighbours by SWAPs of j down to i + 1 and back.  Gates as in footnote_circuit: ("1q" | "2q", site, words).
    The H entries 2^-1/2 are rounded to wds words; every other entry is exact."""
    assert n >= 3 and kind in ("balanced", "constant")
    z, o = Fraction(0), Fraction(1)
    from decimal import Decimal, getcontext
    getcontext().prec = 200
    h = Fraction(Decimal(1) / Decimal(2).sqrt())
    H = [[(h, z), (h, z)], [(h, z), (-h, z)]]
    X = [[(z, z), (o, z)], [(o, z), (z, z)]]
    Zg = [[(o, z), (z, z)], [(z, z), (-o, z)]]
    Z0, O1, M1 = (z, z), (o, z), (-o, z)
    CZ = [[O1, Z0, Z0, Z0], [Z0, O1, Z0, Z0], [Z0, Z0, O1, Z0], [Z0, Z0, Z0, M1]]
    SWAP = [[O1, Z0, Z0, Z0], [Z0, Z0, O1, Z0], [Z0, O1, Z0, Z0], [Z0, Z0, Z0, O1]]
    g = lambda M: _mat_words(M, wds)
    Hw, Xw, Zw, CZw, SWw = g(H), g(X), g(Zg), g(CZ), g(SWAP)
    ni = n - 1
    edges = dj_edges(ni, w, seed)

    def phase_layer():
        out = []
        for (i, j) in edges:
            for q in range(j - 1, i, -1):           # bring qubit j next to i: SWAP (q, q+1) for q = j-1 .. i+1
                out.append(("2q", q, SWw))
            out.append(("2q", i, CZw))
            for q in range(i + 1, j):
                out.append(("2q", q, SWw))
        return out

    gates = [("1q", n - 1, Xw)] + [("1q", q, Hw) for q in range(n)]
    if kind == "balanced":
        gates += [("1q", 0, Zw)] + phase_layer()
    else:
        gates += phase_layer() + phase_layer()
    gates += [("1q", q, Hw) for q in range(ni)]
    return n, gates, edges
