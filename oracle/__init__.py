"""ORACLE: test infrastructure only.

Plain, slow, independent CPU implementation of what the accurate-eigensolve path computes:

* ``eigh``: cyclic-by-row complex Jacobi at 320 bits (the plain definition of Hermitian
  diagonalisation, the dominant cost named in Section 2.1 of the paper);
* ``residual``: ||A v - lambda v|| and ||V^H V - I|| at 320 bits;
* ``matmul``: plain 320-bit complex products (the refinement's dense products);
* ``Statevector``: brute-force state vector at 320 bits, plus Schmidt values at a cut and the
  amplitudes of a Vidal MPS (Section 1: MPS = nested Schmidt decomposition);
* ``mps_site_defect``: the Vidal canonical (weighted orthonormality) conditions of one MPS site, a
  property of every exact gate update that holds at any qubit count;
* ``Statevector.vidal``: the Vidal MPS of a state from its Schmidt decompositions at every cut;
* ``mps_two_products``: the Vidal MPS of a sum of two product states at any qubit count, such as the
  state of the paper's footnote example;
* ``mps_sample``: a bit string from the Born distribution of a canonical MPS by the chain rule;
* ``mps_apply2``: one two-site gate update of a Vidal MPS (theta, SVD, truncation, split back);
* ``svd``: one-sided Jacobi singular value decomposition at 320 bits (the SVD variant of the gate update);
* ``Statevector.expect1`` and ``mps_expect1``: one-qubit expectation values, from the state vector by
  definition and from a canonical MPS through its local tensor and Schmidt weights;
* ``graph_state_schmidt_rank``: the Schmidt rank of a graph state at a cut (GF(2) rank of the cut's
  edges), the closed form of the Deutsch-Jozsa-style circuits' Schmidt values (Section 3.1).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package.  It shares no code with the CUDA path; both receive their inputs from ``workloads``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_SRC = ["mp.c", "eigh.c", "statevec.c", "products.c", "svd.c", "mpsgate.c"]
_lib = None
_lock = threading.Lock()

WORDS = 6  # 6 doubles cover the 320-bit results


def compile_library(src_dir: str, out: str) -> str:
    """Compile the oracle's C sources found in src_dir into the shared library `out`."""
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", out]
                          + [os.path.join(src_dir, s) for s in _SRC] + ["-lm"])
    return out


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "mp.h")]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        compile_library(_HERE, tmp)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load_library(_SO)
    return _lib


def load_library(path: str):
    """ctypes handle of an oracle library with every entry point's signature set (the tests that plant
    mistakes in copies of the oracle load their builds through this, then swap `_lib`)."""
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.oracle_eigh.restype = I
    L.oracle_eigh.argtypes = [I, P, I, I, P, P, P]
    L.oracle_residual.restype = I
    L.oracle_residual.argtypes = [I, P, I, P, P, I, I, P, P, P]
    L.oracle_matmul.restype = I
    L.oracle_matmul.argtypes = [I, I, I, I, P, I, P, I, P, I]
    L.oracle_rewords.restype = None
    L.oracle_rewords.argtypes = [ctypes.c_long, P, I, P, I]
    L.oracle_scalar.restype = None
    L.oracle_scalar.argtypes = [I, P, P, I, P, I]
    L.oracle_sv_new.restype = P
    L.oracle_sv_new.argtypes = [I]
    L.oracle_sv_free.argtypes = [P]
    for nm in ("oracle_sv_apply1", "oracle_sv_apply2"):
        getattr(L, nm).restype = I
        getattr(L, nm).argtypes = [P, I, P, I]
    L.oracle_sv_apply_mcu.restype = I
    L.oracle_sv_apply_mcu.argtypes = [P, I, P, P, I]
    L.oracle_sv_set.argtypes = [P, P, I]
    L.oracle_sv_get.argtypes = [P, P, I]
    L.oracle_sv_norm2.argtypes = [P, P, I]
    L.oracle_sv_schmidt2.restype = I
    L.oracle_sv_schmidt2.argtypes = [P, I, P, I]
    L.oracle_mps_amplitudes.restype = I
    L.oracle_mps_amplitudes.argtypes = [I, P, P, P, I, P, I]
    L.oracle_mps_two_products.restype = I
    L.oracle_mps_two_products.argtypes = [I, P, P, I, I, P, P, P, I]
    L.oracle_mps_sample.restype = I
    L.oracle_mps_sample.argtypes = [I, P, P, P, I, P, P, P, I]
    L.oracle_mps_apply2.restype = I
    L.oracle_mps_apply2.argtypes = [I, P, P, P, I, I, P, I, I, I, P, P, P, I, ctypes.POINTER(D)]
    L.oracle_svd.restype = I
    L.oracle_svd.argtypes = [I, I, P, I, I, P, P, P]
    L.oracle_sv_expect1.restype = I
    L.oracle_sv_expect1.argtypes = [P, I, P, I, P, I]
    L.oracle_mps_expect1.restype = I
    L.oracle_mps_expect1.argtypes = [I, P, P, P, I, I, P, I, P, I]
    L.oracle_sv_vidal.restype = I
    L.oracle_sv_vidal.argtypes = [P, I, P, P, P, I]
    L.oracle_mps_site_defect.restype = I
    L.oracle_mps_site_defect.argtypes = [I, I, P, P, P, I, I, ctypes.POINTER(D)]
    return L


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def eigh(A: np.ndarray, n: int, w_out: int = WORDS):
    """Eigen-decomposition of the Hermitian n x n matrix given as words (n*n, 2, w).

    Returns (lam (n, w_out) descending, V (n*n, 2, w_out) column-major, sweeps)."""
    A = _c(A)
    w = A.shape[-1]
    lam = np.zeros((n, w_out))
    V = np.zeros((n * n, 2, w_out))
    sw = ctypes.c_int(0)
    rc = _load().oracle_eigh(n, A.ctypes.data, w, w_out, lam.ctypes.data, V.ctypes.data, ctypes.byref(sw))
    if rc != 0:
        raise RuntimeError(f"oracle_eigh failed with code {rc}")
    return lam, V, sw.value


def residual(A: np.ndarray, n: int, lam: np.ndarray, V: np.ndarray, cols=None):
    """(max-norm residual per column, orthonormality defect per column) at 320 bits."""
    A, lam, V = _c(A), _c(lam), _c(V)
    wv = V.shape[-1]
    if lam.shape[-1] != wv:
        lam2 = np.zeros((n, wv)); lam2[:, :min(wv, lam.shape[-1])] = lam[:, :min(wv, lam.shape[-1])]
        if lam.shape[-1] > wv:
            raise ValueError("lam has more words than V")
        lam = lam2
    cols_arr = None if cols is None else np.ascontiguousarray(cols, dtype=np.int32)
    nc = n if cols is None else len(cols_arr)
    res = np.zeros(nc); orth = np.zeros(nc)
    rc = _load().oracle_residual(n, A.ctypes.data, A.shape[-1], lam.ctypes.data, V.ctypes.data, wv, nc,
                                 None if cols_arr is None else cols_arr.ctypes.data, res.ctypes.data, orth.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_residual failed")
    return res, orth


def matmul(A, B, m, n, k, opA=0, w_out=WORDS):
    A, B = _c(A), _c(B)
    C = np.zeros((m * n, 2, w_out))
    rc = _load().oracle_matmul(m, n, k, opA, A.ctypes.data, A.shape[-1], B.ctypes.data, B.shape[-1], C.ctypes.data, w_out)
    if rc != 0:
        raise RuntimeError("oracle_matmul failed")
    return C


def scalar(op: str, a, b=(0.0,), w_out: int = WORDS):
    ops = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4}
    a = _c(a); b = _c(b)
    w = max(a.size, b.size)
    aa = np.zeros(w); aa[:a.size] = a
    bb = np.zeros(w); bb[:b.size] = b
    out = np.zeros(w_out)
    _load().oracle_scalar(ops[op], aa.ctypes.data, bb.ctypes.data, w, out.ctypes.data, w_out)
    return out


class Statevector:
    """2^n amplitudes at 320 bits."""

    def __init__(self, n: int):
        self.n = n
        self._h = _load().oracle_sv_new(n)
        if not self._h:
            raise ValueError("statevector size out of range")

    def __del__(self):
        if getattr(self, "_h", None):
            _load().oracle_sv_free(self._h)
            self._h = None

    def apply1(self, site, U):
        U = _c(U)
        assert _load().oracle_sv_apply1(self._h, site, U.ctypes.data, U.shape[-1]) == 0

    def apply2(self, site, G):
        G = _c(G)
        assert _load().oracle_sv_apply2(self._h, site, G.ctypes.data, G.shape[-1]) == 0

    def apply_mcu(self, target, ctrl, U):
        U = _c(U)
        c = np.ascontiguousarray(ctrl, dtype=np.int32)
        assert _load().oracle_sv_apply_mcu(self._h, target, c.ctypes.data, U.ctypes.data, U.shape[-1]) == 0

    def set(self, amps):
        amps = _c(amps)
        _load().oracle_sv_set(self._h, amps.ctypes.data, amps.shape[-1])

    def amplitudes(self, w=WORDS):
        out = np.zeros((1 << self.n, 2, w))
        _load().oracle_sv_get(self._h, out.ctypes.data, w)
        return out

    def norm2(self, w=WORDS):
        out = np.zeros(w)
        _load().oracle_sv_norm2(self._h, out.ctypes.data, w)
        return out

    def expect1(self, site, O, w=WORDS):
        """<psi| O_site |psi> for a 2x2 operator O given as words (4, 2, wo), row-major: (re words, im words)."""
        O = _c(O)
        out = np.zeros((2, w))
        if _load().oracle_sv_expect1(self._h, site, O.ctypes.data, O.shape[-1], out.ctypes.data, w):
            raise ValueError("bad site")
        return out

    def vidal(self, tol_log2=200, w=WORDS):
        """Vidal MPS of the state (chi, gammas (elements, 2, w), lambdas (values, w)) in the layout of
        mps_amplitudes, from the Schmidt decomposition at every cut; Schmidt values with lambda^2 at or below
        2^-tol_log2 lambda_0^2 are dropped."""
        n = self.n
        cmax = [1 << min(c, n - c) for c in range(n + 1)]
        ge = sum(2 * cmax[l] * cmax[l + 1] for l in range(n))
        chi = np.zeros(n - 1, dtype=np.int32)
        gam = np.zeros((ge, 2, w)); lam = np.zeros((sum(cmax[1:n]), w))
        rc = _load().oracle_sv_vidal(self._h, tol_log2, chi.ctypes.data, gam.ctypes.data, lam.ctypes.data, w)
        if rc:
            raise RuntimeError(f"oracle_sv_vidal failed ({rc})")
        dims = [1] + [int(c) for c in chi] + [1]
        used = sum(2 * dims[l] * dims[l + 1] for l in range(n))
        return chi, gam[:used], lam[:int(chi.sum())]

    def schmidt2(self, cut, w=WORDS):
        m = 1 << min(cut, self.n - cut)
        out = np.zeros((m, w))
        rc = _load().oracle_sv_schmidt2(self._h, cut, out.ctypes.data, w)
        if rc:
            raise RuntimeError("schmidt2 failed")
        return out


def mps_amplitudes(n, chi, gammas, lambdas, w, w_out=WORDS):
    """Amplitudes (2^n, 2, w_out) of the Vidal MPS (Gamma tensors (s, alpha, beta) row-major, lambda
    vectors), both as concatenated word arrays."""
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    g = _c(gammas); l = _c(lambdas) if len(lambdas) else np.zeros(1)
    out = np.zeros((1 << n, 2, w_out))
    rc = _load().oracle_mps_amplitudes(n, chi.ctypes.data, g.ctypes.data, l.ctypes.data, w, out.ctypes.data, w_out)
    if rc:
        raise RuntimeError(f"oracle_mps_amplitudes failed ({rc})")
    return out


def mps_site_defect(a, b, gamma, lam_left, lam_right, w, side):
    """max |G - I| of the Vidal canonical Gram matrix of one site (Section 1: the MPS is a nested Schmidt
    decomposition).  gamma: (2 a b, 2, w) words of Gamma (s, alpha, beta) row-major; lam_left (a, w) and
    lam_right (b, w) words or None (all 1).  side 0: sum over s, alpha of lam_left^2 Gamma^H Gamma (b x b);
    side 1: sum over s, beta of Gamma lam_right^2 Gamma^H (a x a)."""
    g = _c(gamma)
    assert g.size == 2 * a * b * 2 * w
    lp = [None if x is None else _c(x) for x in (lam_left, lam_right)]
    out = ctypes.c_double()
    rc = _load().oracle_mps_site_defect(a, b, g.ctypes.data, None if lp[0] is None else lp[0].ctypes.data,
                                        None if lp[1] is None else lp[1].ctypes.data, w, side, ctypes.byref(out))
    if rc:
        raise ValueError("bad arguments to oracle_mps_site_defect")
    return out.value


def mps_two_products(vecs, coef, tol_log2=200, w_out=WORDS):
    """Vidal MPS (chi, gammas, lambdas; the layout of mps_amplitudes) of psi = coef[0] (x)_l vecs[0][l] +
    coef[1] (x)_l vecs[1][l], at any number of sites: vecs (2, n, 2, 2, w) words of the local 2-vectors
    (amplitude, re/im), coef (2, 2, w).  Schmidt rank is at most 2 at every cut."""
    vecs = _c(vecs); coef = _c(coef)
    n, w = vecs.shape[1], vecs.shape[-1]
    assert vecs.shape == (2, n, 2, 2, w) and coef.shape == (2, 2, w)
    chi = np.zeros(n - 1, dtype=np.int32)
    gam = np.zeros((8 * n, 2, w_out)); lam = np.zeros((2 * (n - 1), w_out))
    rc = _load().oracle_mps_two_products(n, vecs.ctypes.data, coef.ctypes.data, w, tol_log2, chi.ctypes.data,
                                         gam.ctypes.data, lam.ctypes.data, w_out)
    if rc:
        raise RuntimeError(f"oracle_mps_two_products failed ({rc})")
    dims = [1] + [int(c) for c in chi] + [1]
    used = sum(2 * dims[l] * dims[l + 1] for l in range(n))
    return chi, gam[:used], lam[:int(chi.sum())]


def mps_apply2(n, chi, gammas, lambdas, w, site, G, tol_log2=300, r_max=1 << 20, w_out=WORDS):
    """One two-site gate update of a Vidal MPS at 320 bits (theta contraction, one-sided Jacobi SVD of the
    reshaped tensor, truncation to sigma^2 > 2^-tol_log2 sum sigma^2 and at most r_max values,
    renormalisation, split back).  G: (16, 2, wg) words, row-major in (i j) x (k m) with i the bit of
    `site`.  Returns (chi, gammas, lambdas, discarded weight)."""
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    g = _c(gammas); l = _c(lambdas); G = _c(G)
    dims = [1] + [int(c) for c in chi] + [1]
    a, d = dims[site], dims[site + 2]
    new = min(2 * a, 2 * d, r_max)
    dims2 = list(dims); dims2[site + 1] = new
    ge = sum(2 * dims2[k] * dims2[k + 1] for k in range(n))
    chi_o = np.zeros(n - 1, dtype=np.int32)
    gam_o = np.zeros((ge, 2, w_out)); lam_o = np.zeros((sum(dims2[1:n]), w_out))
    disc = ctypes.c_double()
    rc = _load().oracle_mps_apply2(n, chi.ctypes.data, g.ctypes.data, l.ctypes.data if l.size else None, w, site,
                                   G.ctypes.data, G.shape[-1], tol_log2, r_max, chi_o.ctypes.data, gam_o.ctypes.data,
                                   lam_o.ctypes.data, w_out, ctypes.byref(disc))
    if rc:
        raise RuntimeError(f"oracle_mps_apply2 failed ({rc})")
    dims3 = [1] + [int(c) for c in chi_o] + [1]
    used = sum(2 * dims3[k] * dims3[k + 1] for k in range(n))
    return chi_o, gam_o[:used], lam_o[:int(chi_o.sum())], disc.value


def mps_sample(n, chi, gammas, lambdas, w, u, w_out=WORDS):
    """A bit string drawn from the Born distribution of a canonical Vidal MPS by the chain rule, with the
    uniform numbers u (n of them, in [0, 1)) passed in: returns (bits, probability words)."""
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    g = _c(gammas); l = _c(lambdas) if len(lambdas) else np.zeros(1); u = _c(u)
    bits = np.zeros(n, dtype=np.int32); prob = np.zeros(w_out)
    if _load().oracle_mps_sample(n, chi.ctypes.data, g.ctypes.data, l.ctypes.data, w, u.ctypes.data,
                                 bits.ctypes.data, prob.ctypes.data, w_out):
        raise ValueError("bad arguments to oracle_mps_sample")
    return bits, prob


def svd(M, m, n, w_out=WORDS):
    """Singular value decomposition of the complex m x n matrix given as words (m*n, 2, w), column-major,
    by one-sided Jacobi at 320 bits.  Returns (sigma (n, w_out) descending, U (m*n, 2, w_out),
    V (n*n, 2, w_out)) with M = U diag(sigma) V^H."""
    M = _c(M)
    sig = np.zeros((n, w_out)); U = np.zeros((m * n, 2, w_out)); V = np.zeros((n * n, 2, w_out))
    rc = _load().oracle_svd(m, n, M.ctypes.data, M.shape[-1], w_out, sig.ctypes.data, U.ctypes.data, V.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_svd failed ({rc})")
    return sig, U, V


def mps_expect1(n, chi, gammas, lambdas, w, site, O, w_out=WORDS):
    """<O_site> of a Vidal MPS in canonical form from site's tensor and its two weight vectors."""
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    g = _c(gammas); l = _c(lambdas) if len(lambdas) else np.zeros(1); O = _c(O)
    out = np.zeros((2, w_out))
    if _load().oracle_mps_expect1(n, chi.ctypes.data, g.ctypes.data, l.ctypes.data, w, site, O.ctypes.data,
                                  O.shape[-1], out.ctypes.data, w_out):
        raise ValueError("bad arguments to oracle_mps_expect1")
    return out


def graph_state_schmidt_rank(n: int, edges, cut: int) -> int:
    """Schmidt rank exponent r of the graph state of a graph on vertices 0..n-1 at the cut {0..cut-1} |
    {cut..n-1}: the rank over GF(2) of the cut's biadjacency matrix (the graph state is
    prod_{(i,j) in E} CZ_ij |+>^n; every one of its 2^r Schmidt coefficients at the cut equals 2^(-r/2)).
    Plain Gaussian elimination over GF(2) on bit rows."""
    rows = []
    for i in range(cut):
        bits = 0
        for (a, b) in edges:
            if a == i and b >= cut:
                bits ^= 1 << (b - cut)
            elif b == i and a >= cut:
                bits ^= 1 << (a - cut)
        rows.append(bits)
    r = 0
    for col in range(n - cut):
        piv = next((k for k in range(r, len(rows)) if (rows[k] >> col) & 1), None)
        if piv is None:
            continue
        rows[r], rows[piv] = rows[piv], rows[r]
        for k in range(len(rows)):
            if k != r and (rows[k] >> col) & 1:
                rows[k] ^= rows[r]
        r += 1
    return r


def to_fraction(words) -> Fraction:
    return sum((Fraction(float(x)) for x in np.asarray(words).ravel()), Fraction(0))
