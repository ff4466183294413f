"""MPS gate updates at the sizes the brickwork benchmark reaches, on states uploaded from the oracle, with
truncation at r_max, and on the paper's footnote example (Section 1 and its footnote; Section 2: theta
contraction, eigensolve of the reduced matrix, truncation and split back at each gate).

* A 14-qubit brickwork (bond dimension 128 at the centre, reduced matrices up to 128 x 128: the multi-CTA
  Jacobi and the large split-product tiles run inside the gate update) against the 320-bit state vector:
  every amplitude, every bond's squared weights against the state vector's Schmidt values at that cut, and
  the Vidal canonical conditions of every site.
* Exact starting states uploaded through zkq_mps_upload (the oracle's Vidal form of an entangled state, full
  bond dimension), one gate on the device against the oracle's gate update (oracle.mps_apply2): new weights,
  amplitudes, discarded weight; the same with the kept rank capped at r_max.
* The footnote state C^{n-1}-Z |+...+>|-> from the oracle's two-product Vidal form at n = 64, 120, 180:
  gates on the target bond keep the squared Schmidt coefficients 1 - 2^-(n-1), 2^-(n-1) within 2^-200 in
  quad double; double double (null-space threshold 2^-96) drops the small one beyond n = 97.
* The footnote circuit (workloads.footnote_circuit: C^k-Z as nearest-neighbour gates with an ancilla ladder)
  run gate by gate on the device for k = 39 and 63 controls: every bond's weights against the oracle's
  two-product Vidal form of the final state."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W
from tests._util import fr
from tests import _mps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2402_11868_gb300 as Z
    Z.build()
    c = Z.Context(0)
    yield c
    c.close()


def _amps_max_diff(a, b):
    return max(abs(fr(a[x, p]) - fr(b[x, p])) for x in range(a.shape[0]) for p in range(2))


def test_brickwork14_every_bond_against_the_state_vector(ctx):
    import paper_2402_11868_gb300 as Z
    n, depth = 14, 14
    circ = W.brickwork_circuit(29, n, depth, w=4)
    mps = Z.MPS(ctx, n, r_max=128, words=4)
    sv = oracle.Statevector(n)
    max_rho = 0
    for site, G in circ:
        chi = mps.bond_dims()
        a = 1 if site == 0 else int(chi[site - 1])
        d = 1 if site + 1 == n - 1 else int(chi[site + 1])
        max_rho = max(max_rho, 2 * min(a, d))
        _, disc = mps.apply2q(site, G, trunc_tau=2.0**-200)
        assert disc <= 2.0**-180
        sv.apply2(site, G)
    assert max_rho == 128
    chi, g, lam = mps.download()
    assert list(chi) == [min(2 ** min(c, n - c), 128) for c in range(1, n)]
    amps = oracle.mps_amplitudes(n, chi, g, lam, 4)
    ref = sv.amplitudes()
    assert _amps_max_diff(amps, ref) <= Fraction(1, 2**185)
    assert _mps.canonical_defect(n, chi, g, lam, 4) <= 2.0**-185
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        s2 = list(ex.map(sv.schmidt2, range(1, n)))
    for l, (wts, ref2) in enumerate(zip(_mps.bond_weights(chi, lam), s2)):
        vals = [fr(x) for x in wts]
        assert abs(sum(v * v for v in vals) - 1) <= Fraction(1, 2**195), l
        for b in range(len(vals)):
            assert abs(vals[b] ** 2 - fr(ref2[b])) <= Fraction(1, 2**190), (l, b)


def _entangled_vidal(n, depth, seed):
    sv = oracle.Statevector(n)
    for site, G in W.brickwork_circuit(seed, n, depth, w=4):
        sv.apply2(site, G)
    chi, g, lam = sv.vidal()
    return sv, chi, g, lam


@pytest.mark.parametrize("site", [3, 1, 6])
def test_uploaded_full_rank_state_gate_matches_the_oracle_update(ctx, site):
    import paper_2402_11868_gb300 as Z
    n = 8
    sv, chi, g, lam = _entangled_vidal(n, 6, 31)
    assert list(chi) == [2, 4, 8, 16, 8, 4, 2]
    mps = Z.MPS(ctx, n, r_max=16, words=4)
    mps.upload(chi, g[..., :4], lam[..., :4])
    G = W.haar_gate(32, site, w=4)
    nb, disc = mps.apply2q(site, G, trunc_tau=2.0**-200)
    chi_o, g_o, lam_o, disc_o = oracle.mps_apply2(n, chi, g, lam, oracle.WORDS, site, G, tol_log2=200)
    chi_d, g_d, lam_d = mps.download()
    assert list(chi_d) == list(chi_o) and nb == chi_o[site]
    assert disc <= 2.0**-180 and disc_o <= 2.0**-180        # only values at the rounding level are dropped
    for wd, wo in zip(_mps.bond_weights(chi_d, lam_d), _mps.bond_weights(chi_o, lam_o)):
        for x, y in zip(wd, wo):
            assert abs(fr(x) - fr(y)) <= Fraction(1, 2**195)
    ref = sv.amplitudes(); sv2 = oracle.Statevector(n); sv2.set(ref); sv2.apply2(site, G)
    assert _amps_max_diff(oracle.mps_amplitudes(n, chi_d, g_d, lam_d, 4), sv2.amplitudes()) <= Fraction(1, 2**190)
    assert _mps.canonical_defect(n, chi_d, g_d, lam_d, 4) <= 2.0**-185


def test_truncation_at_r_max_matches_the_oracle_update(ctx):
    """States whose bonds are capped at r_max = 4, built by the oracle's own gate updates; a gate that would
    raise the centre bond to 8 is truncated to 4 on the device: kept weights (renormalised), discarded weight
    1 - sum kept sigma^2 / sum sigma^2 and the amplitudes of the truncated state match the oracle's."""
    import paper_2402_11868_gb300 as Z
    n, r_max = 8, 4
    one, zero = Fraction(1), Fraction(0)
    chi, g, lam = _mps.product_state([((one, zero), (zero, zero))] * n, oracle.WORDS)
    circ = W.brickwork_circuit(33, n, 5, w=4)
    for site, G in circ:
        chi, g, lam, _ = oracle.mps_apply2(n, chi, g, lam, oracle.WORDS, site, G, tol_log2=200, r_max=r_max)
    assert max(chi) == r_max
    checked = 0
    for t, site in enumerate((3, 2, 4)):
        dims = _mps.dims_of(n, chi)
        if 2 * min(dims[site], dims[site + 2]) <= r_max:
            continue
        G = W.haar_gate(34, t, w=4)
        mps = Z.MPS(ctx, n, r_max=r_max, words=4)
        mps.upload(chi, g[..., :4], lam[..., :4])
        nb, disc = mps.apply2q(site, G, trunc_tau=2.0**-200)
        chi_o, g_o, lam_o, disc_o = oracle.mps_apply2(n, chi, g, lam, oracle.WORDS, site, G, tol_log2=200, r_max=r_max)
        chi_d, g_d, lam_d = mps.download()
        assert nb == r_max and list(chi_d) == list(chi_o)
        assert disc_o > 1e-6 and abs(disc - disc_o) <= 2.0**-48, (disc, disc_o)
        wd, wo = _mps.bond_weights(chi_d, lam_d)[site], _mps.bond_weights(chi_o, lam_o)[site]
        for x, y in zip(wd, wo):
            assert abs(fr(x) - fr(y)) <= Fraction(1, 2**190)
        amps_d = oracle.mps_amplitudes(n, chi_d, g_d, lam_d, 4)
        amps_o = oracle.mps_amplitudes(n, chi_o, g_o, lam_o, oracle.WORDS)
        assert _amps_max_diff(amps_d, amps_o) <= Fraction(1, 2**185)
        checked += 1
        mps.close()
    assert checked >= 2


# ------------------------------------------------------------------------------------------------------
# the paper's footnote example
def _golden_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "footnote_schmidt.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {int(r[0]): ([int(c) for c in r[1]], int(r[2])) for r in rows}


def _two_product_words(vecs, coef, w=oracle.WORDS):
    n = len(vecs[0])
    V = np.zeros((2, n, 2, 2, w)); C = np.zeros((2, 2, w))
    for t in range(2):
        for l in range(n):
            for s in range(2):
                for p in range(2):
                    V[t, l, s, p] = W.words_of(Fraction(vecs[t][l][s][p]), w)
        for p in range(2):
            C[t, p] = W.words_of(Fraction(coef[t][p]), w)
    return V, C


def _footnote_vidal(n, ctrl):
    """Normalised Vidal MPS of C^{n-1}-Z |+...+>|-> (target last): unnormalised |+...+>|-> + |c>(0, 2) from the
    oracle's two-product form, norm^2 2^n, rescaled exactly (n even)."""
    one, zero = Fraction(1), Fraction(0)
    plus, minus = ((one, zero), (one, zero)), ((one, zero), (-one, zero))
    e = lambda b: (((one, zero), (zero, zero)) if b == 0 else ((zero, zero), (one, zero)))
    vecs = [[plus] * (n - 1) + [minus], [e(b) for b in ctrl] + [((zero, zero), (Fraction(2), zero))]]
    V, C = _two_product_words(vecs, [(one, zero), (one, zero)])
    chi, g, lam = oracle.mps_two_products(V, C)
    g, lam = _mps.scale_norm(n, chi, g, lam, n // 2)
    return chi, g, lam


def _product_gate(seed, w):
    """U (x) V for two Haar one-qubit gates, as a 4x4 in (i j) x (k m)."""
    U = W.haar_gate(seed, 0, w=8, dim=2); V = W.haar_gate(seed, 1, w=8, dim=2)
    Uc = [[(fr(U[r * 2 + c, 0]), fr(U[r * 2 + c, 1])) for c in range(2)] for r in range(2)]
    Vc = [[(fr(V[r * 2 + c, 0]), fr(V[r * 2 + c, 1])) for c in range(2)] for r in range(2)]
    G = np.zeros((16, 2, w))
    for i in range(2):
        for j in range(2):
            for k in range(2):
                for m in range(2):
                    a, b = Uc[i][k], Vc[j][m]
                    G[(2 * i + j) * 4 + 2 * k + m, 0] = W.words_of(a[0] * b[0] - a[1] * b[1], w)
                    G[(2 * i + j) * 4 + 2 * k + m, 1] = W.words_of(a[0] * b[1] + a[1] * b[0], w)
    return G


@pytest.mark.parametrize("n", [64, 120, 180])
def test_footnote_state_keeps_its_tiny_schmidt_coefficient_in_quad_double(ctx, n):
    import paper_2402_11868_gb300 as Z
    ctrl, e = _golden_rows()[n]
    assert e == -(n - 1)
    chi, g, lam = _footnote_vidal(n, ctrl)
    eps = Fraction(1, 2 ** (n - 1))
    I4 = np.zeros((16, 2, 4))
    for r in range(4):
        I4[r * 4 + r, 0, 0] = 1.0
    for G in (I4, _product_gate(50 + n, 4)):
        mps = Z.MPS(ctx, n, r_max=4, words=4)
        mps.upload(chi, g[..., :4], lam[..., :4])
        nb, disc = mps.apply2q(n - 2, G, trunc_tau=2.0**-200)
        assert nb == 2
        _, _, lam_d = mps.download()
        l0, l1 = fr(lam_d[-2]) ** 2, fr(lam_d[-1]) ** 2
        assert abs(l0 - (1 - eps)) <= Fraction(1, 2**200) and abs(l1 - eps) <= Fraction(1, 2**200), float(l1 / eps)
        mps.close()
    # double double: eps below its null-space threshold 2^-96 is dropped, the bond collapses to rank 1
    mps = Z.MPS(ctx, n, r_max=4, words=2)
    mps.upload(chi, g[..., :2], lam[..., :2])
    nb, disc = mps.apply2q(n - 2, I4[..., :2], trunc_tau=2.0**-96)
    assert nb == (2 if eps > Fraction(1, 2**96) else 1)


@pytest.mark.parametrize("n", [40, 64])
def test_footnote_circuit_on_the_device_matches_the_two_product_state(ctx, n):
    """C^k-Z with k = n - 1 controls as nearest-neighbour gates (ancilla ladder), run gate by gate on a
    quad-double device MPS from |+...+>|0...0>|-> (uploaded as a product state): every bond's weights equal
    the oracle's two-product Vidal form of the final state, and the cut before the target has squared Schmidt
    coefficients 1 - 2^-k and 2^-k within 2^-200."""
    import paper_2402_11868_gb300 as Z
    ctrl, _ = _golden_rows()[n]
    k = n - 1
    sites, gates = W.footnote_circuit(ctrl, w=4)
    pos = [0] + [2 * l - 1 for l in range(1, k)]
    target = 2 * k - 1
    one, zero = Fraction(1), Fraction(0)
    # |+> and |-> with amplitudes 2^-1/2 rounded to 8 words (the oracle's precision); the device takes 4
    h = sum(Fraction(x) for x in _inv_sqrt2_words())
    plus, minus, zero_v = ((h, zero), (h, zero)), ((h, zero), (-h, zero)), ((one, zero), (zero, zero))
    local = [plus if q in pos else (minus if q == target else zero_v) for q in range(sites)]
    chi0, g0, lam0 = _mps.product_state(local, 4)
    mps = Z.MPS(ctx, sites, r_max=8, words=4)
    mps.upload(chi0, g0, lam0)
    for kind, s, G in gates:
        if kind == "1q":
            mps.apply1q(s, G)
        else:
            mps.apply2q(s, G, trunc_tau=2.0**-200)
    chi_d, g_d, lam_d = mps.download()
    # the oracle's Vidal form of |+..+>|0..0>|-> + |c>|0..0>(0, 2), normalised (norm^2 2^(k+1))
    e0, e1 = ((one, zero), (zero, zero)), ((zero, zero), (one, zero))
    P, M = ((one, zero), (one, zero)), ((one, zero), (-one, zero))
    t0 = [P if q in pos else (M if q == target else e0) for q in range(sites)]
    t1 = [(e1 if ctrl[pos.index(q)] else e0) if q in pos else
          (((zero, zero), (Fraction(2), zero)) if q == target else e0) for q in range(sites)]
    V, C = _two_product_words([t0, t1], [(one, zero), (one, zero)])
    chi_o, _, lam_o = oracle.mps_two_products(V, C)
    norm2 = Fraction(2) ** (k + 1)
    wd, wo = _mps.bond_weights(chi_d, lam_d), _mps.bond_weights(chi_o, lam_o)
    assert list(chi_d) == list(chi_o)
    for l in range(sites - 1):
        for x, y in zip(wd[l], wo[l]):
            assert abs(fr(x) ** 2 - fr(y) ** 2 / norm2) <= Fraction(1, 2**200), l
    eps = Fraction(1, 2**k)
    l0, l1 = fr(wd[target - 1][0]) ** 2, fr(wd[target - 1][1]) ** 2
    assert abs(l0 - (1 - eps)) <= Fraction(1, 2**200) and abs(l1 - eps) <= Fraction(1, 2**200)


def _inv_sqrt2_words():
    """2^-1/2 as 8 words (Decimal square root at 200 digits, rounded word by word)."""
    from decimal import Decimal, getcontext
    getcontext().prec = 200
    return W.words_of(Fraction(Decimal(1) / Decimal(2).sqrt()), 8)
