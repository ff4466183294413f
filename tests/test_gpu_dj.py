"""Deutsch-Jozsa-style circuits on the device MPS (Section 3.1; the paper's function structure is not
given, so workloads.dj_circuit specifies one: f(x) = x_0 + a band-graph quadratic form, or the form applied
twice for a constant f).  Checked against the 320-bit state vector at n = 10, and at widths no state vector
reaches against closed forms: every bond's squared Schmidt values are 2^-r with r the GF(2) rank of the
graph's cut (oracle.graph_state_schmidt_rank), <Z> of input 0 is -1 for the balanced function (the all-zeros
outcome has probability 0) and every input's <Z> is +1 for the constant one, and every sampled string says
so."""
from __future__ import annotations

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


def _run(ctx, n, w, kind, seed, words=4, r_max=256):
    import paper_2402_11868_gb300 as Z
    sites, gates, edges = W.dj_circuit(n, w, kind, seed=seed, wds=words)
    mps = Z.MPS(ctx, n, r_max=r_max, words=words)
    max_rho = 0
    for g_kind, s, G in gates:
        if g_kind == "1q":
            mps.apply1q(s, G)
        else:
            chi = mps.bond_dims()
            a = 1 if s == 0 else int(chi[s - 1])
            d = 1 if s + 1 == n - 1 else int(chi[s + 1])
            max_rho = max(max_rho, 2 * min(a, d))
            mps.apply2q(s, G, trunc_tau=2.0 ** -(200 if words == 4 else 96))
    return mps, gates, edges, max_rho


def _z_ops(count, words):
    Zo = np.zeros((count, 4, 2, words)); Zo[:, 0, 0, 0] = 1.0; Zo[:, 3, 0, 0] = -1.0
    return Zo


@pytest.mark.parametrize("kind", ["balanced", "constant"])
def test_dj_width_10_matches_the_state_vector(ctx, kind):
    n = 10
    mps, gates, _, _ = _run(ctx, n, 3, kind, seed=11)
    sv = oracle.Statevector(n)
    for g_kind, s, G in gates:
        (sv.apply2 if g_kind == "2q" else sv.apply1)(s, G)
    chi, g, lam = mps.download()
    amps = oracle.mps_amplitudes(n, chi, g, lam, 4)
    ref = sv.amplitudes()
    worst = max(abs(fr(amps[x, p]) - fr(ref[x, p])) for x in range(1 << n) for p in range(2))
    assert worst <= Fraction(1, 2**190), float(worst)
    mps.close()


@pytest.mark.parametrize("n,w,kind", [(40, 5, "balanced"), (40, 5, "constant"), (64, 4, "balanced")])
def test_dj_closed_forms_at_large_width(ctx, n, w, kind):
    mps, _, edges, max_rho = _run(ctx, n, w, kind, seed=n + w)
    assert max_rho <= 2 ** (w + 2)
    chi, g, lam = mps.download()
    for c, wts in enumerate(_mps.bond_weights(chi, lam), start=1):
        r = 0 if kind == "constant" or c == n - 1 else oracle.graph_state_schmidt_rank(n - 1, edges, c)
        assert len(wts) == 2 ** r, (c, len(wts), r)
        for x in wts:
            assert abs(fr(x) ** 2 - Fraction(1, 2**r)) <= Fraction(1, 2**200), (c, r)
    z = mps.expect1(list(range(n - 1)), _z_ops(n - 1, 4))
    if kind == "balanced":
        assert abs(fr(z[0, 0]) + 1) <= Fraction(1, 2**200)
    else:
        for q in range(n - 1):
            assert abs(fr(z[q, 0]) - 1) <= Fraction(1, 2**200), q
    bits, prob = mps.sample(W.uniform(90 + n, 0, 8 * n).reshape(8, n))
    for t in range(8):
        if kind == "balanced":
            assert bits[t, 0] == 1                  # never all zeros: f is balanced
        else:
            assert not bits[t, :n - 1].any()        # always all zeros: f is constant
    mps.close()
