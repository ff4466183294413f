"""Measurements on the device MPS in its working precision (Section 1: a Vidal MPS is a nested Schmidt
decomposition; in canonical form the rest of the chain reduces to the squared weights): one-qubit
expectation values (zkq_mps_expect1) and chain-rule sampling with the uniform numbers passed in
(zkq_mps_sample), against the 320-bit oracle on the same state words: oracle.mps_expect1 and
Statevector.expect1 (the plain definition <psi|O|psi>), and oracle.mps_sample (same bits, same string
probability)."""
from __future__ import annotations

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


def _ops(w):
    """X, Y, Z and a general complex (non-Hermitian) operator, row-major 2x2, w words."""
    X = np.zeros((4, 2, w)); X[1, 0, 0] = X[2, 0, 0] = 1.0
    Y = np.zeros((4, 2, w)); Y[1, 1, 0] = -1.0; Y[2, 1, 0] = 1.0
    Zo = np.zeros((4, 2, w)); Zo[0, 0, 0] = 1.0; Zo[3, 0, 0] = -1.0
    H = W.haar_gate(61, 0, w=8, dim=2)
    Gn = np.zeros((4, 2, w))                 # 3/4 U + diag(0, i/4) + 1/4 i at (0, 1): neither Hermitian nor unitary
    for e in range(4):
        for p in range(2):
            v = Fraction(3, 4) * fr(H[e, p]) + (Fraction(1, 4) if (p == 1 and e in (1, 3)) else 0)
            Gn[e, p] = W.words_of(v, w)
    return [X, Y, Zo, Gn]


def _entangled_upload(ctx, n, seed, words):
    import paper_2402_11868_gb300 as Z
    sv = oracle.Statevector(n)
    for site, G in W.brickwork_circuit(seed, n, 6, w=4):
        sv.apply2(site, G)
    chi, g, lam = sv.vidal()
    mps = Z.MPS(ctx, n, r_max=1 << (n // 2), words=words)
    mps.upload(chi, g[..., :words], lam[..., :words])
    return mps, sv, chi, g[..., :words], lam[..., :words]


@pytest.mark.parametrize("words", [4, 2])
def test_expectation_values_match_the_oracle_and_the_state_vector(ctx, words):
    n = 8
    mps, sv, chi, g, lam = _entangled_upload(ctx, n, 62, words)
    ops = _ops(words)
    sites = [s for s in range(n) for _ in ops]
    O = np.stack([o for _ in range(n) for o in ops])
    got = mps.expect1(sites, O)
    bound = Fraction(1, 2**(200 if words == 4 else 100))
    for q, (site, op) in enumerate(zip(sites, O)):
        ref = oracle.mps_expect1(n, chi, g, lam, words, site, op)
        for p in range(2):
            assert abs(fr(got[q, p]) - fr(ref[p])) <= bound, (site, q % 4, p)
        # the plain definition on the state vector (the uploaded words differ from it by their rounding)
        ref_sv = sv.expect1(site, op)
        for p in range(2):
            assert abs(fr(got[q, p]) - fr(ref_sv[p])) <= (bound if words == 2 else Fraction(1, 2**195))
    # Hermitian operators give real values, the identity the norm
    for q in range(len(sites)):
        if q % 4 < 3:
            assert abs(fr(got[q, 1])) <= bound
    I2 = np.zeros((1, 4, 2, words)); I2[0, 0, 0, 0] = I2[0, 3, 0, 0] = 1.0
    one = mps.expect1([3], I2)
    assert abs(fr(one[0, 0]) - 1) <= 64 * bound
    mps.close()


def test_sampling_matches_the_oracle_chain_rule(ctx):
    n, shots = 8, 48
    mps, _, chi, g, lam = _entangled_upload(ctx, n, 63, 4)
    u = W.uniform(64, 0, shots * n).reshape(shots, n)
    bits, prob = mps.sample(u)
    for t in range(shots):
        b_ref, p_ref = oracle.mps_sample(n, chi, g, lam, 4, u[t])
        assert list(bits[t]) == list(b_ref), t
        assert abs(fr(prob[t]) - fr(p_ref)) <= fr(p_ref) * Fraction(1, 2**195), t
    # the strings follow the Born rule: each one's probability is |psi_x|^2 of the uploaded state
    amps = oracle.mps_amplitudes(n, chi, g, lam, 4)
    for t in range(4):
        x = int("".join(str(int(b)) for b in bits[t]), 2)
        p_x = fr(amps[x, 0]) ** 2 + fr(amps[x, 1]) ** 2
        assert abs(fr(prob[t]) - p_x) <= Fraction(1, 2**195)
    mps.close()


def test_measurements_on_a_device_evolved_40_qubit_state(ctx):
    """The 40-qubit quad-double brickwork of the benchmark, four layers evolved on the device: expectation values on every fifth site and 6 sampled strings against the oracle on the
    downloaded state."""
    import paper_2402_11868_gb300 as Z
    n = 40
    mps = Z.MPS(ctx, n, r_max=256, words=4)
    for site, G in W.brickwork_circuit(65, n, 4, w=4):
        mps.apply2q(site, G, trunc_tau=2.0**-200)
    chi, g, lam = mps.download()
    assert max(chi) >= 4
    ops = _ops(4)
    sites = list(range(0, n, 5))
    O = np.stack([ops[s % 4] for s in sites])
    got = mps.expect1(sites, O)
    for q, site in enumerate(sites):
        ref = oracle.mps_expect1(n, chi, g, lam, 4, site, O[q])
        for p in range(2):
            assert abs(fr(got[q, p]) - fr(ref[p])) <= Fraction(1, 2**200), (site, p)
    u = W.uniform(66, 0, 6 * n).reshape(6, n)
    bits, prob = mps.sample(u)
    for t in range(6):
        b_ref, p_ref = oracle.mps_sample(n, chi, g, lam, 4, u[t])
        assert list(bits[t]) == list(b_ref), t
        assert abs(fr(prob[t]) - fr(p_ref)) <= fr(p_ref) * Fraction(1, 2**190), t
    mps.close()


def test_measurement_arguments_are_checked(ctx):
    import paper_2402_11868_gb300 as Z
    mps = Z.MPS(ctx, 4, r_max=4, words=4)
    with pytest.raises(Z.ZkqError):
        mps.expect1([4], np.zeros((1, 4, 2, 4)))
    with pytest.raises(Z.ZkqError):
        mps.sample(np.full((1, 4), 1.0))
    bits, prob = mps.sample(np.zeros((2, 4)))      # |0000>: every bit 0 with probability 1
    assert (bits == 0).all() and np.allclose(prob[:, 0], 1.0)
    mps.close()
