"""Serving loop: footprint estimates, admission, continuous batching (CPU checks of the scheduler), and
on the GPU: every result is the same alone and in a mix, gates keep their per-simulation order."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import workloads as W


def test_footprints_grow_with_size_and_precision():
    from paper_2402_11868_gb300.serve import eig_footprint, mps_footprint
    assert eig_footprint(512, 4, 4) > eig_footprint(256, 4, 4) > eig_footprint(16, 4, 4) > 0
    assert eig_footprint(128, 4, 4) > eig_footprint(128, 2, 2)
    assert mps_footprint(40, 256, 4) > mps_footprint(40, 32, 4) > mps_footprint(10, 32, 4)


@pytest.mark.gpu
def test_results_same_alone_and_in_mix_and_admission():
    import paper_2402_11868_gb300 as Z
    from paper_2402_11868_gb300.serve import Engine, eig_footprint
    from tests._util import fr
    Z.build()
    probe = W.herm_spectrum(91, 0, W.spectrum_graded(48, 150), 4)
    eng = Engine(hbm_budget=8 << 30, slots=2)
    try:
        alone = eng.submit_eig(probe.A, probe.n, 4)
        alone.done.wait(300)
        assert alone.error is None and alone.result["rinfo"] == 0
        # the same request among others of different sizes and precisions, arriving while work runs
        others = []
        for i, n in enumerate([16, 96, 33, 130, 64, 20]):
            p = W.herm_spectrum(92, i, W.spectrum_graded(n, 100 if i % 2 else 40), 4)
            others.append(eng.submit_eig(p.A, n, 4 if i % 2 else 2))
        mixed = eng.submit_eig(probe.A, probe.n, 4)
        for r in others + [mixed]:
            assert r.done.wait(600)
            assert r.error is None, r.error
            assert r.result["rinfo"] == 0
        la, lm = alone.result["lam"], mixed.result["lam"]
        anorm = abs(fr(la[0]))
        for i in range(probe.n):
            assert abs(fr(la[i]) - fr(lm[i])) <= anorm / 2**200
        # a request larger than the whole budget is refused at submission
        small = Engine.__new__(Engine)
        small.budget = eig_footprint(64, 4, 4) // 2
        big = Engine._enqueue(small, __import__("paper_2402_11868_gb300.serve", fromlist=["Request"]).Request(
            "eig", -1, {}, eig_footprint(64, 4, 4)))
        assert big.error and "EADMIT" in big.error
        st = eng.latency_stats()
        assert st["count"] >= 8 and st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        eng.close()


@pytest.mark.gpu
def test_gate_requests_keep_order_per_simulation():
    import oracle
    import paper_2402_11868_gb300 as Z
    from paper_2402_11868_gb300.serve import Engine
    from tests._util import fr
    Z.build()
    eng = Engine(hbm_budget=8 << 30, slots=2)
    try:
        n = 5
        sims = [eng.create_simulation(n, 16, 4) for _ in range(2)]
        circs = [W.brickwork_circuit(100 + s, n, 3, w=4) for s in range(2)]
        reqs = []
        for step in range(len(circs[0])):
            for s, sid in enumerate(sims):
                site, G = circs[s][step]
                reqs.append(eng.submit_gate(sid, site, G, 2.0**-200))
        for r in reqs:
            assert r.done.wait(600) and r.error is None, r.error
        for s, sid in enumerate(sims):
            sv = oracle.Statevector(n)
            for site, G in circs[s]:
                sv.apply2(site, G)
            mps, _ = eng.sims[sid]
            chi, g, lam = mps.download()
            amps = oracle.mps_amplitudes(n, chi, g, lam, 4)
            ref = sv.amplitudes()
            worst = max(abs(fr(amps[x, p]) - fr(ref[x, p])) for x in range(1 << n) for p in range(2))
            assert worst <= Fraction(1, 2**185)
    finally:
        eng.close()
