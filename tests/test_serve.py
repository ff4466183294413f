"""Serving loop: footprint estimates and the scheduler with recorded device work (CPU), and
on the GPU: every result is the same alone and in a mix, gates keep their per-simulation order."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import workloads as W


@pytest.mark.gpu
def test_footprints_come_from_the_library_and_grow_with_size_and_precision():
    import paper_2402_11868_gb300 as Z
    from paper_2402_11868_gb300.serve import Engine, caller_bytes
    Z.build()
    eng = Engine(hbm_budget=8 << 30, slots=1)
    try:
        ef, mf = eng.eig_footprint, eng.mps_footprint
        assert ef(512, 4, 4) > ef(256, 4, 4) > ef(16, 4, 4) > 0
        assert ef(128, 4, 4) > ef(128, 2, 2)
        assert mf(40, 256, 4) > mf(40, 32, 4) > mf(10, 32, 4)
        ctx = eng.slots[0][0]
        assert ef(96, 4, 4) == caller_bytes(96, 4, 4) + Z.zkq_workspace_size(ctx, [96], 4, 4, Z.ZKQ_OA_OZAKI)
        state, gate = Z.zkq_mps_footprint(ctx, 12, 16, 4)
        assert mf(12, 16, 4) == state + gate
        # the state figure is what an MPS of that shape holds: Gamma and lambda at capacity
        caps = [min(2 ** min(l + 1, 11 - l), 16) for l in range(11)]
        dims = [1] + caps + [1]
        tensors = sum(2 * dims[l] * dims[l + 1] * 2 * 4 * 8 for l in range(12)) + sum(caps) * 4 * 8
        assert tensors < state < tensors + 4096
    finally:
        eng.close()


@pytest.mark.gpu
def test_results_same_alone_and_in_mix_and_admission():
    import paper_2402_11868_gb300 as Z
    from paper_2402_11868_gb300.serve import Engine
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
        # and against the oracle: every eigenvalue of the probe, 320-bit residuals of every mixed request
        import oracle
        L, _, _ = oracle.eigh(probe.A, probe.n)
        for i in range(probe.n):
            assert abs(fr(lm[i]) - fr(L[i])) <= anorm / 2**200
        for i, (r, n) in enumerate(zip(others, [16, 96, 33, 130, 64, 20])):
            p = W.herm_spectrum(92, i, W.spectrum_graded(n, 100 if i % 2 else 40), 4)
            t = 4 if i % 2 else 2
            lam, V = r.result["lam"], r.result["V"]
            an = max(abs(float(fr(lam[0]))), abs(float(fr(lam[-1]))))
            res, orth = oracle.residual(p.A, n, lam, V, cols=[0, n // 2, n - 1])
            bits = 200 if t == 4 else 100
            assert res.max() <= an * 2.0**-bits and orth.max() <= 2.0**-(bits - 8), (n, t)
        # a request larger than the whole budget is refused at submission
        small = Engine.__new__(Engine)
        small.budget = eng.eig_footprint(64, 4, 4) // 2
        big = Engine._enqueue(small, __import__("paper_2402_11868_gb300.serve", fromlist=["Request"]).Request(
            "eig", -1, {}, eng.eig_footprint(64, 4, 4)))
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


def test_scheduler_admission_order_and_batching_on_cpu():
    """The engine's host-side scheduling with the device work replaced by recorders (no GPU): admitted
    eigensolves never exceed the HBM budget, a batch holds one target precision and at most max_batch
    requests, gates of one simulation run one at a time in submission order, no more batches run at once
    than there are slots, and a request larger than the whole budget is refused."""
    import contextlib
    import itertools
    import threading
    import time
    from paper_2402_11868_gb300.serve import Engine, Request

    class FakeCtx:
        def close(self):
            pass

    class FakeTorch:
        class cuda:
            @staticmethod
            def stream(s):
                return contextlib.nullcontext()

    eng = Engine.__new__(Engine)
    eng.Z, eng.torch, eng.dev = None, FakeTorch, None
    eng.budget, eng.max_batch, eng.method = 1000, 3, 1
    eng.slots = [(FakeCtx(), None) for _ in range(2)]
    eng.free_slots = [0, 1]
    eng.lock = threading.Condition()
    eng.pending, eng.in_use, eng.sims, eng.sim_busy = [], 0, {}, set()
    eng.ids, eng.completed, eng.stop = itertools.count(), [], False
    log = {"batches": [], "running": 0, "max_running": 0, "over_budget": 0, "gates": {0: [], 1: []},
           "gate_overlap": 0}
    mu = threading.Lock()

    def run_eig(ctx, stream, batch):
        with mu:
            log["running"] += 1
            log["max_running"] = max(log["max_running"], log["running"])
            log["batches"].append([(r.payload["target"], r.footprint) for r in batch])
            if eng.in_use > eng.budget:
                log["over_budget"] += 1
        time.sleep(0.01)
        for r in batch:
            r.result = {"ok": True}
        with mu:
            log["running"] -= 1

    class FakeMPS:
        def __init__(self, sid):
            self.sid, self.active = sid, False

        def apply2q(self, site, G, tau, method, stream=None, ctx=None):
            with mu:
                if self.active:
                    log["gate_overlap"] += 1
                self.active = True
                log["gates"][self.sid].append(site)
            time.sleep(0.002)
            with mu:
                self.active = False
            return (1, 0.0)

        def close(self):
            pass

    eng._run_eig = run_eig
    eng.sims = {0: (FakeMPS(0), 0), 1: (FakeMPS(1), 0)}
    eng.thread = threading.Thread(target=eng._loop, daemon=True)
    eng.thread.start()
    reqs, gate_order = [], {0: [], 1: []}
    try:
        rng = np.random.default_rng(7)
        for k in range(40):
            if k % 3 == 2:
                sid = k % 2
                site = int(rng.integers(0, 20))
                gate_order[sid].append(site)
                reqs.append(eng.submit_gate(sid, site, None, 0.0))
            else:
                fp = int(rng.integers(50, 600))
                r = Request("eig", -1, {"target": 2 if k % 2 else 4}, fp)
                reqs.append(eng._enqueue(r))
        big = eng._enqueue(Request("eig", -1, {"target": 4}, 2000))
        assert big.error and "EADMIT" in big.error
        for r in reqs:
            assert r.done.wait(30) and r.error is None, r.error
    finally:
        eng.close()
    assert log["over_budget"] == 0 and eng.in_use == 0
    assert log["max_running"] <= 2
    for b in log["batches"]:
        assert 1 <= len(b) <= 3 and len({t for t, _ in b}) == 1
        assert sum(fp for _, fp in b) <= 1000
    assert sum(len(b) for b in log["batches"]) == sum(1 for r in reqs if r.kind == "eig")
    assert log["gate_overlap"] == 0
    assert log["gates"] == gate_order
