"""Continuous-batching request loop for many concurrent circuit simulations.

Requests (from many simulations) are eigensolves of Hermitian reduced matrices and two-qubit gate
applications on device-resident MPS states.  The engine
  * admits a request when its HBM footprint fits the budget (else it waits; a request larger than the
    whole budget is refused at submission with ZKQ_EADMIT semantics); footprints come from the library
    (zkq_workspace_size, zkq_mps_footprint), so they follow its layouts;
  * packs every admitted eigensolve of the same target precision into one uneven batch (one FP64 Jacobi
    launch + one refinement call) on a free execution slot — each slot owns a library context and a CUDA
    stream, so batches on different slots overlap on the device; requests arriving while batches run join
    the next batch as slots and memory free up;
  * runs gate applications of a simulation in submission order on a slot (the MPS update decides the new
    bond dimension on the host);
  * records arrival, start and completion times for p50/p99 latency.
A result depends only on its own request (kernel choices follow the problem's own size and precision),
so a request gives the same answer alone and in a mix, within the refinement tolerance.

Only marshalling and scheduling live here; every arithmetic step runs in libzkq.
"""
from __future__ import annotations

import itertools
import threading
import time
from dataclasses import dataclass, field

import numpy as np


def caller_bytes(n: int, a_words: int, target: int) -> int:
    """Device bytes of the arrays the engine allocates for one eigensolve request: the input (n^2 complex,
    a_words words), FP64 eigenpairs and info, refined eigenpairs, residual estimates and info."""
    el = n * n
    return int(el * 2 * a_words * 8 + (n * 8 + el * 16 + 4) + (n * target * 8 + el * 2 * target * 8 + n * 8 + 4))


@dataclass(eq=False)
class Request:
    kind: str                      # "eig" or "gate"
    sim: int
    payload: dict
    footprint: int
    rid: int = 0
    t_arrive: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    result: object = None
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)


class Engine:
    def __init__(self, device: int = 0, hbm_budget: int = 64 << 30, slots: int = 2, max_batch: int = 64,
                 method: int | None = None):
        import torch
        import paper_2402_11868_gb300 as Z
        self.Z, self.torch = Z, torch
        self.dev = torch.device("cuda", device)
        self.budget = int(hbm_budget)
        self.max_batch = max_batch
        self.method = Z.ZKQ_OA_OZAKI if method is None else method
        self.slots = [(Z.Context(device), torch.cuda.Stream(device=self.dev)) for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.lock = threading.Condition()
        self.pending: list[Request] = []
        self.in_use = 0
        self.sims: dict[int, object] = {}
        self.sim_busy: set[int] = set()
        self.ids = itertools.count()
        self.completed: list[Request] = []
        self.stop = False
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # ---------------------------------------------------------------- footprints (from the library)
    def eig_footprint(self, n: int, a_words: int, target: int) -> int:
        """Device bytes an eigensolve request holds in flight: its arrays plus the workspace the library
        reports for it (zkq_workspace_size: eigensolve, refinement state and split-product scratch)."""
        ws = self.Z.zkq_workspace_size(self.slots[0][0], [n], a_words, target, self.method)
        return caller_bytes(n, a_words, target) + int(ws)

    def mps_footprint(self, n_qubits: int, r_max: int, words: int) -> int:
        """Device bytes a simulation holds while it exists: its MPS at capacity and the workspace of its
        widest gate update (zkq_mps_footprint)."""
        state, gate = self.Z.zkq_mps_footprint(self.slots[0][0], n_qubits, r_max, words, self.method)
        return int(state + gate)

    # ---------------------------------------------------------------- submission
    def create_simulation(self, n_qubits: int, r_max: int, words: int = 4) -> int:
        sid = self.try_create_simulation(n_qubits, r_max, words)
        if sid is None:
            raise MemoryError("simulation does not fit the HBM budget")
        return sid

    def try_create_simulation(self, n_qubits: int, r_max: int, words: int = 4):
        """Admit a simulation if its footprint fits the budget now (else None: the caller retries once memory
        frees up)."""
        fp = self.mps_footprint(n_qubits, r_max, words)
        with self.lock:
            if fp > self.budget - self.in_use:
                return None
            self.in_use += fp
            sid = next(self.ids)
            ctx = self.slots[0][0]
        try:
            mps = self.Z.MPS(ctx, n_qubits, r_max, words)
        except Exception:
            with self.lock:
                self.in_use -= fp
            raise
        with self.lock:
            self.sims[sid] = (mps, fp)
        return sid

    def destroy_simulation(self, sid: int):
        with self.lock:
            mps, fp = self.sims.pop(sid)
            mps.close()
            self.in_use -= fp
            self.lock.notify_all()

    def submit_eig(self, A_words: np.ndarray, n: int, target: int, sim: int = -1) -> Request:
        a_words = A_words.shape[-1]
        fp = self.eig_footprint(n, a_words, target)
        r = Request("eig", sim, {"A": A_words, "n": n, "target": target, "a_words": a_words}, fp)
        return self._enqueue(r)

    def submit_gate(self, sim: int, site: int, G: np.ndarray, tau: float) -> Request:
        r = Request("gate", sim, {"site": site, "G": G, "tau": tau}, 0)
        return self._enqueue(r)

    def _enqueue(self, r: Request) -> Request:
        if r.footprint > self.budget:
            r.error = "ZKQ_EADMIT: request larger than the HBM budget"
            r.done.set()
            return r
        with self.lock:
            r.rid = next(self.ids)
            r.t_arrive = time.perf_counter()
            self.pending.append(r)
            self.lock.notify_all()
        return r

    def close(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        self.thread.join(timeout=60)
        for sid in list(self.sims):
            self.destroy_simulation(sid)
        for ctx, _ in self.slots:
            ctx.close()

    # ---------------------------------------------------------------- scheduling
    def _take_work(self):
        """Pick the next unit of work: a gate of an idle simulation, else a batch of eigensolves of one
        target precision that fits the remaining budget (called with the lock held)."""
        for r in self.pending:
            if r.kind == "gate" and r.sim not in self.sim_busy:
                # gates of a simulation stay in submission order
                first = next(q for q in self.pending if q.kind == "gate" and q.sim == r.sim)
                if first is r:
                    self.pending.remove(r)
                    self.sim_busy.add(r.sim)
                    return [r]
        eig = [r for r in self.pending if r.kind == "eig"]
        if not eig:
            return None
        target = eig[0].payload["target"]
        batch, need = [], 0
        for r in eig:
            if r.payload["target"] != target or len(batch) >= self.max_batch:
                continue
            if self.in_use + need + r.footprint > self.budget:
                continue
            batch.append(r); need += r.footprint
        if not batch:
            return None
        for r in batch:
            self.pending.remove(r)
        self.in_use += need
        return batch

    def _loop(self):
        workers = []
        while True:
            with self.lock:
                while not self.stop and (not self.free_slots or not self.pending or self._peek_blocked()):
                    self.lock.wait(timeout=0.05)
                    workers = [w for w in workers if w.is_alive()]
                if self.stop and not self.pending:
                    break
                work = self._take_work() if self.free_slots else None
                if not work:
                    continue
                slot = self.free_slots.pop(0)
            t = threading.Thread(target=self._run, args=(slot, work), daemon=True)
            t.start()
            workers.append(t)
        for w in workers:
            w.join(timeout=120)

    def _peek_blocked(self):
        # nothing runnable: only gates of busy simulations or eigensolves that do not fit yet
        for r in self.pending:
            if r.kind == "gate" and r.sim not in self.sim_busy:
                return False
            if r.kind == "eig" and self.in_use + r.footprint <= self.budget:
                return False
        return True

    def _run(self, slot, work):
        ctx, stream = self.slots[slot]
        t0 = time.perf_counter()
        for r in work:
            r.t_start = t0
        try:
            if work[0].kind == "gate":
                r = work[0]
                mps, _ = self.sims[r.sim]
                with self.torch.cuda.stream(stream):
                    r.result = mps.apply2q(r.payload["site"], r.payload["G"], r.payload["tau"], self.method,
                                           stream=stream, ctx=ctx)
            else:
                self._run_eig(ctx, stream, work)
        except Exception as e:  # a failed batch reports the error to each of its requests
            for r in work:
                r.error = str(e)
        t1 = time.perf_counter()
        with self.lock:
            for r in work:
                r.t_done = t1
                self.completed.append(r)
                if r.kind == "eig":
                    self.in_use -= r.footprint
                else:
                    self.sim_busy.discard(r.sim)
            self.free_slots.append(slot)
            self.lock.notify_all()
        for r in work:
            r.done.set()

    def _run_eig(self, ctx, stream, batch):
        Z, torch = self.Z, self.torch
        ns = [r.payload["n"] for r in batch]
        wa = max(r.payload["a_words"] for r in batch)
        target = batch[0].payload["target"]
        a_off, w_off, tot_a, tot_w = Z.batch_offsets(ns)
        host = torch.from_numpy(Z.pack([r.payload["A"] for r in batch], wa)).pin_memory()
        with torch.cuda.stream(stream):
            A = host.to(self.dev, non_blocking=True)
            f64 = dict(dtype=torch.float64, device=self.dev)
            Wd = torch.empty(tot_w, **f64); Vd = torch.empty(2 * tot_a, **f64)
            info = torch.empty(len(ns), dtype=torch.int32, device=self.dev)
            Wo = torch.empty(target * tot_w, **f64); Vo = torch.empty(2 * target * tot_a, **f64)
            err = torch.empty(tot_w, **f64); rinfo = torch.empty(len(ns), dtype=torch.int32, device=self.dev)
            Z.zkq_eigh_batched(ctx, ns, a_off, A, wa, Wd, Vd, info, stream=stream)
            Z.zkq_rqi_refine(ctx, ns, a_off, A, wa, Wd, Vd, target, self.method, Wo, Vo, err, rinfo, stream=stream)
            Wh = Wo.to("cpu", non_blocking=True); Vh = Vo.to("cpu", non_blocking=True)
            ih = info.to("cpu", non_blocking=True); rh = rinfo.to("cpu", non_blocking=True)
        stream.synchronize()
        Wh, Vh, ih, rh = Wh.numpy(), Vh.numpy(), ih.numpy(), rh.numpy()
        for b, r in enumerate(batch):
            n = ns[b]
            r.result = {"lam": Wh[target * w_off[b]: target * (w_off[b] + n)].reshape(n, target),
                        "V": Vh[2 * target * a_off[b]: 2 * target * (a_off[b] + n * n)].reshape(n * n, 2, target),
                        "info": int(ih[b]), "rinfo": int(rh[b])}

    # ---------------------------------------------------------------- statistics
    def latency_stats(self):
        lat = [r.t_done - r.t_arrive for r in self.completed if r.error is None]
        if not lat:
            return {}
        return {"count": len(lat), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "max_ms": 1e3 * max(lat)}
