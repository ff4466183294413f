"""Benchmark: quad-double refined eigenpairs per second (error <= 2^-200 ||A||), p50/p99 step latency,
against the plain RQI path.

One step = one pass of the whole hot path over one batch already resident in HBM:
FP64 Jacobi eigensolve (zkq_eigh_batched) + precision recovery (zkq_rqi_refine).

Workloads (seeded, synthetic; see workloads/):
  batch256_qd      256 complex Hermitian problems, N uniform in {16,...,512}, spectrum graded
                   lambda_k = 2^(-180(k-1)/(N-1)) with 8 near-degenerate pairs (relative split 2^-60),
                   quad-double input; chosen path: Ogita-Aishima refinement with Ozaki split products
                   on tensor cores (default)
  single128_plain  one 128x128 problem, lambda_k = 2^-0.3(k-1), quad-double input, plain RQI path
  brickwork40      MPS simulation of a 40-qubit brickwork circuit of Haar two-qubit gates (r_max = 256,
                   quad-double, truncation 2^-200): one step = one layer of gates on disjoint bonds; the
                   state keeps evolving, so the timed layers follow the warm-up layers (bond dimensions grow)
  serve            continuous-batching engine under Poisson arrivals at 0.7x saturation: 64 MPS simulations
                   (n 24..64, r_max 32..1024, DD/QD) admitted by HBM footprint, gate updates and eigensolves
                   (DD/QD, N <= 512); per-type p50/p99 latency
  dj               Deutsch-Jozsa-style circuits (balanced band-graph function) at widths 16..128 on a quad-double
                   MPS: time per circuit against the width, gates/s, largest diagonalised matrix
The plain RQI path cannot resolve eigenvalues below the FP64 floor (2^-53 ||A||), so the same-accuracy
comparison of the two paths is reported on single128 (both paths), beside the batch number.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
Under torchrun each rank processes its own seeded batch (weak scaling, no data-path collective); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

METRIC = "quad-double refined eigenpairs/sec (err ≤2^-200‖A‖), p50/p99 latency vs plain RQI path"
# FP64 peak of one GB300 from its unit counts and clock: 152 SMs x 2 FP64 operations (FMA, add or multiply)
# per clock per SM x 2.07 GHz = 0.629 T FP64 instructions/s, 1.259 TFLOP/s with an FMA as two flops (the
# nominal 1.25 TFLOP/s).  The roofline fractions use this figure.
FP64_INSTR_PEAK = 152 * 2 * 2.07e9
FP64_TFLOPS_PEAK = 2 * FP64_INSTR_PEAK / 1e12
# a DFMA-throughput microbenchmark on this machine reached 1.006 TFLOP/s (1.6 FMA per clock per SM); reported
# beside the derived peak
FP64_TFLOPS_MEASURED = 1.006
# FP64 instructions of one complex quad-double multiply-add (QD mul 142, QD add 109; 4 mul + 4 add)
QD_CMAC_INSTR = 4 * 142 + 4 * 109


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch256_qd", choices=["batch256_qd", "single128_plain", "brickwork40", "serve", "dj"])
    ap.add_argument("--count", type=int, default=256, help="problems in the batch workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the single128 chosen-vs-plain comparison")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx, self.rows, self.proc = device_index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        num = lambda v: v.replace(".", "", 1).isdigit()
        sm = [float(r[0]) for r in self.rows if num(r[0])]
        mx = [float(r[1]) for r in self.rows if num(r[1])]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------------------------------------------
def load_workload(name, rank, count, world=1):
    """The rank's problems.  The batch workload is one job of count x world problems (seed 1) sharded across
    the ranks by the package's N^3-balanced partition (paper_2402_11868_gb300.shard): weak scaling, about
    count problems' work per GPU, no data-path collective."""
    import workloads as W
    if name == "single128_plain":
        return [W.config_single128(seed=rank)], 4, "plain", "single 128x128 Hermitian, lambda_k=2^-0.3(k-1), QD input"
    total = count * world
    if world == 1:
        mine = None
    else:
        from paper_2402_11868_gb300.shard import my_share
        mine = my_share(W.batch_sizes(1, total), world, rank)
    return (W.config_batch(2, seed=1, count=total, indices=mine), 4, "chosen",
            f"{total} Hermitian problems, N~U{{16..512}}, lambda graded to 2^-180, 8 pairs split 2^-60 (rel), QD "
            f"input" + (f"; sharded by N^3 over {world} ranks" if world > 1 else ""))


class Runner:
    """Device-resident batch + output buffers and one step of the hot path."""

    def __init__(self, Z, torch, dev, problems, words, method, target=4):
        self.Z, self.torch = Z, torch
        self.ns = [p.n for p in problems]
        self.a_off, self.w_off, tot_a, tot_w = Z.batch_offsets(self.ns)
        self.words, self.target = words, target
        self.method = Z.ZKQ_PLAIN_RQI if method == "plain" else Z.ZKQ_OA_OZAKI
        self.A_host = torch.from_numpy(Z.pack([p.A for p in problems], words)).pin_memory()
        self.A = self.A_host.to(dev)
        f64 = dict(dtype=torch.float64, device=dev)
        self.W = torch.zeros(tot_w, **f64); self.V = torch.zeros(2 * tot_a, **f64)
        self.info = torch.zeros(len(self.ns), dtype=torch.int32, device=dev)
        self.Wo = torch.zeros(target * tot_w, **f64); self.Vo = torch.zeros(2 * target * tot_a, **f64)
        self.err = torch.zeros(tot_w, **f64)
        self.rinfo = torch.zeros(len(self.ns), dtype=torch.int32, device=dev)
        self.pairs = tot_w
        self.err_bound = 2.0 ** -(53 * target - 12)

    def step(self, ctx, s):
        Z, torch = self.Z, self.torch
        Z.zkq_eigh_batched(ctx, self.ns, self.a_off, self.A, self.words, self.W, self.V, self.info, stream=s)
        em = torch.cuda.Event(enable_timing=True)
        em.record(s)
        Z.zkq_rqi_refine(ctx, self.ns, self.a_off, self.A, self.words, self.W, self.V, self.target, self.method,
                         self.Wo, self.Vo, self.err, self.rinfo, stream=s)
        return em

    def check(self):
        """(converged, failures, max err): every problem's info flags are 0 and every eigenpair's residual
        estimate ||A v - lambda v|| / ||A|| (err_est, read back from the device) is within 2^-(53 W - 12),
        the target's bound (2^-200 for quad double)."""
        info, rinfo = self.info.cpu().numpy(), self.rinfo.cpu().numpy()
        err = float(self.err.max().item())
        ok = bool((info == 0).all() and (rinfo == 0).all()) and err <= self.err_bound
        return ok, int((info != 0).sum() + (rinfo != 0).sum()), err


def oracle_rate(problems, threads):
    """Oracle (320-bit Jacobi) eigenpairs/s on the given problems, one problem per host thread."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda p: oracle.eigh(p.A, p.n), problems))
    dt = time.perf_counter() - t0
    return sum(p.n for p in problems) / dt, dt


def stratified_sample(problems, sizes=(16, 32, 48, 64, 80, 96, 112, 128)):
    out = []
    for s in sizes:
        for p in problems:
            if p.n == s:
                out.append(p)
                break
    return out or problems[:1]


def oracle_baseline(problems, single):
    """The oracle on a bounded, size-stratified sample: one batch problem of every order 16..128 plus the single
    128x128 problem, one problem per host thread.  Reports the sample's rate, the rate per order, and the rate the
    oracle would reach on the whole batch, from a fit of its time per problem to c N^3 (its work is
    O(N^3) per sweep) over the sampled orders."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    sample = stratified_sample(problems) + list(single)
    cores = min(len(sample), os.cpu_count() or 1)

    def timed(p):
        t0 = time.perf_counter()
        oracle.eigh(p.A, p.n)
        return time.perf_counter() - t0

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        dts = list(ex.map(timed, sample))
    wall = time.perf_counter() - t0
    ns = np.array([p.n for p in sample], dtype=float)
    c = float(np.sum(np.array(dts) * ns**3) / np.sum(ns**6))       # least squares of t = c N^3
    full_s = c * float(sum(p.n ** 3 for p in problems))
    per_n = {}
    for p, dt in zip(sample, dts):
        per_n.setdefault(str(p.n), []).append(p.n / dt)
    return {"value": sum(p.n for p in sample) / wall, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle (320-bit cyclic Jacobi) on {len(sample)} problems: one batch problem of each order "
                      f"{[p.n for p in sample[:-len(single)] or sample]} and the single 128x128 problem, one per "
                      f"thread, {wall:.1f} s wall",
            "per_order_eigenpairs_per_s_one_core": {k: float(np.mean(v)) for k, v in sorted(per_n.items(), key=lambda kv: int(kv[0]))},
            "fit_s_per_problem": f"{c:.3e} N^3",
            "extrapolated_full_batch": {"eigenpairs_per_s": sum(p.n for p in problems) / (full_s / cores),
                                        "on_cores": cores, "batch_cpu_s": full_s}}


def run_ours(args):
    import torch
    import paper_2402_11868_gb300 as Z
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    problems, words, method, desc = load_workload(args.workload, rank, args.count, world)
    R = Runner(Z, torch, dev, problems, words, method)
    ctx = Z.Context(local)
    stream = torch.cuda.Stream(device=dev)
    in_bytes = R.A.numel() * 8
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if in_bytes < (256 << 20) else None
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            R.step(ctx, stream)
    torch.cuda.synchronize()
    ok, nbad, _ = R.check()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    Z.zkq_profile_enable(True)
    Z.zkq_profile_read()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms, jac_ms, ref_ms = [], [], []
    for _ in range(args.steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(1.0)          # evict the inputs from L2 between timed steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            em = R.step(ctx, stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1)); jac_ms.append(e0.elapsed_time(em)); ref_ms.append(em.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof = Z.zkq_profile_read()
    Z.zkq_profile_enable(False)
    clk = clocks.stop()
    ok2, nbad2, max_err = R.check()
    total_ms = float(sum(step_ms))
    job_pairs = R.pairs
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        pc = torch.tensor([float(R.pairs)], device=dev)
        dist.all_reduce(pc, op=dist.ReduceOp.SUM)    # the ranks' shares differ: count them all
        job_pairs = int(pc.item())
    value = job_pairs * args.steps / (total_ms / 1e3)
    # end to end through the C ABI: pinned host input -> device, hot path, results back to pinned host
    Wo_h = torch.empty(R.Wo.numel(), dtype=torch.float64).pin_memory()
    Vo_h = torch.empty(R.Vo.numel(), dtype=torch.float64).pin_memory()
    e2e_ms, parts = [], []
    # one untimed pass first, as for the device-only timing (the first copies into freshly pinned buffers
    # are not representative of the steady state)
    for it in range(1 + max(1, min(args.steps, 3))):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        with torch.cuda.stream(stream):
            R.A.copy_(R.A_host, non_blocking=True)
            ev[1].record(stream)
            R.step(ctx, stream)
            ev[2].record(stream)
            Wo_h.copy_(R.Wo, non_blocking=True)
            Vo_h.copy_(R.Vo, non_blocking=True)
        ev[3].record(stream)
        ev[3].synchronize()
        if it == 0:
            continue
        e2e_ms.append(ev[0].elapsed_time(ev[3]))
        parts.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
    e2e_t = float(np.mean(e2e_ms))
    h2d_ms, e2e_step_ms, d2h_ms = (float(x) for x in np.mean(parts, axis=0))
    if world > 1:
        t = torch.tensor([e2e_t], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
    e2e_value = job_pairs / (e2e_t / 1e3)
    roof = roofline(Z, prof, R.ns, args.steps)
    out = {
        "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "problems": len(R.ns), "eigenpairs_per_step": job_pairs,
                   "target": "quad-double", "method": method, "converged": ok and ok2, "unconverged": nbad2,
                   "max_err_over_normA": max_err, "err_bound": R.err_bound,
                   "l2": "flushed between timed steps" if flush is not None else "inputs larger than L2"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "breakdown_ms": {"jacobi_fp64": float(np.mean(jac_ms)), "refine": float(np.mean(ref_ms))},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "kernel_tflops": {k: v[2] / (v[0] / 1e3) / 1e12 for k, v in prof.items() if v[1] and v[2] > 0},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "eigenpairs/s", "h2d_bytes_per_step": int(in_bytes),
                "d2h_bytes_per_step": int((R.Wo.numel() + R.Vo.numel()) * 8),
                "h2d_ms": h2d_ms, "step_ms": e2e_step_ms, "d2h_ms": d2h_ms},
        "gpu_launches": int(sum(v[1] for v in prof.values())),
    }
    if args.workload == "batch256_qd" and not args.no_compare:
        # same-accuracy comparison of the two precision-recovery paths on the single 128x128 problem
        sp, _, _, _ = load_workload("single128_plain", rank, 1)
        cmp = {}
        for meth in ("plain", "chosen"):
            Rs = Runner(Z, torch, dev, sp, 4, meth)
            with torch.cuda.stream(stream):
                Rs.step(ctx, stream)
            torch.cuda.synchronize()
            ts = []
            for _ in range(2):
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                with torch.cuda.stream(stream):
                    Rs.step(ctx, stream)
                e1.record(stream); e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            cmp[meth] = {"eigenpairs_per_s": Rs.pairs / (float(np.mean(ts)) / 1e3), "ms": float(np.mean(ts)),
                         "converged": Rs.check()[0], "max_err_over_normA": Rs.check()[2]}
            del Rs
        out["plain_rqi_vs_chosen_single128"] = cmp
    if rank == 0 and not args.no_cpu_baseline:
        import workloads as W
        out["cpu_baseline"] = oracle_baseline(problems, [W.config_single128()] if len(problems) > 1 else [])
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def recorded_traffic(kernel_source):
    """DRAM bytes per launch from the committed ncu summary of the kernel, when the summary was taken of the
    kernel source as it is now (its sha256 matches); else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "jacobi_global_traffic.txt")
    try:
        fields = dict(l.split(":", 1) for l in open(path) if ":" in l)
        src = open(os.path.join(ROOT, kernel_source), "rb").read()
        if fields.get("source_sha256", "").strip() != hashlib.sha256(src).hexdigest():
            return None
        return int(fields["dram_bytes_per_launch"].strip())
    except Exception:
        return None


def roofline(Z, prof, ns, steps):
    """Roofline object of the dominant kernel class (by device time in the timed region)."""
    peaks, peak_kind = measured_peaks()
    dom_name, (dom_ms, dom_n, dom_work) = max(prof.items(), key=lambda kv: kv[1][0])
    base = {"launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1), "traffic": None}
    if dom_name == "ozaki_gemm":
        peak = peaks.get("bf16_tflops_sustained", 1700.0)   # fp16 dense = bf16 dense rate
        achieved = dom_work / (dom_ms / 1e3) / 1e12
        kern = ("oz_tc_kernel (tcgen05.mma kind::f16, TMEM accumulators)" if Z.zkq_get_gemm_kernel() == 1
                else "oz_gemm_kernel (mma.sync f16->f32)")
        return dict(base, bound="tensor", kernel=kern, achieved=achieved, peak=peak, unit="TFLOP/s",
                    frac=achieved / peak, peak_source=f"{peak_kind} bf16_tflops_sustained (fp16 dense has the bf16 rate)",
                    work="2 m (2n) (2k) flops per kept slice pair, unpadded sizes")
    if dom_name in ("jacobi", "jacobi_cluster"):
        peak = FP64_TFLOPS_PEAK
        achieved = dom_work / (dom_ms / 1e3) / 1e12
        what = "FP64 eigensolve of the inputs" if dom_name == "jacobi" else "FP64 eigensolves of the refinement's cluster blocks"
        if dom_name == "jacobi":   # the batch's large problems: one jacobi_global_kernel launch per step
            base["traffic"] = recorded_traffic("paper_2402_11868_gb300/csrc/jacobi.cu")
            base["traffic_kernel"] = "jacobi_global_kernel<4> (DRAM read + write per launch, ncu)"
        return dict(base, bound="alu", kernel=f"jacobi_smem/global/grid_kernel ({what})",
                    achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                    peak_source="derived: 152 SMs x 2 FP64 FMA per clock per SM x 2.07 GHz x 2 flops "
                                "(MEASURED_PEAKS.json has no FP64 entry)",
                    peak_measured_dfma=FP64_TFLOPS_MEASURED, frac_of_measured_dfma=achieved / FP64_TFLOPS_MEASURED,
                    work="32 n flops per applied rotation (16 n FMA: scaled Hermitian 2x2-block update of A 8 n + V 8 n)")
    if dom_name == "rqi":
        it = 2.0
        cmacs = sum(nn * (it * (nn ** 3 / 3.0 + nn * nn) + 2 * nn * nn) for nn in ns) * steps
        achieved = cmacs * QD_CMAC_INSTR / (dom_ms / 1e3) / 1e12
        return dict(base, bound="alu", kernel="rqi_kernel<4,4>", achieved=achieved, peak=FP64_INSTR_PEAK / 1e12,
                    unit="TFLOP/s", frac=achieved / (FP64_INSTR_PEAK / 1e12),
                    peak_source="derived: 152 SMs x 2 FP64 instructions per clock per SM x 2.07 GHz",
                    work="FP64 operations, one per DADD, DMUL or DFMA (1004 per complex quad-double multiply-add)")
    return dict(base, bound="alu", kernel=dom_name, achieved=None, peak=FP64_TFLOPS_PEAK, unit="TFLOP/s",
                frac=None)


def run_brickwork(args):
    """Two-qubit gate updates of a device-resident quad-double MPS (40 qubits, r_max 256): theta
    contraction, Gram eigensolve (FP64 Jacobi + refinement), truncation and split back per gate."""
    import torch
    import paper_2402_11868_gb300 as Z
    import workloads as W
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, r_max, words, tau = 40, 256, 4, 2.0 ** -200
    layers = args.warmup + args.steps
    gates, idx = [], 0                           # per layer: [(site, G)] on disjoint bonds
    for t in range(layers):
        layer = []
        for s_ in range(t % 2, n - 1, 2):
            layer.append((s_, W.haar_gate(3 + rank, idx, words)))
            idx += 1
        gates.append(layer)
    ctx = Z.Context(local)
    mps = Z.MPS(ctx, n, r_max=r_max, words=words)
    stream = torch.cuda.Stream(device=dev)
    for t in range(args.warmup):
        for site, G in gates[t]:
            mps.apply2q(site, G, trunc_tau=tau, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    Z.zkq_profile_enable(True)
    Z.zkq_profile_read()
    if world > 1:
        dist.barrier()
    step_ms, ngates, rho_pairs, disc = [], 0, 0, 0.0
    t_wall = time.perf_counter()
    for t in range(args.warmup, layers):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for site, G in gates[t]:
            chi = mps.bond_dims()
            a = 1 if site == 0 else int(chi[site - 1])
            d = 1 if site + 1 == n - 1 else int(chi[site + 1])
            rho_pairs += 2 * min(a, d)
            _, dw = mps.apply2q(site, G, trunc_tau=tau, stream=stream)
            disc += dw
            ngates += 1
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    prof = Z.zkq_profile_read()
    Z.zkq_profile_enable(False)
    clk = clocks.stop()
    total_ms = float(sum(step_ms))
    if world > 1:
        tt = torch.tensor([total_ms, wall], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms, wall = float(tt[0].item()), float(tt[1].item())
    chi = mps.bond_dims()
    out = {
        "metric": "two-qubit gate updates/sec of a quad-double MPS (n=40, r_max=256)",
        "value": ngates * world / (total_ms / 1e3), "unit": "gates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "brickwork40", "desc": "40-qubit brickwork of Haar 4x4 gates, r_max 256, QD, tau 2^-200",
                   "gates_timed": ngates, "layers_timed": args.steps, "max_bond_after": int(chi.max()),
                   "discarded_weight": disc},
        "eigenpairs_per_s": rho_pairs * world / (total_ms / 1e3),
        "latency_ms": {"p50_layer": float(np.percentile(step_ms, 50)), "p99_layer": float(np.percentile(step_ms, 99)),
                       "per_gate": total_ms / max(ngates, 1)},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "roofline": roofline(Z, prof, [], args.steps),
        "clocks": clk,
        "e2e": {"value": ngates * world / wall, "unit": "gates/s",
                "h2d_bytes_per_step": int(16 * 2 * words * 8 * ngates / args.steps),
                "d2h_bytes_per_step": int(12 * ngates / args.steps)},
        "gpu_launches": int(sum(v[1] for v in prof.values())),
    }
    mps.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_serve(args):
    """Continuous-batching request loop (paper_2402_11868_gb300.serve.Engine) on the serving configuration:
    64 MPS simulations with n ~ U{24..64} qubits and r_max ~ 2^U{5..10} (32..1024), half of them double-double
    and half quad-double, admitted by their HBM footprint (zkq_mps_footprint: the MPS at capacity and its
    widest gate update) into a 160 GB budget -- those that do not fit wait until admitted ones finish their
    gate quota and free their memory.  Requests arrive as an open Poisson stream at 0.7x the throughput
    measured with the warm-up requests submitted at once: half are gate updates (the next brickwork gate of
    a random admitted simulation, in its precision), half eigensolves (an order from the 256-problem batch's
    distribution, N <= 512, double-double or quad-double at random).  Per-type p50/p99 latency from arrival to
    completion."""
    import collections
    import torch
    import paper_2402_11868_gb300 as Z
    import workloads as W
    from paper_2402_11868_gb300.serve import Engine
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    per_step, quota, budget = 32, 12, 160 << 30
    rng = np.random.default_rng(4 + rank)
    eng = Engine(device=local, hbm_budget=budget, slots=4, max_batch=32)
    specs = [(int(rng.integers(24, 65)), int(2 ** rng.integers(5, 11)), 4 if k % 2 else 2) for k in range(64)]
    waiting = collections.deque(range(64))
    state = {}                                   # spec index -> [sid, gates issued, gates completed]
    refused = [k for k in range(64) if eng.mps_footprint(*specs[k]) > budget]
    for k in refused:
        waiting.remove(k)
    admitted_total, max_live = 0, 0
    lock = threading.Lock()

    def admit():
        nonlocal admitted_total, max_live
        with lock:
            while waiting:
                k = waiting[0]
                sid = eng.try_create_simulation(*specs[k])
                if sid is None:
                    break
                waiting.popleft()
                state[k] = [sid, 0, 0]
                admitted_total += 1
            max_live = max(max_live, len(state))

    def finished_gate(k):
        with lock:
            st_ = state[k]
            st_[2] += 1
            done = st_[2] >= quota
            if done:
                eng.destroy_simulation(st_[0])
                del state[k]
        if done:
            admit()

    admit()
    total_req = (args.warmup + args.steps) * per_step
    sizes = W.batch_sizes(4 + rank, total_req)
    kinds = rng.random(total_req) < 0.5            # True: eigensolve, False: gate
    precs = rng.random(total_req) < 0.5            # True: quad-double eigensolve

    def make(i):
        if kinds[i]:
            cfg = 2 if precs[i] else 1
            p = W.config_batch(cfg, seed=4 + rank, count=1, sizes=[sizes[i]])[0]
            return ("eig", p, 4 if cfg == 2 else 2)
        with lock:
            live = [k for k, v in state.items() if v[1] < quota]
            if not live:
                return None
            k = live[int(rng.integers(0, len(live)))]
            sid, g = state[k][0], state[k][1]
            state[k][1] += 1
        n_q, _, words = specs[k]
        layer, j = divmod(g, max(1, (n_q - 1) // 2))
        sites = list(range(layer % 2, n_q - 1, 2))
        site = sites[j % len(sites)]
        return ("gate", (k, sid, site, W.haar_gate(5 + rank, g + 1000 * k, words)), words)

    def submit(r):
        if r[0] == "eig":
            return eng.submit_eig(r[1].A, r[1].n, r[2])
        k, sid, site, G = r[1]
        h = eng.submit_gate(sid, site, G, 2.0 ** -(53 * r[2] - 12))
        threading.Thread(target=lambda: (h.done.wait(600), finished_gate(k)), daemon=True).start()
        return h

    def issue(i):
        r = make(i)
        while r is None:                          # every admitted simulation has all its gates issued
            time.sleep(0.01)
            r = make(i)
        return r, submit(r)

    # warm-up: the first half of the warm-up requests (first calls grow the contexts' workspaces and admit the
    # simulations); saturation: the second half submitted at once
    nw = args.warmup * per_step
    for h in [issue(i)[1] for i in range(nw // 2)]:
        h.done.wait(900)
    t0 = time.perf_counter()
    hs = [issue(i)[1] for i in range(nw // 2, nw)]
    for h in hs:
        h.done.wait(900)
    cap = len(hs) / (time.perf_counter() - t0)
    eng.completed.clear()
    rate = 0.7 * cap
    clocks = ClockSampler(local)
    clocks.start()
    gaps = rng.exponential(1.0 / rate, args.steps * per_step)
    t0 = time.perf_counter()
    out_reqs, t_next = [], t0
    for i, gp in zip(range(args.warmup * per_step, total_req), gaps):
        t_next += gp
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        out_reqs.append(issue(i))
    for _, h in out_reqs:
        h.done.wait(900)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    errors = [h.error for _, h in out_reqs if h.error]
    lat = {}
    for (r, h) in out_reqs:
        key = f"{r[0]}_{'qd' if r[2] == 4 else 'dd'}"
        lat.setdefault(key, []).append(1e3 * (h.t_done - h.t_arrive))
    stats = {k: {"count": len(v), "p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
             for k, v in sorted(lat.items())}
    eig_pairs = sum(r[1].n for r, h in out_reqs if r[0] == "eig" and not h.error)
    ngates = sum(1 for r, h in out_reqs if r[0] == "gate" and not h.error)
    all_lat = [x for v in lat.values() for x in v]
    out = {
        "metric": "serving: eigenpairs/s and p50/p99 request latency at 0.7x saturation (Poisson arrivals)",
        "value": eig_pairs / wall, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serve", "simulations": 64, "n_qubits": "U{24..64}", "r_max": "2^U{5..10}",
                   "sim_precision": "half double-double, half quad-double", "hbm_budget_gb": budget >> 30,
                   "gate_quota_per_simulation": quota, "admitted": admitted_total, "max_resident": max_live,
                   "refused_larger_than_budget": len(refused), "requests_timed": len(out_reqs),
                   "arrival_rate_per_s": rate, "saturated_requests_per_s": cap,
                   "eig_sizes": "N from the 256-problem batch distribution (16..512)", "errors": len(errors)},
        "latency_ms": {"p50": float(np.percentile(all_lat, 50)), "p99": float(np.percentile(all_lat, 99)),
                       "by_type": stats},
        "gates_per_s": ngates / wall,
        "clocks": clk,
        "e2e": {"value": eig_pairs / wall, "unit": "eigenpairs/s",
                "h2d_bytes_per_step": int(sum(r[1].A.nbytes for r, _ in out_reqs if r[0] == "eig") / args.steps),
                "d2h_bytes_per_step": int(sum(r[1].n * r[2] * 8 * (1 + 2 * r[1].n) for r, _ in out_reqs if r[0] == "eig") / args.steps)},
    }
    eng.close()
    if rank == 0:
        print(json.dumps(out))


def run_dj(args):
    """Deutsch-Jozsa-style circuits (workloads.dj_circuit: f(x) = x_0 + a band-graph quadratic form of band
    width 5, balanced) run gate by gate on a quad-double device MPS at widths 16, 32, 64 and 128: time per
    circuit against the width (the paper reports its DJ simulation time growing like n^3 with diagonalised
    matrices of at most 56 x 56), two-qubit gates/s, and the largest reduced matrix.  One step = one circuit
    at each width."""
    import torch
    import paper_2402_11868_gb300 as Z
    import workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    widths, w = (16, 32, 64, 128), 5
    ctx = Z.Context(local)
    stream = torch.cuda.Stream(device=dev)
    circuits = {n: W.dj_circuit(n, w, "balanced", seed=100 + n + rank) for n in widths}

    def one(n):
        _, gates, _ = circuits[n]
        mps = Z.MPS(ctx, n, r_max=1024, words=4)
        max_rho, n2 = 0, 0
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for kind, site, G in gates:
            if kind == "1q":
                mps.apply1q(site, G, stream=stream)
            else:
                chi = mps.bond_dims()
                a = 1 if site == 0 else int(chi[site - 1])
                d = 1 if site + 1 == n - 1 else int(chi[site + 1])
                max_rho = max(max_rho, 2 * min(a, d))
                mps.apply2q(site, G, trunc_tau=2.0 ** -200, stream=stream)
                n2 += 1
        e1.record(stream)
        e1.synchronize()
        mps.close()
        return e0.elapsed_time(e1), n2, max_rho

    for _ in range(args.warmup):
        one(widths[0])
    clocks = ClockSampler(local)
    clocks.start()
    per = {n: [] for n in widths}
    meta = {}
    for _ in range(args.steps):
        for n in widths:
            ms, n2, mr = one(n)
            per[n].append(ms)
            meta[n] = (n2, mr)
    clk = clocks.stop()
    t = {n: float(np.median(v)) for n, v in per.items()}
    slope = float(np.polyfit(np.log(widths), np.log([t[n] for n in widths]), 1)[0])
    big = widths[-1]
    total_ms = sum(sum(v) for v in per.values())
    out = {
        "metric": "Deutsch-Jozsa-style circuit simulation: two-qubit gate updates/s (quad double, width 128)",
        "value": meta[big][0] / (t[big] / 1e3), "unit": "gates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "dj", "desc": "f(x) = x_0 + band-graph quadratic form (band 5, edges by seed), "
                   "balanced; quad double, truncation 2^-200", "widths": list(widths)},
        "per_width": {str(n): {"ms_per_circuit": t[n], "two_qubit_gates": meta[n][0], "max_rho": meta[n][1]}
                      for n in widths},
        "time_vs_width_exponent": slope,
        "clocks": clk,
        "e2e": {"value": meta[big][0] / (t[big] / 1e3), "unit": "gates/s",
                "h2d_bytes_per_step": int(sum(16 * 2 * 4 * 8 * meta[n][0] for n in widths)),
                "d2h_bytes_per_step": int(sum(12 * meta[n][0] for n in widths))},
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(out))


def run_reference(args):
    """The oracle, as it stands, on the host cores: a bounded sample of the same workload per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads as W
    if args.workload == "single128_plain":
        sample = [W.herm_spectrum(7, 0, W.spectrum_single128(48), 4)]
        note = "one 48x48 problem with the single128 spectrum law per step"
    else:
        sizes = W.batch_sizes(1, args.count)
        idx = [i for i, n in enumerate(sizes) if n <= 48][:3] or [int(np.argmin(sizes))]
        sample = W.config_batch(2, seed=1, count=args.count, sizes=sizes, indices=idx)
        note = f"batch problems {idx} (N={[p.n for p in sample]}) per step, one per thread"
    threads = min(len(sample), os.cpu_count() or 1)
    for _ in range(args.warmup):
        oracle_rate(sample, threads)
    t = []
    for _ in range(args.steps):
        _, dt = oracle_rate(sample, threads)
        t.append(dt)
    pairs = sum(p.n for p in sample)
    value = pairs * args.steps / sum(t)
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": args.workload, "sample": note},
                      "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": threads, "kind": "oracle",
                                       "sample": note},
                      "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "brickwork40":
        run_brickwork(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "dj":
        run_dj(a)
    else:
        run_ours(a)
