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

METRIC = "quad-double refined eigenpairs/sec (err <=2^-200||A||), p50/p99 latency vs plain RQI path"
# FP64 pipe instruction rate of one GB300 measured by a DFMA-throughput microbenchmark on this machine
# (1.006 TFLOP/s counting an FMA as two flops, i.e. 0.503 T FP64 instructions/s)
FP64_INSTR_PEAK = 0.503e12
# FP64 instructions of one complex quad-double multiply-add (QD mul 142, QD add 109; 4 mul + 4 add)
QD_CMAC_INSTR = 4 * 142 + 4 * 109


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch256_qd", choices=["batch256_qd", "single128_plain"])
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
def load_workload(name, seed, count):
    import workloads as W
    if name == "single128_plain":
        return [W.config_single128(seed=seed)], 4, "plain", "single 128x128 Hermitian, lambda_k=2^-0.3(k-1), QD input"
    return (W.config_batch(2, seed=1 + seed, count=count), 4, "chosen",
            f"{count} Hermitian problems, N~U{{16..512}}, lambda graded to 2^-180, 8 pairs split 2^-60 (rel), QD input")


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

    def step(self, ctx, s):
        Z, torch = self.Z, self.torch
        Z.zkq_eigh_batched(ctx, self.ns, self.a_off, self.A, self.words, self.W, self.V, self.info, stream=s)
        em = torch.cuda.Event(enable_timing=True)
        em.record(s)
        Z.zkq_rqi_refine(ctx, self.ns, self.a_off, self.A, self.words, self.W, self.V, self.target, self.method,
                         self.Wo, self.Vo, self.err, self.rinfo, stream=s)
        return em

    def check(self):
        info, rinfo = self.info.cpu().numpy(), self.rinfo.cpu().numpy()
        return bool((info == 0).all() and (rinfo == 0).all()), int((info != 0).sum() + (rinfo != 0).sum())


def oracle_rate(problems, threads):
    """Oracle (320-bit Jacobi) eigenpairs/s on the given problems, one problem per host thread."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda p: oracle.eigh(p.A, p.n), problems))
    dt = time.perf_counter() - t0
    return sum(p.n for p in problems) / dt, dt


def stratified_sample(problems, sizes=(16, 32, 48, 64, 80)):
    out = []
    for s in sizes:
        for p in problems:
            if p.n == s:
                out.append(p)
                break
    return out or problems[:1]


def run_ours(args):
    import torch
    import paper_2402_11868_gb300 as Z
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    problems, words, method, desc = load_workload(args.workload, rank, args.count)
    R = Runner(Z, torch, dev, problems, words, method)
    ctx = Z.Context(local)
    stream = torch.cuda.Stream(device=dev)
    in_bytes = R.A.numel() * 8
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if in_bytes < (256 << 20) else None
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            R.step(ctx, stream)
    torch.cuda.synchronize()
    ok, nbad = R.check()
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
    ok2, nbad2 = R.check()
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = R.pairs * world * args.steps / (total_ms / 1e3)
    # end to end through the C ABI: pinned host input -> device, hot path, results back to pinned host
    Wo_h = torch.empty(R.Wo.numel(), dtype=torch.float64).pin_memory()
    Vo_h = torch.empty(R.Vo.numel(), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            R.A.copy_(R.A_host, non_blocking=True)
            R.step(ctx, stream)
            Wo_h.copy_(R.Wo, non_blocking=True)
            Vo_h.copy_(R.Vo, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = R.pairs / (float(np.mean(e2e_ms)) / 1e3)
    # dominant kernel class by device time in the timed region
    peaks, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n, dom_work) = dom
    if dom_name == "ozaki_gemm":
        peak = peaks.get("bf16_tflops_sustained", 1700.0)   # fp16 dense = bf16 dense rate
        achieved = dom_work / (dom_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "kernel": "oz_gemm_kernel (mma.sync f16->f32 digit slices)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{peak_kind} bf16_tflops_sustained (fp16 dense has the bf16 rate)",
                "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1)}
    elif dom_name == "jacobi":
        peak = 1.006   # measured DFMA throughput of this GB300 pool, TFLOP/s (FMA = 2 flops)
        achieved = dom_work / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "jacobi_smem_kernel + jacobi_global_kernel (FP64 rotations)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "measured FP64 DFMA microbenchmark (MEASURED_PEAKS.json has no FP64 entry)",
                "work": "48 n flops per applied rotation (24 n FMA: Hermitian 2x2-block update of A 12 n + V 12 n)",
                "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1)}
    elif dom_name == "rqi":
        it = 2.0
        cmacs = sum(nn * (it * (nn ** 3 / 3.0 + nn * nn) + 2 * nn * nn) for nn in R.ns) * args.steps
        achieved = cmacs * QD_CMAC_INSTR / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "rqi_kernel<4,4>", "achieved": achieved, "peak": FP64_INSTR_PEAK / 1e12,
                "unit": "TFLOP/s", "frac": achieved / (FP64_INSTR_PEAK / 1e12), "traffic": None,
                "peak_source": "measured DFMA issue rate (FP64 instructions/s, one op per DADD/DMUL/DFMA)",
                "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1)}
    else:
        roof = {"bound": "alu", "kernel": dom_name, "achieved": None, "peak": FP64_INSTR_PEAK / 1e12, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1)}
    out = {
        "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "problems": len(R.ns), "eigenpairs_per_step": R.pairs,
                   "target": "quad-double", "method": method, "converged": ok and ok2, "unconverged": nbad2,
                   "l2": "flushed between timed steps" if flush is not None else "inputs larger than L2"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "breakdown_ms": {"jacobi_fp64": float(np.mean(jac_ms)), "refine": float(np.mean(ref_ms))},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "kernel_tflops": {k: v[2] / (v[0] / 1e3) / 1e12 for k, v in prof.items() if v[1] and v[2] > 0},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "eigenpairs/s", "h2d_bytes_per_step": int(in_bytes),
                "d2h_bytes_per_step": int((R.Wo.numel() + R.Vo.numel()) * 8)},
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
                         "converged": Rs.check()[0]}
            del Rs
        out["plain_rqi_vs_chosen_single128"] = cmp
    if rank == 0 and not args.no_cpu_baseline:
        sample = stratified_sample(problems) if len(problems) > 1 else problems
        cores = min(len(sample), os.cpu_count() or 1)
        rate, dt = oracle_rate(sample, cores)
        out["cpu_baseline"] = {"value": rate, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
                               "sample": f"oracle (320-bit Jacobi) on {len(sample)} problem(s) of the workload "
                                         f"(N={[p.n for p in sample]}), one per thread, {dt:.1f} s"}
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


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
    run_reference(a) if a.impl == "reference" else run_ours(a)
