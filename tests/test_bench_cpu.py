"""The benchmark's reference arm runs the oracle on host cores and prints one JSON line with the
contract's keys (no GPU needed); the roofline helper keeps the recorded traffic only for the kernel
source it was measured on."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "batch256_qd"


def test_recorded_traffic_needs_the_measured_source(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    import hashlib
    h = hashlib.sha256(b"kernel v1").hexdigest()
    (tmp_path / "profiles" / "jacobi_global_traffic.txt").write_text(
        f"source_sha256: {h}\ndram_bytes_per_launch: 12345\n")
    assert bench.recorded_traffic("k.cu") == 12345
    src.write_text("kernel v2")                      # the kernel changed since the counters were taken
    assert bench.recorded_traffic("k.cu") is None


class _FakeLib:
    @staticmethod
    def zkq_get_gemm_kernel():
        return 1


def test_roofline_objects_of_each_dominant_class():
    """The roofline object has the contract's keys for whichever kernel class dominates; FP64-pipe classes
    use the FP64 peak derived from 152 SMs x 2 operations per clock x 2.07 GHz."""
    sys.path.insert(0, ROOT)
    import bench
    ns = [128]
    for dom, work in (("jacobi", 6.0e11), ("jacobi_cluster", 5.0e11), ("ozaki_gemm", 4.0e14), ("rqi", 0.0),
                      ("oa_elementwise", 0.0)):
        prof = {"jacobi": (100.0, 3, 1.0e10), "ozaki_gemm": (50.0, 7, 1.0e12), dom: (1000.0, 4, work)}
        r = bench.roofline(_FakeLib, prof, ns, 2)
        for k in ("bound", "peak", "unit", "frac", "traffic", "launches", "avg_launch_ms"):
            assert k in r, (dom, k)
        assert r["launches"] == 4 and r["avg_launch_ms"] == 250.0
        assert r["unit"] in ("GB/s", "TFLOP/s")
        if dom == "ozaki_gemm":
            assert r["bound"] == "tensor" and abs(r["achieved"] - 400.0) < 1e-9
        else:
            assert r["bound"] == "alu"
        if dom.startswith("jacobi"):
            assert abs(r["peak"] - 1.25856) < 1e-4 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
            assert r["peak_measured_dfma"] == 1.006


def test_clock_sampler_summary_from_nvidia_smi_rows():
    """The clocks object of the bench line: median SM clock under load, the maximum, and every throttle
    reason seen Active (rows as nvidia-smi prints them with the bench's query fields)."""
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.rows = [["2070", "2070", "900.5", "0x0000000000000000", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["1980", "2070", "1390.2", "0x0000000000000004", "Not Active", "Not Active", "Not Active", "Active"],
               ["2010", "2070", "1200.0", "0x0000000000000000", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]"]]
    r = cs.stop()
    assert r == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    cs.rows = [["1500", "2070", "700", "0x8", "Active", "Not Active", "Not Active", "Not Active"]]
    assert cs.stop()["reasons"] == ["hw_slowdown"]
