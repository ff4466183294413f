"""Host-side scheduling logic of the CUDA path, checked on CPU by compiling the library's own headers and
sources with g++ against the CUDA headers (no GPU, no kernel):
* the parallel (circle) ordering of the Jacobi rounds, `rr_pair` in common.cuh: for m players (an even
  number: the order n, plus one dummy when n is odd) every round is a perfect matching, and the m - 1
  rounds of a sweep meet every unordered pair exactly once;
* the batch layout of the FP64 eigensolve, `eigh_layout` in layout.cu: the problem order (orders <= 80
  in input order, then the larger ones by decreasing order), the eigenvalue and workspace offsets, the
  cluster width (configured, from the tuning table, or by the largest order), and the block groups of the
  cooperative grid for a few large problems;
* the plain RQI layout, `rqi_layout` in layout.cu: the eigenpair-to-problem map, the grid and the
  workspace slots."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_11868_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

RR = r"""
#include "common.cuh"
extern "C" void rr_fill(int m, int* p, int* q) {
  for (int r = 0; r < m - 1; ++r)
    for (int k = 0; k < m / 2; ++k) zkq::rr_pair(m, r, k, p[r * (m / 2) + k], q[r * (m / 2) + k]);
}
"""

# layout.cu with the device-side entry points it references stubbed out; grid occupancy is a parameter
LAYOUT = r"""
#include "internal.cuh"
#include "prof.cuh"
namespace zkq {
static int g_grid_blocks_per_sm = 0;
int jacobi_grid_max_blocks(int, int) { return g_grid_blocks_per_sm; }
void set_last_cuda_error(cudaError_t) {}
unsigned long long* prof_device_counters() { return nullptr; }
Profiler& profiler() { static Profiler p; return p; }
void HostStage::add(void*, const void*, size_t) {}
cudaError_t HostStage::flush(cudaStream_t) { return cudaSuccess; }
zkq_status launch_jacobi(const JacobiBatch&, int, int, int, int, int, int, int, GridBar*, const int32_t*, int,
                         cudaStream_t) { return ZKQ_OK; }
zkq_status launch_rqi(const RqiBatch&, int, int, int, cudaStream_t) { return ZKQ_OK; }
size_t rqi_slot_doubles(int nmax, int W) { return ((size_t)nmax * (nmax + 1) + 2 * (size_t)nmax) * 2 * W; }
}
// the one runtime call layout.cu makes (in the RQI launch, which the test never reaches)
extern "C" cudaError_t cudaMemsetAsync(void*, int, size_t, cudaStream_t) { return cudaErrorNotSupported; }
extern "C" int layout_probe(int batch, const int* n, int cfg_cluster, int num_sms, int per_sm, int ntune,
                            const int* tune, int* scalars, int* order, long long* w_off, long long* ws_off,
                            int* grp, long long* bytes) {
  zkq::g_grid_blocks_per_sm = per_sm;
  std::vector<int64_t> a_off(batch, 0);
  zkq::JacobiTune t;
  for (int i = 0; i < ntune; ++i) t.push_back({tune[2 * i], tune[2 * i + 1]});
  zkq::EighLayout L;
  zkq_status s = zkq::eigh_layout(batch, n, a_off.data(), 4, cfg_cluster, num_sms, &L, &t);
  if (s != ZKQ_OK) return (int)s;
  scalars[0] = L.n_small; scalars[1] = L.n_large; scalars[2] = L.max_small; scalars[3] = L.max_large;
  scalars[4] = L.cluster; scalars[5] = L.grid_blocks; scalars[6] = L.red_stride; scalars[7] = (int)L.grp.size();
  for (int b = 0; b < batch; ++b) { order[b] = L.order[b]; w_off[b] = L.w_off[b]; ws_off[b] = L.ws_off[b]; }
  for (size_t i = 0; i < L.grp.size(); ++i) grp[i] = L.grp[i];
  bytes[0] = (long long)L.ws_need; bytes[1] = (long long)L.red_bytes; bytes[2] = (long long)L.gb_bytes;
  bytes[3] = (long long)L.meta_bytes(); bytes[4] = (long long)L.ws_bytes();
  return 0;
}
extern "C" int rqi_probe(int batch, const int* n, int target_words, int num_sms, long long* scalars, int* pair_prob,
                         long long* w_off) {
  std::vector<int64_t> a_off(batch, 0);
  zkq::RqiLayout L;
  zkq_status s = zkq::rqi_layout(batch, n, a_off.data(), target_words, num_sms, &L);
  if (s != ZKQ_OK) return (int)s;
  scalars[0] = L.total; scalars[1] = L.grid; scalars[2] = (long long)L.slot;
  scalars[3] = (long long)L.meta_bytes(); scalars[4] = (long long)L.ws_bytes();
  for (int64_t i = 0; i < L.total; ++i) pair_prob[i] = L.pair_prob[i];
  for (int b = 0; b < batch; ++b) w_off[b] = L.w_off[b];
  return 0;
}
"""


def _build(tmp, name, src, extra=()):
    (tmp / f"{name}.cpp").write_text(src)
    out = tmp / f"{name}.so"
    # the device helpers of common.cuh call fma unqualified, as nvcc allows: give the host compile ::fma
    # -Bsymbolic: the stubs bind inside this library even when a CUDA runtime is loaded with global symbols
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-Wl,-Bsymbolic", "-include", "math.h",
                    f"-I{CSRC}", f"-I{CUDA_INC}", "-x", "c++", str(tmp / f"{name}.cpp"), *extra, "-o", str(out)],
                   check=True, capture_output=True, text=True)
    return ctypes.CDLL(str(out))


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not available")
    tmp = tmp_path_factory.mktemp("sched")
    rr = _build(tmp, "rr", RR)
    lay = _build(tmp, "layout", LAYOUT, ["-x", "c++", os.path.join(CSRC, "layout.cu")])
    I, P = ctypes.c_int, ctypes.c_void_p
    rr.rr_fill.restype = None
    rr.rr_fill.argtypes = [I, P, P]
    lay.layout_probe.restype = I
    lay.layout_probe.argtypes = [I, P, I, I, I, I, P, P, P, P, P, P, P]
    lay.rqi_probe.restype = I
    lay.rqi_probe.argtypes = [I, P, I, I, P, P, P]
    return rr, lay


@pytest.mark.parametrize("m", [2, 4, 6, 82, 128, 130, 256, 514, 1024])
def test_circle_ordering_is_a_round_robin_tournament(libs, m):
    rr, _ = libs
    P = np.zeros((m - 1) * (m // 2), dtype=np.int32); Q = np.zeros_like(P)
    rr.rr_fill(m, P.ctypes.data, Q.ctypes.data)
    P = P.reshape(m - 1, m // 2); Q = Q.reshape(m - 1, m // 2)
    assert (P < Q).all() and (P >= 0).all() and (Q < m).all()
    for r in range(m - 1):                                   # each round: a perfect matching
        assert np.array_equal(np.sort(np.concatenate([P[r], Q[r]])), np.arange(m))
    key = (P.astype(np.int64) * m + Q).ravel()               # the sweep: every pair exactly once
    assert len(np.unique(key)) == m * (m - 1) // 2 == key.size


def _probe(lay, n, cfg_cluster=0, num_sms=152, per_sm=0, tune=()):
    b = len(n)
    na = np.array(n, dtype=np.int32)
    tn = np.array([x for pr in tune for x in pr] or [0], dtype=np.int32)
    sc = np.zeros(8, dtype=np.int32); order = np.zeros(b, dtype=np.int32)
    w_off = np.zeros(b, dtype=np.int64); ws_off = np.zeros(b, dtype=np.int64)
    grp = np.zeros(b + 1, dtype=np.int32); by = np.zeros(5, dtype=np.int64)
    rc = lay.layout_probe(b, na.ctypes.data, cfg_cluster, num_sms, per_sm, len(tune), tn.ctypes.data, sc.ctypes.data,
                          order.ctypes.data, w_off.ctypes.data, ws_off.ctypes.data, grp.ctypes.data, by.ctypes.data)
    if rc:
        return rc
    return dict(n_small=sc[0], n_large=sc[1], max_small=sc[2], max_large=sc[3], cluster=sc[4], grid_blocks=sc[5],
                red_stride=sc[6], grp=list(grp[:sc[7]]), order=list(order), w_off=list(w_off), ws_off=list(ws_off),
                ws_need=by[0], red_bytes=by[1], gb_bytes=by[2], meta=by[3], ws=by[4])


al = lambda x: (x + 255) // 256 * 256


def test_eigh_layout_order_offsets_and_cluster_width(libs):
    _, lay = libs
    n = [16, 200, 81, 512, 80, 300, 200, 3]
    L = _probe(lay, n)
    small = [i for i, x in enumerate(n) if x <= 80]
    large = sorted([i for i, x in enumerate(n) if x > 80], key=lambda i: (-n[i], i))
    assert L["order"] == small + large
    assert (L["n_small"], L["n_large"], L["max_small"], L["max_large"]) == (3, 5, 80, 512)
    assert L["w_off"] == list(np.cumsum([0] + n[:-1]))
    acc = 0
    for i in large:                                          # A and V copies of the large problems, in order
        assert L["ws_off"][i] * 8 == acc
        acc += al(n[i] * n[i] * 4 * 8)
    assert all(L["ws_off"][i] == 0 for i in small) and L["ws_need"] == acc
    assert L["cluster"] == 8                                 # largest order above 256, no grid (occupancy 0)
    assert L["grid_blocks"] == 0 and L["grp"] == []
    assert L["ws"] == L["ws_need"] + L["red_bytes"] + L["gb_bytes"]
    for top, width in ((128, 2), (256, 4), (257, 8)):
        assert _probe(lay, [16, top])["cluster"] == width
    assert _probe(lay, [300], cfg_cluster=16)["cluster"] == 16
    tune = [(128, 4), (512, 16)]
    assert _probe(lay, [100, 300], tune=tune)["cluster"] == 16   # first table order >= 300
    assert _probe(lay, [100, 120], tune=tune)["cluster"] == 4
    assert _probe(lay, [1000], tune=tune)["cluster"] == 16       # beyond the table: its last entry
    assert _probe(lay, [16, 4097]) == 1 and _probe(lay, [0]) == 1   # ZKQ_EINVAL


def test_eigh_layout_block_groups_for_few_large_problems(libs):
    """A few large problems (cluster width x 2 x count <= SMs) run as block groups of one cooperative grid:
    about n^2 / 2048 blocks (2 .. 128) per problem, in the problem order, scaled down by each problem's
    share of the n^3 work when they do not fit the co-resident blocks."""
    _, lay = libs
    L = _probe(lay, [512, 300, 40], per_sm=4)                # co-resident: 4 x 152 = 608 blocks
    want = [min(128, max(2, x * x // 2048)) for x in (512, 300)]
    assert L["grp"] == [0, want[0], want[0] + want[1]] and L["grid_blocks"] == sum(want)
    assert L["red_stride"] == 2 * max(want) + 64
    assert L["red_bytes"] == max(al(64 * 2 * 8), al(L["red_stride"] * 2 * 8))
    L = _probe(lay, [512] * 9, per_sm=4)                     # 9 x 128 > 608: scaled by the n^3 share
    each = max(1, min(128, int(608 * 512**3 / (9 * 512**3))))
    assert L["grp"] == [each * k for k in range(10)] and L["grid_blocks"] <= 608
    assert _probe(lay, [512] * 10, per_sm=4)["grid_blocks"] == 0   # 10 x 8 x 2 > 152: a cluster each
    assert _probe(lay, [512, 300], per_sm=0)["grid_blocks"] == 0   # no co-residency information: clusters


def test_rqi_layout_maps_every_eigenpair_to_its_problem(libs):
    """The plain RQI layout: one work item per eigenpair, mapped to its problem in batch order, a grid of
    min(eigenpairs, SMs) persistent blocks, each with a workspace slot sized for the largest order (the
    LU of A - mu I plus two vectors, complex, W words)."""
    _, lay = libs
    n = [3, 5, 2, 1, 4]
    na = np.array(n, dtype=np.int32)
    sc = np.zeros(5, dtype=np.int64); pp = np.zeros(sum(n), dtype=np.int32); wo = np.zeros(len(n), dtype=np.int64)
    assert lay.rqi_probe(len(n), na.ctypes.data, 4, 152, sc.ctypes.data, pp.ctypes.data, wo.ctypes.data) == 0
    assert sc[0] == sum(n) and sc[1] == min(sum(n), 152)
    assert list(pp) == [b for b, x in enumerate(n) for _ in range(x)]
    assert list(wo) == list(np.cumsum([0] + n[:-1]))
    nmax = max(n)
    assert sc[2] == (nmax * (nmax + 1) + 2 * nmax) * 2 * 4 and sc[4] == sc[2] * 8 * sc[1]
    big = np.array([300] * 2, dtype=np.int32)
    pp2 = np.zeros(600, dtype=np.int32)
    assert lay.rqi_probe(2, big.ctypes.data, 2, 152, sc.ctypes.data, pp2.ctypes.data, wo.ctypes.data) == 0
    assert sc[1] == 152
