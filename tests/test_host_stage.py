"""The pinned staging ring of a context (HostStage, stage.cu) on CPU, against a simulated CUDA runtime in
which the device reads a copy's pinned source only later, when an event recorded behind the copy (or the
stream) is synchronised, as an asynchronous DMA may.  If the ring handed out a region while a copy that
reads it was still pending, the later copy would move the overwritten bytes.  Thousands of uploads of
mixed sizes, batched uploads and synchronous downloads, including growth of the ring past its first
capacity, must all deliver their exact bytes.  stage.cu is compiled with g++ against the CUDA headers;
the runtime entry points it calls are defined by the test (no GPU, no libcudart)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_11868_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

SIM = r"""
#include <cstdlib>
#include <cstring>
#include <vector>
#include "internal.cuh"
struct CUevent_st { size_t mark; };
namespace {
struct Copy { void* dst; const void* src; size_t n; };
std::vector<Copy> g_pending;      // issued, not yet performed
size_t g_done = 0;                // copies performed so far (a prefix of g_pending)
long g_event_syncs = 0;
void perform(size_t upto) {
  for (; g_done < upto && g_done < g_pending.size(); ++g_done)
    std::memcpy(g_pending[g_done].dst, g_pending[g_done].src, g_pending[g_done].n);
}
}
extern "C" {
cudaError_t cudaHostAlloc(void** p, size_t n, unsigned int) { *p = std::malloc(n); return *p ? cudaSuccess : cudaErrorMemoryAllocation; }
cudaError_t cudaFreeHost(void* p) { std::free(p); return cudaSuccess; }
cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned int) { *e = new CUevent_st{0}; return cudaSuccess; }
cudaError_t cudaEventDestroy(cudaEvent_t e) { delete e; return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t) { e->mark = g_pending.size(); return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t e) { ++g_event_syncs; perform(e->mark); return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { perform(g_pending.size()); return cudaSuccess; }
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind, cudaStream_t) {
  g_pending.push_back({d, s, n}); return cudaSuccess;
}
cudaError_t cudaGetDevice(int* d) { *d = 0; return cudaSuccess; }
cudaError_t cudaDeviceGetAttribute(int* v, cudaDeviceAttr, int) { *v = 0; return cudaSuccess; }
cudaError_t cudaFuncGetAttributes(cudaFuncAttributes* a, const void*) { std::memset(a, 0, sizeof(*a)); return cudaSuccess; }
cudaError_t cudaFuncSetAttribute(const void*, cudaFuncAttribute, int) { return cudaSuccess; }

void* stage_new() { return new zkq::HostStage(); }
void stage_free(void* h) { perform(g_pending.size()); delete (zkq::HostStage*)h; }
int stage_upload(void* h, void* dst, const void* src, size_t n) { return (int)((zkq::HostStage*)h)->upload(dst, src, n, nullptr); }
void stage_add(void* h, void* dst, const void* src, size_t n) { ((zkq::HostStage*)h)->add(dst, src, n); }
int stage_flush(void* h) { return (int)((zkq::HostStage*)h)->flush(nullptr); }
int stage_download(void* h, void* dst, const void* src, size_t n) { return (int)((zkq::HostStage*)h)->download_sync(dst, src, n, nullptr); }
void sim_finish() { perform(g_pending.size()); }
long sim_event_syncs() { return g_event_syncs; }
long sim_pending() { return (long)(g_pending.size() - g_done); }
}
"""


@pytest.fixture(scope="module")
def sim(tmp_path_factory):
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not available")
    d = tmp_path_factory.mktemp("stage")
    (d / "sim.cpp").write_text(SIM)
    so = d / "stage_sim.so"
    # -Bsymbolic: the simulated runtime entry points bind inside this library even when a real CUDA runtime
    # is already loaded into the process with global symbols
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-Wl,-Bsymbolic", "-include", "math.h",
                    f"-I{CSRC}", f"-I{CUDA_INC}", "-x", "c++", str(d / "sim.cpp"), "-x", "c++",
                    os.path.join(CSRC, "stage.cu"), "-o", str(so)], check=True, capture_output=True, text=True)
    L = ctypes.CDLL(str(so))
    P, S = ctypes.c_void_p, ctypes.c_size_t
    L.stage_new.restype = P
    L.stage_free.argtypes = [P]
    for nm in ("stage_upload", "stage_download"):
        getattr(L, nm).restype = ctypes.c_int
        getattr(L, nm).argtypes = [P, P, P, S]
    L.stage_add.argtypes = [P, P, P, S]
    L.stage_flush.restype = ctypes.c_int
    L.stage_flush.argtypes = [P]
    L.sim_event_syncs.restype = ctypes.c_long
    L.sim_pending.restype = ctypes.c_long
    return L


def test_staged_copies_deliver_their_bytes_when_the_device_reads_late(sim):
    rng = np.random.default_rng(5)
    h = sim.stage_new()
    keep, checks = [], []
    sizes = list(rng.integers(1, 200_000, 1500)) + [20 << 20, 3 << 20, 40 << 20]   # the last ones grow the ring
    rng.shuffle(sizes)
    i = 0
    while i < len(sizes):
        kind = rng.integers(0, 10)
        if kind < 6:                                          # one upload
            n = int(sizes[i]); i += 1
            src = rng.integers(0, 256, n, dtype=np.uint8); dst = np.zeros(n, dtype=np.uint8)
            assert sim.stage_upload(h, dst.ctypes.data, src.ctypes.data, n) == 0
            keep.append((src, dst)); checks.append((src.copy(), dst))
            src[:] = 0                                        # the caller may reuse its memory at once
        elif kind < 9:                                        # a batch of pieces, one flush
            k = int(rng.integers(1, 6))
            for _ in range(min(k, len(sizes) - i)):
                n = int(sizes[i]) // 7 + 1; i += 1
                src = rng.integers(0, 256, n, dtype=np.uint8); dst = np.zeros(n, dtype=np.uint8)
                sim.stage_add(h, dst.ctypes.data, src.ctypes.data, n)
                keep.append((src, dst)); checks.append((src.copy(), dst))
                src[:] = 0
            assert sim.stage_flush(h) == 0
        else:                                                 # a synchronous read-back
            n = int(sizes[i]) // 3 + 1; i += 1
            dev = rng.integers(0, 256, n, dtype=np.uint8); out = np.zeros(n, dtype=np.uint8)
            assert sim.stage_download(h, out.ctypes.data, dev.ctypes.data, n) == 0
            assert np.array_equal(out, dev)                   # complete on return
            keep.append((dev, out))
    assert sim.sim_pending() > 0                              # the device is still behind at the end
    sim.sim_finish()
    for want, dst in checks:
        assert np.array_equal(dst, want)
    assert sim.sim_event_syncs() > 0                          # the ring did wait for copies to reuse space
    sim.stage_free(h)
