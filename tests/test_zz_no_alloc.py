"""The no-allocation FP64 eigensolve entry point (for callers that cannot allocate device memory, e.g.
code that runs while another part of the process captures a CUDA graph, or a host with a fixed memory
budget).  It must give the results of zkq_eigh_batched on the same inputs, on consecutive calls that share
its fixed scratch, and refuse requests larger than that scratch.  Collected last on purpose."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _problems():
    # orders <= 80 run from shared memory; larger ones use the fixed scratch
    sizes = [5, 33, 80, 96, 130, 200]
    return [W.herm_spectrum(71, i, W.spectrum_graded(n, 40), 4) for i, n in enumerate(sizes)]


def _run(Z, torch, probs, use_noalloc, ctx=None):
    ns = [p.n for p in probs]
    a_off, w_off, tot_a, tot_w = Z.batch_offsets(ns)
    A = torch.from_numpy(Z.pack([p.A for p in probs], 4)).cuda()
    Wd = torch.full((tot_w,), np.nan, dtype=torch.float64, device="cuda")
    Vd = torch.full((2 * tot_a,), np.nan, dtype=torch.float64, device="cuda")
    info = torch.full((len(ns),), -7, dtype=torch.int32, device="cuda")
    if use_noalloc:
        Z.zkq_eigh_batched_noalloc(ns, a_off, A, 4, Wd, Vd, info)
    else:
        Z.zkq_eigh_batched(ctx, ns, a_off, A, 4, Wd, Vd, info)
    torch.cuda.synchronize()
    return Wd.cpu().numpy(), Vd.cpu().numpy(), info.cpu().numpy(), a_off, w_off


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch
    import paper_2402_11868_gb300 as Z
    Z.build()
    probs = _problems()
    with Z.Context(0) as ctx:
        W_ref, V_ref, info_ref, a_off, w_off = _run(Z, torch, probs, False, ctx)
    assert (info_ref == 0).all()
    for call in range(2):
        Wn, Vn, info, _, _ = _run(Z, torch, probs, True)
        assert (info == 0).all(), (call, info)
        for b, p in enumerate(probs):
            n = p.n
            lam = Wn[w_off[b]:w_off[b] + n]
            lam_ref = W_ref[w_off[b]:w_off[b] + n]
            anorm = max(abs(lam_ref).max(), 1e-300)
            tol = 8 * n * 2.0**-53 * anorm          # the FP64-stage tolerance of the parity tests
            assert np.all(np.abs(lam - lam_ref) <= tol), (call, n)
            V = Vn[2 * a_off[b]:2 * (a_off[b] + n * n)].reshape(n * n, 2, 1)
            Vr = V_ref[2 * a_off[b]:2 * (a_off[b] + n * n)].reshape(n * n, 2, 1)
            # the allocating path runs these three orders above 80 on its cooperative-grid kernel, the
            # no-allocation path on the cluster kernel: the eigenvectors agree within the FP64 tolerance
            assert np.abs(V - Vr).max() <= tol, (call, n)
            res, orth = oracle.residual(p.A, n, lam.reshape(n, 1), V, cols=list(range(min(n, 8))))
            assert res.max() <= tol and orth.max() <= 8 * n * 2.0**-53, (call, n, res.max(), orth.max())


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    import paper_2402_11868_gb300 as Z
    Z.build()
    n = 1100                                   # needs 32 n^2 bytes = 38.7 MB > 32 MiB of scratch
    assert 32 * n * n > Z.ZKQ_NOALLOC_SCRATCH_BYTES
    A = torch.zeros(16, dtype=torch.float64, device="cuda")
    Wd = torch.zeros(16, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(Z.ZkqError) as ei:
        Z.zkq_eigh_batched_noalloc([n], [0], A, 4, Wd, Wd, info)
    assert ei.value.status == Z.ZKQ_ETOOBIG


def test_noalloc_bitwise_equal_where_both_take_the_cluster_kernel():
    """40 problems of orders 81..120: too many for the allocating path's cooperative-grid class (40 problems
    x 2 CTAs x 2 > 152 SMs), so both paths run the cluster kernel at the same width and must give the same
    bits."""
    import torch
    import paper_2402_11868_gb300 as Z
    Z.build()
    sizes = [81 + (7 * i) % 40 for i in range(40)]
    probs = [W.herm_spectrum(73, i, W.spectrum_graded(n, 40), 2) for i, n in enumerate(sizes)]

    def run(use_noalloc, ctx=None):
        ns = [p.n for p in probs]
        a_off, _, tot_a, tot_w = Z.batch_offsets(ns)
        A = torch.from_numpy(Z.pack([p.A for p in probs], 2)).cuda()
        Wd = torch.full((tot_w,), np.nan, dtype=torch.float64, device="cuda")
        Vd = torch.full((2 * tot_a,), np.nan, dtype=torch.float64, device="cuda")
        info = torch.full((len(ns),), -7, dtype=torch.int32, device="cuda")
        if use_noalloc:
            Z.zkq_eigh_batched_noalloc(ns, a_off, A, 2, Wd, Vd, info)
        else:
            Z.zkq_eigh_batched(ctx, ns, a_off, A, 2, Wd, Vd, info)
        torch.cuda.synchronize()
        return Wd.cpu().numpy(), Vd.cpu().numpy(), info.cpu().numpy()

    with Z.Context(0) as ctx:
        W_ref, V_ref, info_ref = run(False, ctx)
    assert (info_ref == 0).all()
    for call in range(2):
        Wn, Vn, info = run(True)
        assert (info == 0).all(), (call, info)
        assert np.array_equal(Wn, W_ref) and np.array_equal(Vn, V_ref), call


def test_noalloc_refuses_to_run_inside_a_stream_capture():
    """The call uploads its metadata from host memory that it frees on return, so it must not be recorded
    into a CUDA graph: it returns ZKQ_EINVAL on a capturing stream and enqueues nothing."""
    import torch
    import paper_2402_11868_gb300 as Z
    Z.build()
    n = 12
    p = W.herm_spectrum(74, 0, W.spectrum_graded(n, 40), 4)
    A = torch.from_numpy(Z.pack([p.A], 4)).cuda()
    Wd = torch.zeros(n, dtype=torch.float64, device="cuda")
    Vd = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    raised = None
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            x.add_(1.0)
            try:
                Z.zkq_eigh_batched_noalloc([n], [0], A, 4, Wd, Vd, info, stream=s)
            except Z.ZkqError as e:
                raised = e
    assert raised is not None and raised.status == Z.ZKQ_EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    # outside the capture the same call runs
    Z.zkq_eigh_batched_noalloc([n], [0], A, 4, Wd, Vd, info)
    torch.cuda.synchronize()
    assert int(info[0]) == 0
