"""GPU parity of the split (Ozaki) products and of the Ogita-Aishima refinement against the oracle."""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._util import fr
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2402_11868_gb300 as Z
    Z.build()
    c = Z.Context(0)
    yield c
    c.close()


def rand_mw(rng, count, w, spread=6):
    """complex multi-word entries (count, 2, w) with per-entry exponents spread over 2^-spread..2^spread"""
    x = np.zeros((count, 2, w))
    e = rng.integers(-spread, spread + 1, size=(count, 2))
    x[:, :, 0] = np.ldexp(rng.standard_normal((count, 2)), e)
    for k in range(1, w):
        x[:, :, k] = x[:, :, k - 1] * 2.0**-54 * rng.uniform(-1, 1, (count, 2))
    return x


CASES = [(1, 1, 1, 0), (3, 5, 7, 1), (17, 33, 16, 0), (130, 40, 70, 1), (64, 48, 512, 0), (40, 3, 600, 1)]


@pytest.mark.parametrize("kernel", [1, 0])
@pytest.mark.parametrize("method", [1, 2, 0])
@pytest.mark.parametrize("wa,wb,wc", [(4, 4, 4), (4, 2, 4), (2, 1, 2), (1, 4, 4)])
def test_split_products_match_exact(ctx, method, wa, wb, wc, kernel):
    import torch
    import paper_2402_11868_gb300 as Z
    if method == 0 and kernel == 0:
        pytest.skip("method 0 does not use the slice-GEMM kernels")
    Z.zkq_set_gemm_kernel(kernel)
    rng = np.random.default_rng(1000 * wa + 100 * wb + 10 * wc + method)
    As, Bs, ms, ns, ks, ops = [], [], [], [], [], []
    for (m, n, k, op) in CASES:
        A = rand_mw(rng, m * k, wa)
        B = rand_mw(rng, k * n, wb)
        As.append(A); Bs.append(B); ms.append(m); ns.append(n); ks.append(k); ops.append(op)
    a_off = np.cumsum([0] + [a.shape[0] for a in As[:-1]]); b_off = np.cumsum([0] + [b.shape[0] for b in Bs[:-1]])
    c_sz = [m * n for m, n in zip(ms, ns)]; c_off = np.cumsum([0] + c_sz[:-1])
    dA = torch.from_numpy(np.concatenate([a.reshape(-1) for a in As])).cuda()
    dB = torch.from_numpy(np.concatenate([b.reshape(-1) for b in Bs])).cuda()
    dC = torch.zeros(sum(c_sz) * 2 * wc, dtype=torch.float64, device="cuda")
    p_bits = 53 * wc + 6
    Z.zkq_mw_gemm(ctx, ms, ns, ks, ops, dA, a_off, wa, dB, b_off, wb, dC, c_off, wc, p_bits, method)
    torch.cuda.synchronize()
    Z.zkq_check_device_waits()
    Z.zkq_set_gemm_kernel(1)
    Ch = dC.cpu().numpy()
    for i, (m, n, k, op) in enumerate(CASES):
        ref = oracle.matmul(As[i], Bs[i], m, n, k, opA=op)
        got = Ch[2 * wc * c_off[i]: 2 * wc * (c_off[i] + m * n)].reshape(m * n, 2, wc)
        Am = np.abs(As[i][:, :, 0]).max(axis=1)
        # row maxima of op(A): A is m x k (element i + l m) or, for op = A^H, k x m (element l + i k)
        rowmax = Am.reshape(k, m).max(axis=0) if op == 0 else Am.reshape(m, k).max(axis=1)
        colmax = np.abs(Bs[i][:, :, 0]).max(axis=1).reshape(k, n, order="F").max(axis=0)
        for jj in range(n):
            for ii in range(m):
                e = ii + jj * m
                if method in (1, 2):
                    bound = k * 2.0 ** -p_bits * (8 * rowmax[ii]) * (8 * colmax[jj]) * 2
                else:
                    bound = k * 2.0 ** -(53 * wc - 4) * rowmax[ii] * colmax[jj] * 4
                for part in range(2):
                    d = abs(float(fr(got[e, part]) - fr(ref[e, part])))
                    assert d <= bound, (i, ii, jj, part, d, bound)


def dyadic_mw(rng, count, w, ibits, espread):
    """complex entries (count, 2, w): integers below 2^ibits times 2^e with e in [-espread, espread] (the leading
    word holds them exactly; lower words zero)"""
    x = np.zeros((count, 2, w))
    ints = rng.integers(-(1 << ibits) + 1, 1 << ibits, size=(count, 2)).astype(np.float64)
    x[:, :, 0] = np.ldexp(ints, rng.integers(-espread, espread + 1, size=(count, 2)))
    return x


@pytest.mark.parametrize("kernel", [1, 0])
@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("w", [4, 2])
def test_split_products_bit_exact_on_representable_products(ctx, method, w, kernel):
    """Inputs whose every bit lies inside the split's fixed-point window (small integers times powers of two
    within a window) make the slice products and their recombination exact: the CRT form's dropped low x low
    product is zero and the digit form's dropped pairs are zero, and the exact result fits in w words.  Then
    C must equal the exact product bit for bit (compared as exact rationals), for both slice-GEMM kernels,
    including tiles whose pairs are split over several CTAs (one small product) and ragged shapes."""
    import torch
    import paper_2402_11868_gb300 as Z
    Z.zkq_set_gemm_kernel(kernel)
    ibits, espread = (19, 20) if w == 4 else (9, 10)
    rng = np.random.default_rng(77 + 10 * w + method + 100 * kernel)
    cases = [(1, 1, 1, 0), (5, 9, 13, 1), (128, 64, 96, 0), (33, 130, 70, 1), (200, 17, 512, 0)]
    As, Bs = [], []
    for (m, n, k, op) in cases:
        As.append(dyadic_mw(rng, m * k, w, ibits, espread)); Bs.append(dyadic_mw(rng, k * n, w, ibits, espread))
    a_off = np.cumsum([0] + [a.shape[0] for a in As[:-1]]); b_off = np.cumsum([0] + [b.shape[0] for b in Bs[:-1]])
    c_sz = [m * n for (m, n, _, _) in cases]; c_off = np.cumsum([0] + c_sz[:-1])
    dA = torch.from_numpy(np.concatenate([a.reshape(-1) for a in As])).cuda()
    dB = torch.from_numpy(np.concatenate([b.reshape(-1) for b in Bs])).cuda()
    dC = torch.full((sum(c_sz) * 2 * w,), np.nan, dtype=torch.float64, device="cuda")
    try:
        Z.zkq_mw_gemm(ctx, [c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases],
                      dA, a_off, w, dB, b_off, w, dC, c_off, w, 53 * w + 6, method)
        torch.cuda.synchronize()
        Z.zkq_check_device_waits()
    finally:
        Z.zkq_set_gemm_kernel(1)
    Ch = dC.cpu().numpy()
    for i, (m, n, k, op) in enumerate(cases):
        ref = oracle.matmul(As[i], Bs[i], m, n, k, opA=op)
        got = Ch[2 * w * c_off[i]: 2 * w * (c_off[i] + m * n)].reshape(m * n, 2, w)
        for e in range(m * n):
            for part in range(2):
                assert fr(got[e, part]) == fr(ref[e, part]), (i, e, part)


def oracle_eig(cache, key, p):
    if key not in cache:
        cache[key] = oracle.eigh(p.A, p.n)
    return cache[key]


@pytest.fixture(scope="module")
def cache():
    return {}


def check_refined(res, probs, target, bits, cache, tag):
    for b, p in enumerate(probs):
        lam, V = _gpu.problem_views(res, b, target)
        L, _, _ = oracle_eig(cache, (tag, b), p)
        anorm = abs(fr(L[0]))
        worst = max(abs(fr(lam[i]) - fr(L[i])) for i in range(p.n))
        assert worst <= anorm / 2**bits, (p.n, float(worst / anorm))
        r, o = oracle.residual(p.A, p.n, lam, V)
        assert r.max() <= float(anorm) * 2.0**-bits, (p.n, r.max())


@pytest.mark.parametrize("method", [1, 2])
def test_oa_refine_double_double_graded_with_pairs(ctx, cache, method):
    sizes = [2, 16, 24, 40, 66]
    probs = []
    for i, n in enumerate(sizes):
        lam, lo, pairs, w = W.batch_problem_spec(1, 5, i, n)
        probs.append(W.herm_spectrum(5, i, lam, w, lam_lo=lo, pairs=pairs))
    res = _gpu.refine_batch(ctx, probs, 2, 2, method)
    assert (res["rinfo"].cpu().numpy() == 0).all(), res["rinfo"]
    check_refined(res, probs, 2, 100, cache, "dd5")


@pytest.mark.parametrize("method", [1, 2])
def test_oa_refine_quad_double_graded_2m180_with_pairs(ctx, cache, method):
    sizes = [3, 16, 32, 48, 96]
    probs = []
    for i, n in enumerate(sizes):
        lam, lo, pairs, w = W.batch_problem_spec(2, 6, i, n)
        probs.append(W.herm_spectrum(6, i, lam, w, lam_lo=lo, pairs=pairs))
    res = _gpu.refine_batch(ctx, probs, 4, 4, method)
    assert (res["rinfo"].cpu().numpy() == 0).all(), res["rinfo"]
    check_refined(res, probs, 4, 200, cache, "qd6")


def test_oa_refine_quad_double_single128_spectrum(ctx, cache):
    import paper_2402_11868_gb300 as Z
    probs = [W.herm_spectrum(8, 0, W.spectrum_single128(64), 4), W.herm_spectrum(8, 1, W.spectrum_single128(17), 4)]
    res = _gpu.refine_batch(ctx, probs, 4, 4, Z.ZKQ_OA_OZAKI)
    assert (res["rinfo"].cpu().numpy() == 0).all(), res["rinfo"]
    check_refined(res, probs, 4, 200, cache, "s8")
