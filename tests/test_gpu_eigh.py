"""GPU parity of the FP64 Jacobi stage, the device multi-word arithmetic and plain RQI refinement
against the 320-bit oracle, on seeded problems (sizes span several tiles, odd and ragged orders)."""
from __future__ import annotations

from fractions import Fraction

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


@pytest.fixture(scope="module")
def oracle_cache():
    return {}


def oracle_solution(cache, key, p):
    if key not in cache:
        cache[key] = oracle.eigh(p.A, p.n)
    return cache[key]


def small_problems(seed, sizes, grade=40, w=4):
    return [W.herm_spectrum(seed, i, W.spectrum_graded(n, grade), w) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("words", [2, 4])
@pytest.mark.parametrize("op", [0, 1, 2, 3, 4, 5, 6])
def test_device_multiword_ops_within_bounds(ctx, words, op):
    import torch
    import paper_2402_11868_gb300 as Z
    from tests.test_abi_cpu import BOUND, random_mw
    rng = np.random.default_rng(7 * words + op)
    count = 300
    cplx = op >= 5
    shape = (count, 2, words) if cplx else (count, words)
    a = random_mw(rng, count * (2 if cplx else 1), words).reshape(shape)
    b = random_mw(rng, count * (2 if cplx else 1), words).reshape(shape)
    if op == 4:
        a = np.abs(a[..., :1]) * np.ones_like(a) * 0 + a * np.sign(a[..., :1])
    da = torch.from_numpy(a).cuda(); db = torch.from_numpy(b).cuda(); do = torch.zeros_like(da)
    Z.zkq_mw_op(op, words, count, da, db, do, on_device=True)
    out = do.cpu().numpy()
    name = {0: "add", 1: "sub", 2: "mul", 3: "div", 4: "sqrt"}
    for i in range(count):
        if not cplx:
            ref = fr(oracle.scalar(name[op], a[i], b[i]))
            scale = max(abs(ref), abs(fr(a[i])) * 2.0**-(53 * words - 10)) if op < 2 else abs(ref)
            assert abs(fr(out[i]) - ref) <= BOUND[words][op] * scale, (op, i)
        else:
            ar, ai, br, bi = fr(a[i, 0]), fr(a[i, 1]), fr(b[i, 0]), fr(b[i, 1])
            if op == 5:
                rr, ri = ar * br - ai * bi, ar * bi + ai * br
                scale = (ar * ar + ai * ai) * (br * br + bi * bi)
            else:
                d = br * br + bi * bi
                rr, ri = (ar * br + ai * bi) / d, (ai * br - ar * bi) / d
                scale = (ar * ar + ai * ai) / d
            tol = (2.0**-100 if words == 2 else 2.0**-203) * float(scale) ** 0.5
            assert abs(float(fr(out[i, 0]) - rr)) <= tol and abs(float(fr(out[i, 1]) - ri)) <= tol, (op, i)


SIZES = [1, 2, 3, 5, 16, 17, 33, 64, 80, 81, 96, 130]


def test_jacobi_fp64_matches_oracle(ctx, oracle_cache):
    probs = small_problems(21, SIZES)
    res = _gpu.eigh_batch(ctx, probs, 4)
    info = res["info"].cpu().numpy()
    assert (info == 0).all(), info
    for b, p in enumerate(probs):
        lam, V = _gpu.problem_views(res, b)
        L, _, _ = oracle_solution(oracle_cache, ("s21", b), p)
        anorm = abs(float(fr(L[0])))
        tol = 8 * p.n * 2.0**-53 * anorm + 1e-300
        for i in range(p.n):
            assert abs(lam[i, 0] - float(fr(L[i]))) <= tol, (p.n, i)
        res_, orth = oracle.residual(p.A, p.n, lam, V)
        assert res_.max() <= tol and orth.max() <= 8 * p.n * 2.0**-53, (p.n, res_.max(), orth.max())
        # eigenvector phase convention: first largest-modulus component real positive
        Vc = V[:, 0, 0] + 1j * V[:, 1, 0]
        Vc = Vc.reshape(p.n, p.n, order="F")
        for c in range(p.n):
            k = int(np.argmax(np.abs(Vc[:, c])))
            assert Vc[k, c].imag == 0 and Vc[k, c].real > 0


def test_jacobi_large_order_keeps_its_scales_in_range(ctx):
    """Order 1500 (one problem, cooperative-grid class): the fast rotations' scales shrink by c >= 2^-1/2
    per rotation and a sweep has 1499 rotations per index, so they are folded back every 256 rounds.  The
    FP64 eigenvalues match LAPACK's within 8 n 2^-53 ||A|| and V is orthonormal to the same level."""
    import torch
    import paper_2402_11868_gb300 as Z
    n = 1500
    rng = np.random.default_rng(15)
    Zm = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = (Zm + Zm.conj().T) / 2
    ref = np.linalg.eigvalsh(A)[::-1]
    words = np.zeros((n * n, 2, 1))
    Af = A.reshape(-1, order="F")
    words[:, 0, 0], words[:, 1, 0] = Af.real, Af.imag
    class P:
        def __init__(self, n, A): self.n, self.A = n, A
    res = _gpu.eigh_batch(ctx, [P(n, words)], 1)
    assert int(res["info"].cpu().numpy()[0]) == 0
    lam, V = _gpu.problem_views(res, 0)
    anorm = np.abs(ref).max()
    assert np.all(np.isfinite(lam)) and np.abs(lam[:, 0] - ref).max() <= 8 * n * 2.0**-53 * anorm
    Vc = (V[:, 0, 0] + 1j * V[:, 1, 0]).reshape(n, n, order="F")
    assert np.abs(Vc.conj().T @ Vc - np.eye(n)).max() <= 8 * n * 2.0**-53
    assert np.abs(A @ Vc - Vc * lam[:, 0]).max() <= 8 * n * 2.0**-53 * anorm


def test_jacobi_degenerate_and_trivial_inputs(ctx):
    import torch
    import paper_2402_11868_gb300 as Z
    # zero matrix, identity, diagonal with repeated entries, 1x1
    mats, ns = [], [4, 5, 3, 1]
    Z0 = np.zeros((16, 2, 1))
    I5 = np.zeros((25, 2, 1)); I5[[0, 6, 12, 18, 24], 0, 0] = 1.0
    D3 = np.zeros((9, 2, 1)); D3[0, 0, 0] = 2.0; D3[4, 0, 0] = 2.0; D3[8, 0, 0] = -1.0
    S1 = np.array([[[-3.5]], [[0.0]]]).reshape(1, 2, 1)
    class P:  # minimal problem record
        def __init__(self, n, A): self.n, self.A = n, A
    res = _gpu.eigh_batch(ctx, [P(4, Z0), P(5, I5), P(3, D3), P(1, S1)], 1)
    assert (res["info"].cpu().numpy() == 0).all()
    Wv = res["W"].cpu().numpy()
    assert list(Wv[:4]) == [0, 0, 0, 0]
    assert list(Wv[4:9]) == [1, 1, 1, 1, 1]
    assert list(Wv[9:12]) == [2, 2, -1]
    assert Wv[12] == -3.5


@pytest.mark.parametrize("target", [2, 4])
def test_plain_rqi_matches_oracle_small(ctx, oracle_cache, target):
    import paper_2402_11868_gb300 as Z
    sizes = [2, 3, 16, 17, 40]
    probs = [W.herm_spectrum(31, i, W.spectrum_single128(n), 4) for i, n in enumerate(sizes)]
    res = _gpu.refine_batch(ctx, probs, 4, target, Z.ZKQ_PLAIN_RQI)
    assert (res["rinfo"].cpu().numpy() == 0).all(), res["rinfo"]
    bound_bits = 200 if target == 4 else 100
    for b, p in enumerate(probs):
        lam, V = _gpu.problem_views(res, b, target)
        L, _, _ = oracle_solution(oracle_cache, ("r31", b), p)
        anorm = abs(fr(L[0]))
        for i in range(p.n):
            assert abs(fr(lam[i]) - fr(L[i])) <= anorm / 2**bound_bits, (p.n, i)
        r, o = oracle.residual(p.A, p.n, lam, V)
        assert r.max() <= float(anorm) * 2.0**-bound_bits, (p.n, r.max())
        # eigenvectors come from independent inverse iterations: their mutual orthogonality is limited by
        # residual / gap (Davis-Kahan), not by the working precision
        vals = [float(fr(L[i])) for i in range(p.n)]
        gap = min([abs(vals[i] - vals[j]) for i in range(p.n) for j in range(p.n) if i != j] or [1.0])
        assert o.max() <= 4 * float(anorm) * 2.0**-bound_bits / gap + 2.0**-bound_bits, (p.n, o.max())
