"""The SVD variant of the gate update (Section 2, ZKCM_CUS paragraph: singular value decomposition beside the
Hermitian diagonalisation): the FP64 one-sided Jacobi SVD (zkq_svd_batched) against the oracle's 320-bit SVD
(oracle.svd), including matrices with graded rows, where the singular values keep their relative accuracy far
below the 2^-26 sigma_max floor of the Gram route; orthonormal singular vectors and reconstruction; and MPS
gate updates by ZKQ_SVD_OA against the oracle's gate update and the paper's footnote state."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W
from tests._util import fr
from tests import _mps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2402_11868_gb300 as Z
    Z.build()
    c = Z.Context(0)
    yield c
    c.close()


def _matrix(m, n, seed, grade=0.0, rank=None):
    """Complex m x n (column-major words (m n, 2, 2)): Gaussian, rows scaled by 2^(-grade i/(m-1)), optionally of
    lower rank (a product of Gaussian factors, exact in double-double)."""
    z = W.cgauss(seed, 1, m * n).reshape(n, m).T            # [i, j]
    if rank is not None:
        a = W.cgauss(seed, 2, m * rank).reshape(rank, m).T
        b = W.cgauss(seed, 3, rank * n).reshape(n, rank).T
        a = np.round(a * 64) / 64; b = np.round(b * 64) / 64
        z = a @ b                                            # exact: dyadic entries, short sums
    if grade:
        z = z * (2.0 ** (-grade * np.arange(m) / max(m - 1, 1)))[:, None]
    A = np.zeros((m * n, 2, 2))
    A[:, 0, 0] = z.T.reshape(-1).real
    A[:, 1, 0] = z.T.reshape(-1).imag
    return A


def _svd(ctx, mats, shapes):
    import torch
    import paper_2402_11868_gb300 as Z
    a_off, u_off, v_off, s_tot = [], [], [], 0
    ao = uo = vo = 0
    for (m, n) in shapes:
        k = min(m, n)
        a_off.append(ao); u_off.append(uo); v_off.append(vo)
        ao += m * n; uo += m * k; vo += n * k; s_tot += k
    A = torch.from_numpy(Z.pack(mats, 2)).cuda()
    S = torch.full((s_tot,), np.nan, dtype=torch.float64, device="cuda")
    U = torch.full((2 * uo,), np.nan, dtype=torch.float64, device="cuda")
    V = torch.full((2 * vo,), np.nan, dtype=torch.float64, device="cuda")
    info = torch.full((len(shapes),), -7, dtype=torch.int32, device="cuda")
    Z.zkq_svd_batched(ctx, [m for m, _ in shapes], [n for _, n in shapes], a_off, A, 2, S, U, u_off, V, v_off, info)
    torch.cuda.synchronize()
    return S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy(), info.cpu().numpy(), u_off, v_off


def test_svd_matches_the_oracle_on_a_ragged_batch(ctx):
    shapes = [(12, 7), (7, 12), (33, 33), (1, 5), (5, 1), (40, 96), (96, 40), (8, 5)]
    mats = [_matrix(m, n, 200 + i, rank=3 if (m, n) == (8, 5) else None) for i, (m, n) in enumerate(shapes)]
    S, U, V, info, u_off, v_off = _svd(ctx, mats, shapes)
    assert (info == 0).all(), info
    so = 0
    for (m, n), A, uo, vo in zip(shapes, mats, u_off, v_off):
        k = min(m, n)
        sig_ref, _, _ = oracle.svd(A, m, n) if m >= n else oracle.svd(_conj_t(A, m, n), n, m)
        s = S[so:so + k]; so += k
        smax = float(fr(sig_ref[0]))
        for i in range(k):
            assert abs(s[i] - float(fr(sig_ref[i]))) <= 8 * k * 2.0**-53 * smax, ((m, n), i)
        assert np.all(np.diff(s) <= 0)
        Uc = (U[2 * uo:2 * (uo + m * k):2] + 1j * U[2 * uo + 1:2 * (uo + m * k):2]).reshape(k, m).T
        Vc = (V[2 * vo:2 * (vo + n * k):2] + 1j * V[2 * vo + 1:2 * (vo + n * k):2]).reshape(k, n).T
        Ac = (A[:, 0, 0] + A[:, 0, 1] + 1j * (A[:, 1, 0] + A[:, 1, 1])).reshape(n, m).T
        tol = 64 * max(m, n) * 2.0**-53
        assert np.abs(Ac - Uc @ np.diag(s) @ Vc.conj().T).max() <= tol * smax
        keep = s > tol * smax                     # the vectors of (numerically) zero singular values are free
        if (m, n) != (8, 5):
            assert keep.all()
        assert np.abs(Uc[:, keep].conj().T @ Uc[:, keep] - np.eye(int(keep.sum()))).max() <= tol
        assert np.abs(Vc.conj().T @ Vc - np.eye(k)).max() <= tol if m >= n else True
        if (m, n) == (8, 5):
            assert (s[3:] <= tol * smax).all()


def _conj_t(A, m, n):
    """words of A^H (n x m) from words of A (m x n)."""
    out = np.zeros_like(A)
    for i in range(m):
        for j in range(n):
            out[j + i * n, 0] = A[i + j * m, 0]
            out[j + i * n, 1] = -A[i + j * m, 1]
    return out


@pytest.mark.parametrize("shape,grade", [((24, 24), 80.0), ((16, 40), 80.0), ((40, 16), 200.0)])
def test_svd_keeps_relative_accuracy_on_graded_rows(ctx, shape, grade):
    """Rows scaled from 1 down to 2^-grade: every singular value (the smallest below 2^-50 of the largest)
    within 2^-40 of its own size, where the Gram matrix would have lost everything below 2^-26.5 of the
    largest."""
    m, n = shape
    A = _matrix(m, n, 300 + m, grade=grade)
    S, _, _, info, _, _ = _svd(ctx, [A], [shape])
    assert info[0] == 0
    sig_ref, _, _ = oracle.svd(A, m, n) if m >= n else oracle.svd(_conj_t(A, m, n), n, m)
    ref = np.array([float(fr(x)) for x in sig_ref])
    assert ref[-1] < 2.0**-50 * ref[0]            # a spectrum far below the Gram floor
    assert np.all(np.abs(S - ref) <= 2.0**-40 * ref), np.abs(S - ref) / ref


def test_gate_update_by_svd_matches_the_oracle_update(ctx):
    import paper_2402_11868_gb300 as Z
    n = 8
    sv = oracle.Statevector(n)
    for site, G in W.brickwork_circuit(91, n, 6, w=4):
        sv.apply2(site, G)
    chi, g, lam = sv.vidal()
    for site in (3, 1, 5):
        mps = Z.MPS(ctx, n, r_max=16, words=4)
        mps.upload(chi, g[..., :4], lam[..., :4])
        G = W.haar_gate(92, site, w=4)
        nb, disc = mps.apply2q(site, G, trunc_tau=2.0**-200, method=Z.ZKQ_SVD_OA)
        chi_o, g_o, lam_o, _ = oracle.mps_apply2(n, chi, g, lam, oracle.WORDS, site, G, tol_log2=200)
        chi_d, g_d, lam_d = mps.download()
        assert list(chi_d) == list(chi_o)
        for x, y in zip(_mps.bond_weights(chi_d, lam_d)[site], _mps.bond_weights(chi_o, lam_o)[site]):
            assert abs(fr(x) - fr(y)) <= Fraction(1, 2**195)
        ref = oracle.Statevector(n); ref.set(sv.amplitudes()); ref.apply2(site, G)
        amps = oracle.mps_amplitudes(n, chi_d, g_d, lam_d, 4)
        worst = max(abs(fr(amps[x, p]) - fr(ref.amplitudes()[x, p])) for x in range(0, 1 << n, 3) for p in range(2))
        assert worst <= Fraction(1, 2**190)
        mps.close()


def test_footnote_state_by_svd_variant(ctx):
    """The footnote's Schmidt coefficients 1 - 2^-179, 2^-179 at n = 180 through the SVD variant."""
    import paper_2402_11868_gb300 as Z
    from tests.test_gpu_mps_parity import _footnote_vidal, _golden_rows
    n = 180
    ctrl, _ = _golden_rows()[n]
    chi, g, lam = _footnote_vidal(n, ctrl)
    mps = Z.MPS(ctx, n, r_max=4, words=4)
    mps.upload(chi, g[..., :4], lam[..., :4])
    I4 = np.zeros((16, 2, 4))
    for r in range(4):
        I4[r * 4 + r, 0, 0] = 1.0
    nb, _ = mps.apply2q(n - 2, I4, trunc_tau=2.0**-200, method=Z.ZKQ_SVD_OA)
    assert nb == 2
    _, _, lam_d = mps.download()
    eps = Fraction(1, 2 ** (n - 1))
    assert abs(fr(lam_d[-2]) ** 2 - (1 - eps)) <= Fraction(1, 2**200)
    assert abs(fr(lam_d[-1]) ** 2 - eps) <= Fraction(1, 2**200)
    mps.close()
