"""Autotuning of the Jacobi cluster width (zkq_autotune_jacobi) and of the split-product GEMM tile width
(zkq_autotune_gemm): the chosen widths are valid, the library uses them, and no result depends on them (the
same bits as with the built-in choice)."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_autotuned_width_is_valid_and_results_do_not_change():
    import paper_2402_11868_gb300 as Z
    Z.build()
    probs = [W.herm_spectrum(41, i, W.spectrum_graded(n, 40), 4) for i, n in enumerate([96, 160, 96, 160] * 20)]
    plain = Z.Context(0)
    try:
        ref = _gpu.eigh_batch(plain, probs, 4)
    finally:
        plain.close()
    tuned = Z.Context(0)
    try:
        best = tuned.autotune_jacobi([96, 160], a_words=4, reps=1)
        assert len(best) == 2 and all(b in (2, 4, 8, 16) for b in best), best
        got = _gpu.eigh_batch(tuned, probs, 4)
        assert (got["info"].cpu().numpy() == 0).all()
        assert np.array_equal(got["W"].cpu().numpy(), ref["W"].cpu().numpy())
        assert np.array_equal(got["V"].cpu().numpy(), ref["V"].cpu().numpy())
    finally:
        tuned.close()


def _products(Z, torch, ctx, n, count, seed, words=4):
    """count n x n x n complex products C_i = A_i B_i (words per real) by the split products; returns C."""
    rng = np.random.default_rng(seed)
    el = n * n
    A = torch.from_numpy(rng.standard_normal(count * el * 2 * words) * (0.5 ** np.tile(np.arange(words) * 53, count * el * 2))).cuda()
    B = torch.from_numpy(rng.standard_normal(count * el * 2 * words) * (0.5 ** np.tile(np.arange(words) * 53, count * el * 2))).cuda()
    C = torch.zeros(count * el * 2 * words, dtype=torch.float64, device="cuda")
    offs = [i * el for i in range(count)]
    Z.zkq_mw_gemm(ctx, [n] * count, [n] * count, [n] * count, [0] * count, A, offs, words, B, offs, words, C, offs,
                  words, 53 * words + 6, 1)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def test_gemm_tile_width_autotune_is_valid_and_results_do_not_change():
    """zkq_autotune_gemm picks 256- or 128-column tiles per order; every width gives the same bits (the slice
    products are exact integers either way), forced widths and the tuned table alike."""
    import torch
    import paper_2402_11868_gb300 as Z
    Z.build()
    with Z.Context(0) as ctx:
        try:
            Z.zkq_set_gemm_tile_width(256)
            ref = _products(Z, torch, ctx, 96, 6, 3)
            ref2 = _products(Z, torch, ctx, 200, 3, 4)
            Z.zkq_set_gemm_tile_width(128)
            assert np.array_equal(_products(Z, torch, ctx, 96, 6, 3), ref)
            assert np.array_equal(_products(Z, torch, ctx, 200, 3, 4), ref2)
            best = ctx.autotune_gemm([96, 200], words=4, reps=1)
            assert len(best) == 2 and all(b in (128, 256) for b in best), best
            assert np.array_equal(_products(Z, torch, ctx, 96, 6, 3), ref)
            assert np.array_equal(_products(Z, torch, ctx, 200, 3, 4), ref2)
        finally:
            Z.zkq_set_gemm_tile_width(0)
    with pytest.raises(Z.ZkqError):
        Z.zkq_set_gemm_tile_width(64)
