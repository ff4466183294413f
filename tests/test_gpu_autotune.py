"""Autotuning of the Jacobi cluster width (zkq_autotune_jacobi): the chosen widths are valid, the context
uses them, and the eigensolve's results do not depend on them (the same bits as with the built-in
choice)."""
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
