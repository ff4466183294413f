"""The bounded device waits' expiry path, driven without faulting or hanging the GPU: a test hook makes the
cooperative-grid Jacobi's barrier wait for one arrival that never comes (a generation flag that nothing
advances) with a short poll limit.  The wait must give up, the affected problems must report info = -1,
problems in the same batch that need no barrier must still be right, and the same context must then give
correct results once the hook is off."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_grid_barrier_expiry_reports_failure_and_leaves_the_context_usable():
    import paper_2402_11868_gb300 as Z
    Z.build()
    # two problems above order 80 (few enough for the cooperative-grid class) and one in shared memory
    sizes = [200, 130, 24]
    probs = [W.herm_spectrum(81, i, W.spectrum_graded(n, 40), 2) for i, n in enumerate(sizes)]
    with Z.Context(0) as ctx:
        try:
            Z.zkq_test_grid_barrier_hook(1, 12)
            res = _gpu.eigh_batch(ctx, probs, 2)
        finally:
            Z.zkq_test_grid_barrier_hook(0, 22)
        info = res["info"].cpu().numpy()
        assert list(info[:2]) == [-1, -1], info
        assert info[2] == 0
        lam, V = _gpu.problem_views(res, 2)
        L, _, _ = oracle.eigh(probs[2].A, probs[2].n)
        anorm = abs(float(L[0].sum()))
        assert np.abs(lam[:, 0] - L[:, :2].sum(axis=1)).max() <= 8 * 24 * 2.0**-53 * anorm
        # hook off: the same context diagonalises the same batch correctly
        res = _gpu.eigh_batch(ctx, probs, 2)
        assert (res["info"].cpu().numpy() == 0).all()
        for b, p in enumerate(probs):
            lam, V = _gpu.problem_views(res, b)
            anorm = float(np.abs(lam).max())
            r, o = oracle.residual(p.A, p.n, lam, V, cols=[0, p.n // 2, p.n - 1])
            assert r.max() <= 8 * p.n * 2.0**-53 * anorm and o.max() <= 8 * p.n * 2.0**-53
        Z.zkq_check_device_waits()


def test_grid_barrier_hook_rejects_bad_settings():
    import paper_2402_11868_gb300 as Z
    Z.build()
    for extra, lim in ((2, 12), (-1, 12), (0, 3), (0, 23)):
        with pytest.raises(Z.ZkqError) as ei:
            Z.zkq_test_grid_barrier_hook(extra, lim)
        assert ei.value.status == Z.ZKQ_EINVAL
