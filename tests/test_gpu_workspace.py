"""zkq_workspace_size against the workspace a fresh context actually holds afterwards
(zkq_ctx_workspace_bytes).  The figure is exact for the FP64 eigensolve, plain RQI and the refinement with
FP64-pipe products; with split products it is an upper bound that the held bytes reach within the
scratch's growth slack (a quarter).  The spectra are graded gently enough that no eigenvalue falls within
the refinement's cluster threshold, so no cluster step adds products beyond those the figure covers."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from tests import _gpu

pytestmark = pytest.mark.gpu

WIDE = [12, 40, 81, 100, 130, 200]
NARROW = [12, 40, 81, 100]


def problems(sizes, grade, w):
    return [W.herm_spectrum(43, i, W.spectrum_graded(n, grade), w) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("a_words,target,method,sizes,grade,exact", [
    (4, 0, 0, WIDE, 20, True),        # eigensolve only
    (4, 4, 0, NARROW, 12, True),      # plain RQI
    (4, 4, 2, NARROW, 20, True),      # refinement, FP64-pipe products
    (4, 4, 1, WIDE, 20, False),       # refinement, split products (quad-double)
    (2, 2, 1, WIDE, 20, False),       # refinement, split products (double-double)
])
def test_workspace_size_matches_what_the_context_holds(a_words, target, method, sizes, grade, exact):
    import paper_2402_11868_gb300 as Z
    Z.build()
    probs = problems(sizes, grade, a_words)
    with Z.Context(0) as ctx:
        assert ctx.workspace_bytes() == 0
        want = Z.zkq_workspace_size(ctx, sizes, a_words, target, method)
        assert ctx.workspace_bytes() == 0                    # the query allocates nothing
        eig = _gpu.eigh_batch(ctx, probs, a_words)
        assert (eig["info"].cpu().numpy() == 0).all()
        if target:
            res = _gpu.refine_batch(ctx, probs, a_words, target, method, eig=eig)
            if method != 0:
                assert (res["rinfo"].cpu().numpy() == 0).all()
                assert float(res["err"].max()) <= 2.0 ** -(53 * target - 12)
        held = ctx.workspace_bytes()
    if exact:
        assert held == want, (held, want)
    else:
        assert 0.8 * want <= held <= want, (held, want)


def test_workspace_size_grows_with_the_batch():
    import paper_2402_11868_gb300 as Z
    Z.build()
    with Z.Context(0) as ctx:
        one = Z.zkq_workspace_size(ctx, [300], 4, 4, Z.ZKQ_OA_OZAKI)
        two = Z.zkq_workspace_size(ctx, [300, 300], 4, 4, Z.ZKQ_OA_OZAKI)
        mixed = Z.zkq_workspace_size(ctx, [300, 700], 4, 4, Z.ZKQ_OA_OZAKI)
        big = Z.zkq_workspace_size(ctx, [700], 4, 4, Z.ZKQ_OA_OZAKI)
        assert one < two < 2 * one + (4 << 20)
        assert mixed >= big and mixed > one
        assert Z.zkq_workspace_size(ctx, [], 4, 4, Z.ZKQ_OA_OZAKI) == 0
        with pytest.raises(Z.ZkqError):
            Z.zkq_workspace_size(ctx, [4096], 4, 4, Z.ZKQ_OA_OZAKI)      # refinement orders stop at 2048
        assert Z.zkq_workspace_size(ctx, [4096], 4, 0) > 32 * 4096 ** 2
        assert ctx.workspace_bytes() == 0
