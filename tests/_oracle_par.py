"""Threaded calls of the 320-bit oracle for the full-size parity tests (the oracle's C routines release the
GIL, so threads run them in parallel), with oracle eigenvalues cached on disk under the git-ignored build
folder, keyed by a hash of the exact input words."""
from __future__ import annotations

import hashlib
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle

_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "oracle_cache")


def threads() -> int:
    return max(1, os.cpu_count() or 1)


def residual_all_columns(A, n, lam, V, chunk=8):
    """(residual, orthonormality defect) of every column at 320 bits, columns split over threads."""
    cols = list(range(n))
    parts = [cols[i:i + chunk] for i in range(0, n, chunk)]
    with ThreadPoolExecutor(max_workers=threads()) as ex:
        out = list(ex.map(lambda c: oracle.residual(A, n, lam, V, cols=c), parts))
    return np.concatenate([r for r, _ in out]), np.concatenate([o for _, o in out])


def _key(A) -> str:
    return hashlib.sha256(np.ascontiguousarray(A, dtype=np.float64).tobytes()).hexdigest()[:32]


def eig_values(problems):
    """Oracle eigenvalues (n, 6 words) of each problem, in parallel over problems (largest first), cached."""
    os.makedirs(_CACHE, exist_ok=True)
    out = [None] * len(problems)
    todo = []
    for i, p in enumerate(problems):
        f = os.path.join(_CACHE, f"eig_{p.n}_{_key(p.A)}.npy")
        if os.path.exists(f):
            out[i] = np.load(f)
        else:
            todo.append((i, f))

    def one(item):
        i, f = item
        L, _, _ = oracle.eigh(problems[i].A, problems[i].n)
        tmp = f + f".{os.getpid()}.{i}.tmp.npy"
        np.save(tmp, L)
        os.replace(tmp, f)
        return i, L

    todo.sort(key=lambda it: -problems[it[0]].n)
    with ThreadPoolExecutor(max_workers=threads()) as ex:
        for i, L in ex.map(one, todo):
            out[i] = L
    return out
