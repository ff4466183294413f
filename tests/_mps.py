"""Host-side helpers for the MPS parity tests: Vidal MPS arrays in the layout of zkq_mps_upload /
oracle.mps_amplitudes (Gamma (s, alpha, beta) row-major, concatenated; lambda per bond, concatenated), built
exactly from local vectors or rescaled exactly by powers of two, and per-site views for the canonical checks."""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import oracle
import workloads as W


def dims_of(n, chi):
    return [1] + [int(c) for c in chi] + [1]


def product_state(local, w):
    """Vidal MPS of the product state (x)_l local[l], local[l] = ((re0, im0), (re1, im1)) Fractions, unit norm
    assumed: chi = 1, Gamma[l]^s = local[l][s], lambda = 1."""
    n = len(local)
    g = np.zeros((2 * n, 2, w))
    for l in range(n):
        for s in range(2):
            g[2 * l + s, 0, :] = W.words_of(Fraction(local[l][s][0]), w)
            g[2 * l + s, 1, :] = W.words_of(Fraction(local[l][s][1]), w)
    lam = np.zeros((n - 1, w)); lam[:, 0] = 1.0
    return np.ones(n - 1, dtype=np.int32), g, lam


def scale_norm(n, chi, g, lam, log2_norm):
    """Normalise a Vidal MPS whose squared norm is 2^(2 log2_norm) (canonical inside, with the norm carried by
    the weights): weights / 2^log2_norm, interior Gammas * 2^log2_norm.  Exact (powers of two)."""
    dims = dims_of(n, chi)
    g = g.copy(); lam = lam * 2.0 ** -log2_norm
    go = 0
    for l in range(n):
        e = 2 * dims[l] * dims[l + 1]
        if 0 < l < n - 1:
            g[go:go + e] *= 2.0 ** log2_norm
        go += e
    return g, lam


def site_views(n, chi, g, lam):
    """(a, b, Gamma words, left weights, right weights) of every site."""
    dims = dims_of(n, chi)
    out, go, lo = [], 0, 0
    for l in range(n):
        a, b = dims[l], dims[l + 1]
        left = lam[lo - a:lo] if l > 0 else None
        right = lam[lo:lo + b] if l < n - 1 else None
        out.append((a, b, g[go:go + 2 * a * b], left, right))
        go += 2 * a * b
        if l < n - 1:
            lo += b
    return out


def canonical_defect(n, chi, g, lam, w):
    """max over sites and both sides of the Vidal canonical defect (0 for an exact normalised canonical MPS)."""
    worst = 0.0
    for l, (a, b, gl, left, right) in enumerate(site_views(n, chi, g, lam)):
        worst = max(worst, oracle.mps_site_defect(a, b, gl, left, None, w, 0),
                    oracle.mps_site_defect(a, b, gl, None, right, w, 1))
    return worst


def bond_weights(chi, lam):
    """lambda words of each bond, as a list of (chi_l, w) arrays."""
    out, lo = [], 0
    for c in chi:
        out.append(lam[lo:lo + int(c)])
        lo += int(c)
    return out
