"""Partition-agreement metrics (host side, evaluation only).

NMI with the arithmetic-mean normalisation I(U;V) / ((H(U)+H(V))/2), and the
Hubert-Arabie adjusted Rand index, both from an exact int64 contingency table.
These evaluate a partition; they are not part of the partitioning path.
"""
from __future__ import annotations

import numpy as np


def _contingency(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    if a.shape != b.shape:
        raise ValueError("label arrays differ in length")
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    na = int(ai.max()) + 1 if ai.size else 0
    nb = int(bi.max()) + 1 if bi.size else 0
    table = np.bincount(ai.astype(np.int64) * nb + bi, minlength=na * nb).reshape(na, nb)
    return table


def nmi(a, b) -> float:
    t = _contingency(a, b).astype(np.float64)
    n = t.sum()
    if n == 0:
        return 1.0
    pa = t.sum(axis=1) / n
    pb = t.sum(axis=0) / n
    ha = -np.sum(pa[pa > 0] * np.log(pa[pa > 0]))
    hb = -np.sum(pb[pb > 0] * np.log(pb[pb > 0]))
    if ha == 0.0 and hb == 0.0:
        return 1.0
    nz = t > 0
    pij = t[nz] / n
    mi = np.sum(pij * (np.log(pij) - np.log(np.outer(pa, pb)[nz])))
    mi = max(mi, 0.0)
    return float(mi / (0.5 * (ha + hb)))


def ari(a, b) -> float:
    t = _contingency(a, b).astype(np.int64)
    n = int(t.sum())

    def c2(x):
        x = np.asarray(x, dtype=np.float64)
        return x * (x - 1) / 2.0

    sum_ij = c2(t).sum()
    sum_a = c2(t.sum(axis=1)).sum()
    sum_b = c2(t.sum(axis=0)).sum()
    total = n * (n - 1) / 2.0
    if total == 0:
        return 1.0
    expected = sum_a * sum_b / total
    max_idx = 0.5 * (sum_a + sum_b)
    if max_idx == expected:
        return 1.0
    return float((sum_ij - expected) / (max_idx - expected))
