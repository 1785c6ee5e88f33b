"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

import oracle

REL = 1e-5


def near_tie_queries(Cr, Qr, nprobe):
    """Queries whose nprobe-th and (nprobe+1)-th centroid distances are within
    REL in FP64 (their probe sets are not determined at FP32 precision)."""
    if nprobe >= Cr.shape[0]:
        return np.zeros(Qr.shape[0], bool)
    _, pd = oracle.probe(Cr, Qr, nprobe + 1)
    a, b = pd[:, nprobe - 1], pd[:, nprobe]
    with np.errstate(invalid="ignore"):
        return (b - a) <= REL * np.maximum(b, 1e-30)


def kth_near_tie(d2, K):
    if d2.shape[1] <= K:
        return np.zeros(d2.shape[0], bool)
    a, b = d2[:, K - 1], d2[:, K]
    with np.errstate(invalid="ignore"):
        return (b - a) <= REL * np.maximum(b, 1e-30)


def topk_row_mismatch(ids, d2, eids, ed2):
    """True when one query's GPU top-K differs from the oracle's beyond FP32
    order: id sets equal (padding aside), order equal except between oracle
    distances within REL, distances within REL."""
    v = eids >= 0
    if not np.array_equal(ids[~v], eids[~v]) or set(ids[v]) != set(eids[v]):
        return True
    e = ed2[v]
    tie = np.zeros(e.shape[0], bool)
    close = np.abs(np.diff(e)) <= REL * np.maximum(e[1:], 1e-30)
    tie[1:] |= close
    tie[:-1] |= close
    if np.any((ids[v] != eids[v]) & ~tie):
        return True
    return bool(np.any(np.abs(d2[v] - e) > REL * np.maximum(e, 1e-30)))
