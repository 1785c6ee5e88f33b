"""The library's maximum sizes (include/adsx.h): K = ADSX_MAX_K, nprobe =
ADSX_MAX_NPROBE, D = ADSX_MAX_D, a large query batch; and the first values
beyond them are rejected."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09855_gb300 import workloads as W
from gpu_helpers import kth_near_tie, near_tie_queries, topk_row_mismatch

pytestmark = pytest.mark.gpu

MAX_K, MAX_NPROBE, MAX_D = 1024, 1024, 4080


@pytest.fixture(scope="module")
def lib():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    return adsx


def _exact_rows(ids, d2, eids, ed2, Cr, Qr, nprobe, K):
    skip = near_tie_queries(Cr, Qr, nprobe) | kth_near_tie(ed2, K)
    bad = [q for q in range(ids.shape[0])
           if not skip[q] and topk_row_mismatch(ids[q], d2[q], eids[q, :K], ed2[q, :K])]
    return bad, int((~skip).sum())


def test_max_K_and_max_nprobe(lib):
    wl = W.random_small(24_000, 32, 12, 1024, seed=41, kmeans_iters=3)
    ix = lib.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    try:
        Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
        for K, nprobe in ((MAX_K, 64), (10, MAX_NPROBE), (MAX_K, MAX_NPROBE)):
            ids, d2 = ix.search(wl.Q, K, nprobe, eps0=math.inf)
            eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K + 1, nprobe)
            bad, n = _exact_rows(ids, d2, eids, ed2, Cr, Qr, nprobe, K)
            assert not bad and n >= 6, (K, nprobe, bad)
            a_ids, a_d2 = ix.search(wl.Q, K, nprobe, eps0=2.1, delta_d=16)
            for q in range(Qr.shape[0]):
                for i, d in zip(a_ids[q], a_d2[q]):
                    if i >= 0:
                        ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                        assert abs(d - ex) <= 1e-5 * ex + 1e-6
        with pytest.raises(lib.AdsxError):
            ix.search(wl.Q, MAX_K + 1, 8)
        with pytest.raises(lib.AdsxError):
            ix.search(wl.Q, 10, MAX_NPROBE + 1)
    finally:
        ix.close()


def test_max_dimension(lib):
    D, N = MAX_D, 300
    rng = np.random.default_rng(43)
    centres = rng.normal(0, 1.0, size=(6, D))
    X = (centres[rng.integers(0, 6, size=N)] + 0.5 * rng.standard_normal((N, D))).astype(np.float32)
    Q = (centres[rng.integers(0, 6, size=5)] + 0.5 * rng.standard_normal((5, D))).astype(np.float32)
    P = W.make_P(D, 44).astype(np.float32)
    C = centres.astype(np.float32)
    assign = np.argmin(((X[:, None, :] - C[None]) ** 2).sum(-1), 1).astype(np.int32)
    ix = lib.build_index(X, P, C, assign)
    try:
        Y, Cr, Qr = (oracle.rotate(P, a) for a in (X, C, Q))
        ids, d2 = ix.search(Q, 20, 3, eps0=math.inf)
        eids, ed2 = oracle.ivf_exact(Y, Cr, assign, Qr, 21, 3)
        bad, n = _exact_rows(ids, d2, eids, ed2, Cr, Qr, 3, 20)
        assert not bad and n >= 3
        rot = ix.rotate(Q)
        assert np.max(np.abs(rot - Qr) / np.linalg.norm(Qr, axis=1, keepdims=True)) < 1e-5
        a_ids, a_d2 = ix.search(Q, 20, 3, eps0=2.1, delta_d=64)
        for q in range(5):
            for i, d in zip(a_ids[q], a_d2[q]):
                if i >= 0:
                    ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                    assert abs(d - ex) <= 1e-5 * ex
    finally:
        ix.close()
    with pytest.raises(lib.AdsxError):
        Pb = np.eye(MAX_D + 1, dtype=np.float32)
        lib.build_index(np.zeros((4, MAX_D + 1), np.float32), Pb,
                        np.zeros((1, MAX_D + 1), np.float32), np.zeros(4, np.int32))


def test_large_query_batch(lib):
    wl = W.gen_gaussian_mixture()
    ix = lib.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    try:
        big = np.tile(wl.Q, (1000, 1))                       # 100k queries in one call
        ids, d2 = ix.search(big, 10, 10, eps0=math.inf)
        ref_ids, ref_d2 = ix.search(wl.Q, 10, 10, eps0=math.inf)
        assert np.array_equal(ids[:100], ref_ids) and np.array_equal(ids[-100:], ref_ids)
        assert np.array_equal(d2[50_000:50_100], ref_d2)
    finally:
        ix.close()
