"""Kac-walk rotation (Sec. 6.2.3: the random rotation in O(D log D)) through
the C ABI, against the FP64 oracle applying the same walk:
  - the rotated queries (adsx_rotate) within 1e-5 of ||q||, also for odd D;
  - eps0 = inf: ids equal the oracle's exact IVF on the walk-rotated data
    except near-ties, distances within 1e-5 relative;
  - eps0 = 2.1: every returned distance exact, the bracket invariant, recall
    no worse than the sequential oracle's minus 0.01;
  - malformed walks (an index repeated in a layer, c^2 + s^2 != 1) are
    rejected.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import REL, kth_near_tie, near_tie_queries, topk_row_mismatch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kac():
    from paper_2303_09855_gb300 import adsx, build
    from paper_2303_09855_gb300 import workloads as W
    build.build()
    wl = W.gen_gaussian_mixture()
    pairs, cs = W.make_kac_walk(wl.D, 14, 91)           # 2 log2(128) layers
    ix = adsx.build_index_kac(wl.X, pairs, cs, wl.centroids, wl.assign)
    Y = oracle.kac_apply(pairs, cs, wl.X)
    Cr = oracle.kac_apply(pairs, cs, wl.centroids)
    Qr = oracle.kac_apply(pairs, cs, wl.Q)
    yield adsx, W, wl, ix, Y, Cr, Qr
    ix.close()


def test_kac_rotation_matches_oracle(kac):
    adsx, W, wl, ix, Y, Cr, Qr = kac
    rot = ix.rotate(wl.Q)
    scale = np.linalg.norm(Qr, axis=1, keepdims=True)
    assert np.max(np.abs(rot - Qr) / scale) < 1e-5
    # odd D: one coordinate rests in every layer
    rng = np.random.default_rng(92)
    D = 37
    X = rng.normal(size=(500, D)).astype(np.float32)
    C = X[:4].copy()
    assign = rng.integers(0, 4, 500).astype(np.int32)
    pairs, cs = W.make_kac_walk(D, 12, 93)
    ix2 = adsx.build_index_kac(X, pairs, cs, C, assign)
    try:
        Q = rng.normal(size=(9, D)).astype(np.float32)
        ex = oracle.kac_apply(pairs, cs, Q)
        got = ix2.rotate(Q)
        assert np.max(np.abs(got - ex) / np.linalg.norm(ex, axis=1, keepdims=True)) < 1e-5
    finally:
        ix2.close()


def test_kac_exact_mode_and_adsampling(kac):
    adsx, W, wl, ix, Y, Cr, Qr = kac
    K, nprobe = 10, 10
    ids, d2 = ix.search(wl.Q, K, nprobe, eps0=math.inf)
    eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K + 1, nprobe)
    skip = near_tie_queries(Cr, Qr, nprobe) | kth_near_tie(ed2, K)
    bad = [q for q in range(wl.Q.shape[0])
           if not skip[q] and topk_row_mismatch(ids[q], d2[q], eids[q, :K], ed2[q, :K])]
    assert not bad and (~skip).sum() >= 90, bad
    eps0, dd = 2.1, 32
    a_ids, a_d2 = ix.search(wl.Q, K, nprobe, eps0=eps0, delta_d=dd)
    oids, _, _, _ = oracle.ivf_ads(Y, Cr, wl.assign, Qr, K, nprobe, eps0, dd)
    for q in range(wl.Q.shape[0]):
        for i, d in zip(a_ids[q], a_d2[q]):
            if i >= 0:
                ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                assert abs(d - ex) <= REL * ex + 1e-6, (q, i, d, ex)
        if skip[q]:
            continue
        top = eids[q, :K]
        dec, _, mar = oracle.dco_fixed_r(Y[top], Qr[q:q + 1], np.array([ed2[q, K - 1]]), eps0, dd)
        must = set(top[(dec[0] == oracle.POSITIVE) & (mar[0] >= REL)].tolist())
        assert must <= set(a_ids[q].tolist()), q
    assert oracle.recall_at(a_ids, eids[:, :K], K) >= oracle.recall_at(oids, eids[:, :K], K) - 0.01


def test_kac_malformed_walks_rejected(kac):
    adsx, W, wl, ix, Y, Cr, Qr = kac
    pairs, cs = W.make_kac_walk(wl.D, 4, 94)
    bad = pairs.copy()
    bad[2, 5] = bad[2, 6]                               # repeated index in one layer
    with pytest.raises(adsx.AdsxError):
        adsx.build_index_kac(wl.X, bad, cs, wl.centroids, wl.assign)
    bad_cs = cs.copy()
    bad_cs[1, 0], bad_cs[1, 1] = 1.0, 0.5              # c^2 + s^2 = 1.25
    with pytest.raises(adsx.AdsxError):
        adsx.build_index_kac(wl.X, pairs, bad_cs, wl.centroids, wl.assign)
    oob = pairs.copy()
    oob[0, 0] = wl.D                                    # out of range
    with pytest.raises(adsx.AdsxError):
        adsx.build_index_kac(wl.X, oob, cs, wl.centroids, wl.assign)
