"""Precision form: vectors stored in BF16 or FP16 in the dim-blocked layout,
partial sums in FP32, and every candidate that reaches d = D and may be
positive recomputed exactly in FP32 from an FP32 row copy.  Checked against
the FP64 oracle on a GIST-shaped slice (D = 960, values in [0, 1]).

Acceptance:
  - returned distances are exact FP32 distances: within 1e-5 relative of the
    oracle's FP64 distance for the same id (the low precision never reaches
    a returned value);
  - eps0 = inf: ids identical to exact IVF (the recheck bound is rigorous);
  - fixed-r decisions agree with the oracle except where the oracle's margin
    is below the storage type's error allowance (BF16 0.1, FP16 0.02
    relative) -- low precision moves reject decisions near the threshold;
  - the bracket invariant with the same allowance, and recall@K no worse
    than the oracle's IVF+ recall minus 0.01.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09855_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5
ALLOW = {1: 0.1, 2: 0.02}


@pytest.fixture(scope="module")
def gist():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    wl = W.gen_gist_like(N=20_000, nq=60, ncomp=40, nlist=64, kmeans_iters=6)
    Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
    idx = {st: adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign, storage=st)
           for st in (adsx.F32, adsx.BF16, adsx.F16)}
    yield adsx, wl, idx, Y, Cr, Qr
    for ix in idx.values():
        ix.close()


def _exact_dists_ok(ids, d2, Y, Qr):
    for q in range(ids.shape[0]):
        for i, d in zip(ids[q], d2[q]):
            if i >= 0:
                ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                assert abs(d - ex) <= REL * ex + 1e-6, (q, i, d, ex)


@pytest.mark.parametrize("st", [1, 2])
def test_low_precision_fd_is_exact_ivf(gist, st):
    adsx, wl, idx, Y, Cr, Qr = gist
    K, nprobe = 10, 8
    ids, d2 = idx[st].search(wl.Q, K, nprobe, eps0=math.inf)
    eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K + 1, nprobe)
    f_ids, f_d2 = idx[0].search(wl.Q, K, nprobe, eps0=math.inf)
    a, b = ed2[:, K - 1], ed2[:, K]
    ok = (b - a) > REL * b
    for q in np.nonzero(ok)[0]:
        assert set(ids[q]) == set(eids[q, :K]) == set(f_ids[q])
    _exact_dists_ok(ids, d2, Y, Qr)


@pytest.mark.parametrize("st", [1, 2])
def test_low_precision_fixed_r_decisions(gist, st):
    adsx, wl, idx, Y, Cr, Qr = gist
    _, kd = oracle.knn_exact(Y, Qr[:20], 10)
    r2 = (kd[:, -1] * 1.2).astype(np.float32)
    for eps0, dd in ((2.1, 32), (1.0, 64)):
        dec, dims = idx[st].dco_fixed_r(wl.Q[:20], r2, eps0, dd)
        edec, edims, emar = oracle.dco_fixed_r(Y, Qr[:20], r2.astype(np.float64), eps0, dd)
        near = emar < ALLOW[st]
        agree = dec == edec
        assert np.all(agree | near), int((~agree & ~near).sum())
        assert (~agree).mean() < 0.01
        # at d = D the decision uses the exact FP32 distance
        both_D = (edec != oracle.REJECTED) & (dec != oracle.REJECTED)
        assert np.all((dec == edec)[both_D & (emar >= REL)])


@pytest.mark.parametrize("st", [1, 2])
def test_low_precision_ads_bracket_and_recall(gist, st):
    adsx, wl, idx, Y, Cr, Qr = gist
    K, nprobe, eps0, dd = 10, 8, 2.1, 32
    ids, d2, dims = idx[st].search(wl.Q, K, nprobe, eps0=eps0, delta_d=dd, return_dims=True)
    _exact_dists_ok(ids, d2, Y, Qr)
    eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K, nprobe)
    oids, _, _, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, K, nprobe, eps0, dd)
    gt, _ = oracle.knn_exact(Y, Qr, K)
    for q in range(Qr.shape[0]):
        top = eids[q][eids[q] >= 0]
        dec, _, mar = oracle.dco_fixed_r(Y[top], Qr[q:q + 1], np.array([ed2[q, K - 1]]), eps0, dd)
        must = set(top[(dec[0] == oracle.POSITIVE) & (mar[0] >= ALLOW[st])].tolist())
        assert must <= set(ids[q].tolist()), q
    assert oracle.recall_at(ids, gt, K) >= oracle.recall_at(oids, gt, K) - 0.01
    assert np.all(dims <= ncand * wl.D) and np.all(dims >= ncand * dd)


def test_low_precision_halves_the_index(gist):
    adsx, wl, idx, *_ = gist
    n, dp = wl.N, (wl.D + 15) // 16 * 16
    assert idx[1].device_bytes - idx[0].device_bytes == pytest.approx(n * dp * 2 + n * 4, rel=0.01)
