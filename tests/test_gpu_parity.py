"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Acceptance (FP32 storage):
  - rotation within 1e-5 relative of the FP64 rotation of the same inputs;
  - probed clusters identical except selection near-ties (the nprobe-th and
    (nprobe+1)-th centroid distances within 1e-5 relative in FP64);
  - fixed-r DCO decisions bit-exact except boundary cases whose oracle
    margin is below 1e-5 relative (counted), dims equal where decisions agree;
  - eps0 = inf: ids identical to exact IVF except near-tie queries, distances
    within 1e-5 relative;
  - eps0 = 2.1: every returned distance exact to 1e-5, the bracket invariant
    (every true IVF top-K member that passes its DCO at the exact K-th
    distance is returned), recall@K no worse than the sequential oracle's
    IVF+ recall minus 0.002;
  - FDScanning (eps0 = inf) and delta_d >= D bit-identical.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09855_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def adsx_mod():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    return adsx


@pytest.fixture(scope="module")
def c1(adsx_mod):
    """10k x 128 Gaussian mixture, 100 queries, nlist 100 (the small
    correctness configuration), with its oracle-side rotated arrays."""
    wl = W.gen_gaussian_mixture()
    ix = adsx_mod.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    Y = oracle.rotate(wl.P, wl.X)
    Cr = oracle.rotate(wl.P, wl.centroids)
    Qr = oracle.rotate(wl.P, wl.Q)
    yield wl, ix, Y, Cr, Qr
    ix.close()


def _near_tie_queries(Cr, Qr, nprobe):
    """Queries whose nprobe-th and (nprobe+1)-th centroid distances are within
    REL in FP64 (their probe sets are not determined at FP32 precision)."""
    if nprobe >= Cr.shape[0]:
        return np.zeros(Qr.shape[0], bool)
    _, pd = oracle.probe(Cr, Qr, nprobe + 1)
    a, b = pd[:, nprobe - 1], pd[:, nprobe]
    return (b - a) <= REL * np.maximum(b, 1e-30)


def _kth_near_tie(d2, K):
    if d2.shape[1] <= K:
        return np.zeros(d2.shape[0], bool)
    a, b = d2[:, K - 1], d2[:, K]
    return (b - a) <= REL * np.maximum(b, 1e-30)


def _topk_mismatch(ids, d2, eids, ed2):
    """Rows where the GPU top-K differs from the oracle's beyond FP32 order:
    the id sets (padding -1 aside) must be equal, the ids in the same order
    except between oracle distances within REL of each other, and the
    distances within REL."""
    bad = []
    for q in range(ids.shape[0]):
        v = eids[q] >= 0
        if not np.array_equal(ids[q][~v], eids[q][~v]) or set(ids[q][v]) != set(eids[q][v]):
            bad.append(q)
            continue
        e = ed2[q][v]
        tie = np.zeros(e.shape[0], bool)
        close = np.abs(np.diff(e)) <= REL * np.maximum(e[1:], 1e-30)
        tie[1:] |= close
        tie[:-1] |= close
        if np.any((ids[q][v] != eids[q][v]) & ~tie):
            bad.append(q)
            continue
        if np.any(np.abs(d2[q][v] - e) > REL * np.maximum(e, 1e-30)):
            bad.append(q)
    return bad


def test_rotation_matches_fp64(c1):
    wl, ix, Y, Cr, Qr = c1
    got = ix.rotate(wl.Q)
    scale = np.linalg.norm(Qr, axis=1, keepdims=True)
    assert np.max(np.abs(got - Qr) / scale) < REL


def test_probe_matches_oracle(c1):
    wl, ix, Y, Cr, Qr = c1
    for nprobe in (1, 10, 37, 100):
        pr, pd = ix.probe(wl.Q, nprobe)
        epr, epd = oracle.probe(Cr, Qr, nprobe)
        tie = _near_tie_queries(Cr, Qr, nprobe)
        assert tie.mean() < 0.05
        ok = ~tie
        # ordering inside the set may differ only between near-equal distances
        assert all(set(pr[q]) == set(epr[q]) for q in np.nonzero(ok)[0])
        assert np.max(np.abs(pd[ok] - epd[ok]) / np.maximum(epd[ok], 1e-30)) < 1e-4


def test_probe_duplicate_centroids_take_lowest_ids(adsx_mod):
    """Exact ties in the centroid ranking: 4 distinct centroids, each repeated
    150 times under shuffled ids.  Equal rows give bit-identical distances on
    both sides, so the probe lists must equal the oracle's exactly (ties by
    ascending cluster id), for nprobe below and above 64 and with tie groups
    larger than the selection's fast-path capacity."""
    rng = np.random.default_rng(81)
    D = 32
    base = rng.normal(0.0, 3.0, size=(4, D)).astype(np.float32)
    C = np.repeat(base, 150, axis=0)[rng.permutation(600)]
    X = (C[rng.integers(0, 600, 5000)] + rng.normal(0, 0.1, (5000, D))).astype(np.float32)
    assign = rng.integers(0, 600, 5000).astype(np.int32)
    P = W.make_P(D, 82).astype(np.float32)
    Q = (base[rng.integers(0, 4, 12)] + rng.normal(0, 0.5, (12, D))).astype(np.float32)
    ix = adsx_mod.build_index(X, P, C, assign)
    try:
        Cr, Qr = oracle.rotate(P, C), oracle.rotate(P, Q)
        for nprobe in (1, 20, 64, 150, 200, 600):
            pr, _ = ix.probe(Q, nprobe)
            epr, _ = oracle.probe(Cr, Qr, nprobe)
            assert np.array_equal(pr, epr), nprobe
    finally:
        ix.close()


def test_fixed_r_decisions_bit_exact(c1):
    wl, ix, Y, Cr, Qr = c1
    _, kd = oracle.knn_exact(Y, Qr, 10)
    for scale, eps0, dd in ((1.0, 2.1, 32), (1.0, 1.0, 16), (1.5, 2.1, 48), (0.7, 0.5, 16),
                            (1.0, math.inf, 32), (1.0, 2.1, 128), (1.0, 0.0, 64)):
        r2 = kd[:, -1] * scale
        dec, dims = ix.dco_fixed_r(wl.Q, r2.astype(np.float32), eps0, dd)
        edec, edims, emar = oracle.dco_fixed_r(Y, Qr, r2.astype(np.float32).astype(np.float64),
                                               eps0, dd)
        boundary = emar < REL
        agree = dec == edec
        assert np.all(agree | boundary), (scale, eps0, dd, int((~agree & ~boundary).sum()))
        assert np.all(dims[agree] == edims[agree])
        assert boundary.mean() < 1e-3


def test_fd_scan_matches_exact_ivf(c1):
    wl, ix, Y, Cr, Qr = c1
    for K, nprobe in ((10, 10), (1, 3), (100, 25), (10, 100)):
        ids, d2, dims = ix.search(wl.Q, K, nprobe, eps0=math.inf, delta_d=32, return_dims=True)
        eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K + 1, nprobe)
        skip = _near_tie_queries(Cr, Qr, nprobe) | _kth_near_tie(ed2, K)
        ok = ~skip
        assert skip.mean() < 0.05
        bad = _topk_mismatch(ids[ok], d2[ok], eids[ok, :K], ed2[ok, :K])
        assert not bad, (K, nprobe, bad[:5])
        _, _, _, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, K, nprobe, math.inf, 32)
        assert np.array_equal(dims[ok], (ncand * wl.D)[ok])


def test_pdscanning_is_exact_ivf_with_fewer_dims(adsx_mod, c1):
    """Sec. 6.1 PDScanning (IVF*): exact DCOs, so the results equal exact IVF.
    The dims read depend on how fast r tightens (sequential in the oracle,
    shared lazily across warps on the GPU), so they are only bounded: at least
    the first step of every candidate, at most FDScanning, and early stops
    do happen."""
    wl, ix, Y, Cr, Qr = c1
    for K, nprobe, dd in ((10, 10, 16), (100, 20, 32)):
        ids, d2, dims = adsx_mod.search_pdscan(ix, wl.Q, K, nprobe, dd, return_dims=True)
        eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K + 1, nprobe)
        skip = _near_tie_queries(Cr, Qr, nprobe) | _kth_near_tie(ed2, K)
        assert not _topk_mismatch(ids[~skip], d2[~skip], eids[~skip, :K], ed2[~skip, :K])
        _, _, fdims, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, K, nprobe, math.inf, dd)
        assert np.all(dims <= fdims) and np.all(dims >= ncand * dd)
        assert dims.sum() < fdims.sum()
        _, _, odims = oracle.ivf_pd(Y, Cr, wl.assign, Qr, K, nprobe, dd)
        assert odims.sum() < fdims.sum()


def test_fd_equals_full_step_bit_identical(c1):
    wl, ix, *_ = c1
    a = ix.search(wl.Q, 10, 10, eps0=math.inf, delta_d=32)
    b = ix.search(wl.Q, 10, 10, eps0=2.1, delta_d=128)
    c = ix.search(wl.Q, 10, 10, eps0=0.5, delta_d=256)
    for x, y in ((a, b), (a, c)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])


@pytest.mark.parametrize("K,nprobe,eps0,dd", [(10, 10, 2.1, 32), (10, 20, 2.1, 16),
                                              (100, 10, 2.1, 32), (1, 5, 1.5, 32),
                                              (10, 10, 0.5, 16)])
def test_ads_search_bracket_and_recall(c1, K, nprobe, eps0, dd):
    wl, ix, Y, Cr, Qr = c1
    ids, d2, dims = ix.search(wl.Q, K, nprobe, eps0=eps0, delta_d=dd, return_dims=True)
    eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K + 1, nprobe)
    oids, od2, odims, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, K, nprobe, eps0, dd)
    gt_ids, _ = oracle.knn_exact(Y, Qr, K)
    tie = _near_tie_queries(Cr, Qr, nprobe)
    ok = ~tie
    # every returned distance is the exact distance of that id
    for q in np.nonzero(ok)[0]:
        for i, d in zip(ids[q], d2[q]):
            if i < 0:
                continue
            ex = np.sum((Y[i] - Qr[q]) ** 2)
            assert abs(d - ex) <= REL * ex + 1e-6
    # bracket: members passing their DCO at r* (the exact K-th candidate distance)
    rstar = ed2[:, K - 1]
    for q in np.nonzero(ok)[0]:
        top = eids[q, :K]
        top = top[top >= 0]
        dec, _, mar = oracle.dco_fixed_r(Y[top], Qr[q:q + 1], np.array([rstar[q]]), eps0, dd)
        must = set(top[(dec[0] == oracle.POSITIVE) & (mar[0] >= REL)].tolist())
        assert must <= set(ids[q].tolist()), q
    # recall no worse than the sequential oracle (the shared r is never below it
    # at the same candidate set, so the GPU rejects no more true neighbours)
    r_gpu = oracle.recall_at(ids[ok], gt_ids[ok], K)
    r_orc = oracle.recall_at(oids[ok], gt_ids[ok], K)
    assert r_gpu >= r_orc - 0.002, (r_gpu, r_orc)
    # dims accounting: at least the first step of every candidate, at most all
    first = min(dd, wl.D)
    assert np.all(dims >= ncand * first) and np.all(dims <= ncand * wl.D)


def test_split_and_unsplit_scans_agree(c1):
    """Few queries are split over several warps (shared r via atomicMin,
    partial lists merged by a finalize kernel); many queries run one warp per
    query.  With FDScanning both must return identical results; with the
    test on, both keep the bracket (checked above) and their returned
    distances are exact."""
    wl, ix, Y, Cr, Qr = c1
    many = np.tile(wl.Q, (80, 1))                  # 8000 queries -> one warp each
    for K, nprobe in ((10, 10), (100, 16)):
        a_ids, a_d = ix.search(wl.Q, K, nprobe, eps0=math.inf)
        b_ids, b_d = ix.search(many, K, nprobe, eps0=math.inf)
        assert np.array_equal(a_ids, b_ids[:100]) and np.array_equal(a_d, b_d[:100])
        assert np.array_equal(b_ids[:100], b_ids[7900:])
        c_ids, c_d, c_dims = ix.search(many, K, nprobe, eps0=2.1, delta_d=16, return_dims=True)
        _, _, _, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, K, nprobe, math.inf, 32)
        assert np.all(c_dims <= np.tile(ncand, 80) * wl.D)
        for q in range(0, 8000, 997):
            qq = q % 100
            for i, d in zip(c_ids[q], c_d[q]):
                if i >= 0:
                    ex = np.sum((Y[i] - Qr[qq]) ** 2)
                    assert abs(d - ex) <= REL * ex + 1e-6


def test_device_pointer_path_matches_host_path(c1):
    import torch
    wl, ix, *_ = c1
    a_ids, a_d = ix.search(wl.Q, 10, 10, eps0=math.inf)
    Qd = torch.from_numpy(wl.Q).cuda()
    b_ids, b_d = ix.search(Qd, 10, 10, eps0=math.inf)
    torch.cuda.synchronize()
    assert np.array_equal(a_ids, b_ids.cpu().numpy())
    assert np.array_equal(a_d, b_d.cpu().numpy())
    pr_h, _ = ix.probe(wl.Q, 10)
    pr_d, _ = ix.probe(Qd, 10)
    assert np.array_equal(pr_h, pr_d.cpu().numpy())


def test_ragged_shapes_and_padding(adsx_mod):
    """D not a multiple of 16 (zero-padded to 112), N not a multiple of 32,
    empty and single-member clusters, K above the candidate count, nprobe =
    nlist, one query and zero queries."""
    rng = np.random.default_rng(5)
    N, D, nlist = 1001, 100, 40
    X = rng.standard_normal((N, D)).astype(np.float32)
    Q = rng.standard_normal((7, D)).astype(np.float32)
    P = W.make_P(D, 77).astype(np.float32)
    C = rng.standard_normal((nlist, D)).astype(np.float32)
    assign = rng.integers(0, nlist - 3, size=N).astype(np.int32)   # 3 empty clusters
    assign[0] = nlist - 3                                            # a 1-member cluster
    ix = adsx_mod.build_index(X, P, C, assign)
    Y, Cr, Qr = (oracle.rotate(P, a) for a in (X, C, Q))
    try:
        for K, nprobe, eps0, dd in ((200, 2, math.inf, 32), (5, nlist, math.inf, 16),
                                    (5, 4, 2.1, 16), (3, 1, 1.0, 112), (7, 3, 2.1, 48)):
            ids, d2 = ix.search(Q, K, nprobe, eps0=eps0, delta_d=dd)
            eids, ed2 = oracle.ivf_exact(Y, Cr, assign, Qr, K, nprobe)
            if math.isinf(eps0) or dd >= D:
                ok = ~_near_tie_queries(Cr, Qr, nprobe)
                bad = _topk_mismatch(ids[ok], d2[ok], eids[ok], ed2[ok])
                if bad:
                    q = np.nonzero(ok)[0][bad[0]]
                    gpu_pr, _ = ix.probe(Q[q:q + 1], nprobe)
                    orc_pr, orc_pd = oracle.probe(Cr, Qr[q:q + 1], nprobe + 1)
                    diff = np.nonzero(ids[q] != eids[q])[0][:6]
                    raise AssertionError("K=%d nprobe=%d q=%d probes gpu %s oracle %s (%s) "
                                         "first diffs at %s: gpu %s/%s oracle %s/%s" % (
                                             K, nprobe, q, gpu_pr[0], orc_pr[0], orc_pd[0],
                                             diff, ids[q][diff], d2[q][diff], eids[q][diff],
                                             ed2[q][diff]))
                fin = np.isfinite(ed2[ok])
                assert np.array_equal(np.isfinite(d2[ok]), fin)
            else:
                for q in range(Q.shape[0]):
                    got = [i for i in ids[q] if i >= 0]
                    assert len(set(got)) == len(got)
                    assert set(got) <= set(np.nonzero(np.isin(assign, oracle.probe(Cr, Qr[q:q+1], nprobe)[0][0]))[0])
        one_ids, _ = ix.search(Q[:1], 5, 4, eps0=math.inf)
        assert one_ids.shape == (1, 5)
        z_ids, z_d = ix.search(Q[:0], 5, 4)
        assert z_ids.shape == (0, 5)
        dec, dims = ix.dco_fixed_r(Q[:2], np.array([np.inf, 0.0], np.float32), 2.1, 16)
        assert np.all(dec[0] == oracle.POSITIVE) and np.all(dims[0] == D)
        assert np.all(dec[1] != oracle.POSITIVE)
    finally:
        ix.close()


def test_invalid_arguments_are_rejected(adsx_mod, c1):
    wl, ix, *_ = c1
    bad = [dict(K=0, nprobe=10, delta_d=32), dict(K=10, nprobe=0, delta_d=32),
           dict(K=10, nprobe=101, delta_d=32), dict(K=10, nprobe=10, delta_d=24),
           dict(K=2000, nprobe=10, delta_d=32), dict(K=10, nprobe=10, delta_d=-16)]
    for kw in bad:
        with pytest.raises(adsx_mod.AdsxError) as e:
            ix.search(wl.Q, kw["K"], kw["nprobe"], eps0=2.1, delta_d=kw["delta_d"])
        assert e.value.code == adsx_mod.EINVAL
    with pytest.raises(adsx_mod.AdsxError):
        ix.search(wl.Q, 10, 10, eps0=-1.0)
    P = wl.P.copy()
    P[0, 0] += 0.01
    with pytest.raises(adsx_mod.AdsxError) as e:
        adsx_mod.build_index(wl.X, P, wl.centroids, wl.assign)
    assert e.value.code == adsx_mod.EINVAL
    a = wl.assign.copy()
    a[3] = wl.nlist
    with pytest.raises(adsx_mod.AdsxError):
        adsx_mod.build_index(wl.X, wl.P, wl.centroids, a)
