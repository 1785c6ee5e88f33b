"""Cosine-similarity and inner-product indexes (Sec. 8, extension (1)) through
the C ABI against the FP64 oracle.

Inner product (ADSX_IP): the DCO "is <o,q> at least r" runs Algorithm 1 on
o/||o||, q/||q|| against 2 - 2r/(||o|| ||q||); clusters are probed by the
largest <c, q>.  Acceptance:
  - eps0 = inf: ids equal the oracle's exact IVF for inner products except
    selection and K-th near-ties; returned inner products within 1e-5 of
    ||o|| ||q|| (the scale the FP32 distance of the normalised vectors
    carries) of the exact ones;
  - eps0 = 2.1: every returned value exact to that tolerance; the bracket
    invariant (every true top-K member that passes its DCO at the exact K-th
    inner product r* is returned: the live r is never above r*, and a lower r
    only loosens every threshold); recall no worse than the sequential
    oracle's minus 0.01;
  - BF16 storage (exact FP32 recheck) and the batched form give the same
    exact-mode results.
Cosine (ADSX_COSINE): the Euclidean path on normalised vectors, returning
1 - d^2/2; the same checks against the oracle on normalised rows.  A zero
data row is rejected; adsx_dco_fixed_r and adsx_search_noalloc reject
non-L2 indexes.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import REL, kth_near_tie, near_tie_queries, topk_row_mismatch

pytestmark = pytest.mark.gpu

K, NPROBE = 10, 6


@pytest.fixture(scope="module")
def lib():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    return adsx


@pytest.fixture(scope="module")
def data():
    from paper_2303_09855_gb300 import workloads as W
    rng = np.random.default_rng(71)
    N, D, nq, nlist = 24_000, 96, 60, 40
    centres = rng.normal(0.0, 1.5, size=(nlist, D))
    lab = rng.integers(0, nlist, size=N)
    scale = rng.uniform(0.3, 3.0, size=(N, 1))
    X = ((centres[lab] + rng.standard_normal((N, D))) * scale).astype(np.float32)
    Q = (centres[rng.integers(0, nlist, size=nq)] + rng.standard_normal((nq, D))).astype(np.float32)
    C = np.stack([X[lab == c].mean(0) for c in range(nlist)]).astype(np.float32)
    P = W.make_P(D, 72).astype(np.float32)
    Y, Cr, Qr = oracle.rotate(P, X), oracle.rotate(P, C), oracle.rotate(P, Q)
    return X, Q, C, lab.astype(np.int32), P, Y, Cr, Qr


def _ip_scale(Y, Qr, ids):
    """||o|| ||q|| of each returned (query, id)."""
    on = np.linalg.norm(Y, axis=1)
    qn = np.linalg.norm(Qr, axis=1)
    return on[np.clip(ids, 0, None)] * qn[:, None]


def _ip_skip(Y, Cr, Qr, eids, eip, nprobe, K):
    """Queries whose probe set or K-th member is not determined at FP32
    precision: the nprobe-th / (nprobe+1)-th centroid inner products within
    1e-5 of ||q||^2 + max||c||^2, or the K-th / (K+1)-th inner products within
    1e-5 of ||o|| ||q||."""
    qn2 = np.sum(Qr * Qr, axis=1)
    M2 = np.max(np.sum(Cr * Cr, axis=1))
    cip = -np.sort(-(Qr @ Cr.T), axis=1)
    sel = (cip[:, nprobe - 1] - cip[:, nprobe]) <= 1e-5 * (qn2 + M2)
    sc = _ip_scale(Y, Qr, eids)
    kth = (eip[:, K - 1] - eip[:, K]) <= 1e-5 * np.maximum(sc[:, K - 1], sc[:, K])
    return sel | kth


def _ip_rows_match(ids, ip, eids, eip, scale):
    """Same id set and order except between oracle values within tolerance;
    values within tolerance."""
    tol = 1e-5 * scale
    if set(ids) != set(eids):
        return False
    close = np.abs(np.diff(eip)) <= np.maximum(tol[1:], tol[:-1])
    tie = np.zeros(len(eids), bool)
    tie[1:] |= close
    tie[:-1] |= close
    if np.any((ids != eids) & ~tie):
        return False
    return bool(np.all(np.abs(ip - eip) <= tol + 1e-6))


def test_inner_product_exact_mode(lib, data):
    X, Q, C, lab, P, Y, Cr, Qr = data
    ix = lib.build_index(X, P, C, lab, metric=lib.IP)
    try:
        assert ix.metric == lib.IP
        ids, ip = ix.search(Q, K, NPROBE, eps0=math.inf)
        eids, eip = oracle.ivf_exact_ip(Y, Cr, lab, Qr, K + 1, NPROBE)
        skip = _ip_skip(Y, Cr, Qr, eids, eip, NPROBE, K)
        sc = _ip_scale(Y, Qr, eids[:, :K])
        bad = [q for q in range(Q.shape[0]) if not skip[q] and
               not _ip_rows_match(ids[q], ip[q], eids[q, :K], eip[q, :K], sc[q])]
        assert not bad and (~skip).sum() >= Q.shape[0] - 6, bad
        # results are ordered largest first
        assert np.all(np.diff(ip, axis=1) <= 0)
    finally:
        ix.close()


def test_inner_product_adsampling_bracket_and_recall(lib, data):
    X, Q, C, lab, P, Y, Cr, Qr = data
    eps0, dd = 2.1, 16
    ix = lib.build_index(X, P, C, lab, metric=lib.IP)
    try:
        ids, ip, dims = ix.search(Q, K, NPROBE, eps0=eps0, delta_d=dd, return_dims=True)
        eids, eip = oracle.ivf_exact_ip(Y, Cr, lab, Qr, K + 1, NPROBE)
        oids, _, odims, ncand = oracle.ivf_ads_ip(Y, Cr, lab, Qr, K, NPROBE, eps0, dd)
        skip = _ip_skip(Y, Cr, Qr, eids, eip, NPROBE, K)
        sc = _ip_scale(Y, Qr, ids)
        for q in range(Q.shape[0]):
            for j, (i, v) in enumerate(zip(ids[q], ip[q])):
                if i >= 0:
                    ex = float(Y[i] @ Qr[q])
                    assert abs(v - ex) <= 1e-5 * sc[q, j] + 1e-6, (q, i, v, ex)
            if skip[q]:
                continue
            rstar = eip[q, K - 1]
            must = set()
            for i in eids[q, :K]:
                dec, _, _, mar = oracle.dco_ip(Y[i], Qr[q], rstar, eps0, dd)
                if dec == oracle.POSITIVE and mar >= REL:
                    must.add(int(i))
            assert must <= set(ids[q].tolist()), q
        r_gpu = oracle.recall_at(ids, eids[:, :K], K)
        r_orc = oracle.recall_at(oids, eids[:, :K], K)
        assert r_gpu >= r_orc - 0.01, (r_gpu, r_orc)
        assert dims.sum() < ncand.sum() * X.shape[1]           # early decisions happen
    finally:
        ix.close()


def test_inner_product_bf16_and_batched_agree_in_exact_mode(lib, data):
    X, Q, C, lab, P, Y, Cr, Qr = data
    ix32 = lib.build_index(X, P, C, lab, metric=lib.IP)
    ix16 = lib.build_index(X, P, C, lab, storage=lib.BF16, metric=lib.IP)
    try:
        a_ids, a_ip = ix32.search(Q, K, NPROBE, eps0=math.inf)
        b_ids, b_ip = ix16.search(Q, K, NPROBE, eps0=math.inf)
        nq = Q.shape[0]
        c_ids, c_ip = lib.search_batched(ix32, Q, np.full(nq, K, np.int32),
                                         np.full(nq, NPROBE, np.int32), eps0=math.inf)
        eids, eip = oracle.ivf_exact_ip(Y, Cr, lab, Qr, K + 1, NPROBE)
        skip = _ip_skip(Y, Cr, Qr, eids, eip, NPROBE, K)
        sc = _ip_scale(Y, Qr, eids[:, :K])
        for ids, ip in ((b_ids, b_ip), (c_ids.reshape(nq, K), c_ip.reshape(nq, K))):
            bad = [q for q in range(nq) if not skip[q] and
                   not _ip_rows_match(ids[q], ip[q], eids[q, :K], eip[q, :K], sc[q])]
            assert not bad, bad
    finally:
        ix32.close()
        ix16.close()


def test_cosine_exact_and_adsampling(lib, data):
    X, Q, C, lab, P, Y, Cr, Qr = data
    Yn, Cn, Qn = oracle.normalize_rows(Y), oracle.normalize_rows(Cr), oracle.normalize_rows(Qr)
    ix = lib.build_index(X, P, C, lab, metric=lib.COSINE)
    try:
        ids, cs = ix.search(Q, K, NPROBE, eps0=math.inf)
        eids, ed2 = oracle.ivf_exact(Yn, Cn, lab, Qn, K + 1, NPROBE)
        skip = near_tie_queries(Cn, Qn, NPROBE) | kth_near_tie(ed2, K)
        bad = [q for q in range(Q.shape[0]) if not skip[q] and
               topk_row_mismatch(ids[q], 2.0 * (1.0 - cs[q]), eids[q, :K], ed2[q, :K])
               and not np.allclose(cs[q], 1.0 - ed2[q, :K] / 2.0, atol=1e-5)]
        assert not bad, bad
        for q in np.nonzero(~skip)[0]:
            assert set(ids[q]) == set(eids[q, :K])
            assert np.all(np.abs(cs[q] - (1.0 - ed2[q, :K] / 2.0)) <= 1e-5)
        eps0, dd = 2.1, 16
        a_ids, a_cs = ix.search(Q, K, NPROBE, eps0=eps0, delta_d=dd)
        oids, _, _, _ = oracle.ivf_ads(Yn, Cn, lab, Qn, K, NPROBE, eps0, dd)
        for q in range(Q.shape[0]):
            for i, v in zip(a_ids[q], a_cs[q]):
                if i >= 0:
                    ex = float(Yn[i] @ Qn[q])
                    assert abs(v - ex) <= 1e-5, (q, i, v, ex)
            if skip[q]:
                continue
            top = eids[q, :K]
            dec, _, mar = oracle.dco_fixed_r(Yn[top], Qn[q:q + 1], np.array([ed2[q, K - 1]]),
                                             eps0, dd)
            must = set(top[(dec[0] == oracle.POSITIVE) & (mar[0] >= REL)].tolist())
            assert must <= set(a_ids[q].tolist()), q
        assert oracle.recall_at(a_ids, eids[:, :K], K) >= oracle.recall_at(oids, eids[:, :K], K) - 0.01
    finally:
        ix.close()


def test_metric_argument_checks(lib, data):
    import torch
    X, Q, C, lab, P, Y, Cr, Qr = data
    Xz = X.copy()
    Xz[5] = 0.0
    with pytest.raises(lib.AdsxError) as e:
        lib.build_index(Xz, P, C, lab, metric=lib.COSINE)
    assert e.value.code == lib.EINVAL
    with pytest.raises(lib.AdsxError):
        lib.build_index(X, P, C, lab, metric=7)
    ix = lib.build_index(X, P, C, lab, metric=lib.IP)
    try:
        with pytest.raises(lib.AdsxError):
            ix.dco_fixed_r(Q[:2], np.ones(2, np.float32), 2.1, 16)
        with pytest.raises(lib.AdsxError):
            lib.search_noalloc(ix, torch.from_numpy(Q).cuda(), K, NPROBE)
    finally:
        ix.close()
