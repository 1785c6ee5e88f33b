"""Query rotation q' = P q (Sec. 3.1) on the tensor cores, through the C ABI.

Every query value and every entry of P is split into integer digits; the
digit products are summed by tcgen05.mma, where every partial sum is an
integer that FP32 holds exactly, and the levels are added by compensated
summation and rounded once.  So the result is the FP64 product of the FP32 inputs, rounded
to FP32, up to the truncated digit tails (below 2^-(bT) of each row's largest
value, bT >= 28).  Checked against numpy FP64:
  - every value within half an ulp of the FP64 result plus the tail bound
    2^-22 (max|q| sum_k |P_ck| + max_k |P_ck| sum_k |q_k|), for padded D
    from 16 to 1024 (digit widths 8, 7, 6 and 5), most of them exactly the
    rounded FP64 value;
  - the compensated FP32 mode (ADSX_ROT_FP32) within the same bound;
  - rows spanning 12 orders of magnitude, a zero row, a single huge value;
  - FDScanning with either rotation returns exact IVF on queries away from
    near-ties, with distances within 1e-5;
  - the mode is refused where it cannot run (a Kac-walk index, D > 1024).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09855_gb300 import workloads as W
from gpu_helpers import REL, kth_near_tie, near_tie_queries

pytestmark = pytest.mark.gpu


def _index(D, N=1500, nlist=12, seed=0):
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    wl = W.random_small(N, D, 64, nlist, seed=seed)
    ix = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    return adsx, wl, ix


def _check_against_fp64(P, Q, got):
    # the FP32 inputs the library was given, multiplied in FP64
    P64, Q64 = P.astype(np.float32).astype(np.float64), Q.astype(np.float32).astype(np.float64)
    ref = Q64 @ P64.T
    ref32 = ref.astype(np.float32)
    ulp = np.spacing(np.abs(ref32)).astype(np.float64)
    aq, ap = np.abs(Q64), np.abs(P64)
    tail = 2.0 ** -22 * (np.max(aq, axis=1, keepdims=True) * np.sum(ap, axis=1)[None, :] +
                         np.sum(aq, axis=1, keepdims=True) * np.max(ap, axis=1)[None, :])
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= 0.5 * ulp + tail), float(np.max(err - 0.5 * ulp - tail))
    return float(np.mean(got == ref32))


@pytest.mark.parametrize("D", [16, 37, 64, 128, 300, 960, 1024])
def test_tensor_rotation_is_the_rounded_fp64_product(D):
    adsx, wl, ix = _index(D)
    try:
        ix.set_query_rotation(adsx.ROT_TENSOR)
        got = ix.rotate(wl.Q)
        exact = _check_against_fp64(wl.P, wl.Q, got)
        ix.set_query_rotation(adsx.ROT_FP32)
        got2 = ix.rotate(wl.Q)
        exact2 = _check_against_fp64(wl.P, wl.Q, got2)
        print("D %d: rounded FP64 product exactly in %.3f (tensor) / %.3f (Dot2) of the values"
              % (D, exact, exact2))
        assert exact >= 0.5, exact
        ix.set_query_rotation(adsx.ROT_TENSOR)
        assert np.array_equal(ix.rotate(wl.Q), got)       # deterministic
    finally:
        ix.close()


def test_tensor_rotation_wide_ranges_and_zero_rows():
    adsx, wl, ix = _index(96)
    try:
        ix.set_query_rotation(adsx.ROT_TENSOR)
        rng = np.random.default_rng(3)
        Q = rng.standard_normal((40, 96)).astype(np.float32)
        Q[0] = 0.0                                          # zero row -> zero
        Q[1] *= np.logspace(-6, 6, 96).astype(np.float32)    # 12 decades in one row
        Q[2] = 0.0
        Q[2, 17] = 3.0e30                                    # one huge value
        Q[3] *= 1e-30                                        # a tiny row
        got = ix.rotate(Q)
        assert np.all(got[0] == 0.0)
        _check_against_fp64(wl.P, Q, got)
    finally:
        ix.close()


def test_search_with_either_rotation_is_exact_ivf():
    adsx, wl, ix = _index(128, N=3000, nlist=16, seed=5)
    try:
        Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
        K, nprobe = 10, 4
        eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K + 1, nprobe)
        ok = ~(near_tie_queries(Cr, Qr, nprobe) | kth_near_tie(ed2, K))
        for mode in (adsx.ROT_TENSOR, adsx.ROT_FP32):
            ix.set_query_rotation(mode)
            ids, d2 = ix.search(wl.Q, K, nprobe, eps0=math.inf)
            for q in np.nonzero(ok)[0]:
                assert set(ids[q]) == set(eids[q, :K]), (mode, q)
            assert np.max(np.abs(d2 - ed2[:, :K]) / ed2[:, :K]) <= REL
    finally:
        ix.close()


def test_tensor_rotation_refused_where_unavailable():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    wl = W.random_small(600, 64, 8, 4, seed=2)
    pairs, cs = W.make_kac_walk(64, 12, 1)
    kx = adsx.build_index_kac(wl.X, pairs, cs, wl.centroids, wl.assign)
    try:
        with pytest.raises(adsx.AdsxError):
            kx.set_query_rotation(adsx.ROT_TENSOR)
        kx.set_query_rotation(adsx.ROT_FP32)
    finally:
        kx.close()
    wl = W.random_small(300, 1100, 8, 2, seed=4)
    big = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    try:
        with pytest.raises(adsx.AdsxError):
            big.set_query_rotation(adsx.ROT_TENSOR)
        with pytest.raises(adsx.AdsxError):
            big.set_query_rotation(7)
    finally:
        big.close()
