"""Batched uneven form: per-query K and nprobe in one persistent launch
(device-side plan, longest-first order, long queries split), checked against
the FP64 oracle query by query, against the uniform search, with custom
output offsets, and replayed from a captured CUDA graph."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09855_gb300 import workloads as W
from gpu_helpers import REL, kth_near_tie, near_tie_queries, topk_row_mismatch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    wl = W.gen_gaussian_mixture()
    ix = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
    rng = np.random.default_rng(17)
    Ks = np.array([1, 10, 100], np.int32)[rng.integers(0, 3, size=wl.Q.shape[0])]
    nps = np.rint(np.exp(rng.uniform(0, np.log(100), size=wl.Q.shape[0]))).astype(np.int32)
    yield adsx, wl, ix, Y, Cr, Qr, Ks, nps
    ix.close()


def _split(flat, Ks):
    offs = np.concatenate([[0], np.cumsum(Ks)])
    return [flat[offs[q]:offs[q + 1]] for q in range(len(Ks))]


def test_batched_fd_matches_exact_ivf_per_query(c1):
    adsx, wl, ix, Y, Cr, Qr, Ks, nps = c1
    ids, d2, dims = adsx.search_batched(ix, wl.Q, Ks, nps, eps0=math.inf,
                                                    return_dims=True)
    ids_q, d2_q = _split(ids, Ks), _split(d2, Ks)
    bad = 0
    for q in range(wl.Q.shape[0]):
        K, npb = int(Ks[q]), int(nps[q])
        eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr[q:q + 1], K + 1, npb)
        if near_tie_queries(Cr, Qr[q:q + 1], npb)[0] or kth_near_tie(ed2, K)[0]:
            continue
        bad += topk_row_mismatch(ids_q[q], d2_q[q], eids[0, :K], ed2[0, :K])
        _, _, _, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr[q:q + 1], K, npb, math.inf, 32)
        assert dims[q] == ncand[0] * wl.D
    assert bad == 0


def test_batched_ads_exact_distances_and_bracket(c1):
    adsx, wl, ix, Y, Cr, Qr, Ks, nps = c1
    ids, d2 = adsx.search_batched(ix, wl.Q, Ks, nps, eps0=2.1, delta_d=16)
    ids_q, d2_q = _split(ids, Ks), _split(d2, Ks)
    for q in range(wl.Q.shape[0]):
        K, npb = int(Ks[q]), int(nps[q])
        if near_tie_queries(Cr, Qr[q:q + 1], npb)[0]:
            continue
        for i, d in zip(ids_q[q], d2_q[q]):
            if i >= 0:
                ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                assert abs(d - ex) <= REL * ex + 1e-6
        eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr[q:q + 1], K, npb)
        top = eids[0][eids[0] >= 0]
        dec, _, mar = oracle.dco_fixed_r(Y[top], Qr[q:q + 1], np.array([ed2[0, K - 1]]), 2.1, 16)
        must = set(top[(dec[0] == oracle.POSITIVE) & (mar[0] >= REL)].tolist())
        assert must <= set(ids_q[q].tolist()), q


def test_batched_with_constant_arguments_equals_uniform_search(c1):
    adsx, wl, ix, *_ = c1
    nq = wl.Q.shape[0]
    for K, npb in ((10, 10), (100, 37)):
        a_ids, a_d = ix.search(wl.Q, K, npb, eps0=math.inf)
        b_ids, b_d = adsx.search_batched(ix, wl.Q, np.full(nq, K), np.full(nq, npb), eps0=math.inf)
        assert np.array_equal(a_ids.reshape(-1), b_ids) and np.array_equal(a_d.reshape(-1), b_d)


def test_batched_custom_output_offsets(c1):
    adsx, wl, ix, Y, Cr, Qr, Ks, nps = c1
    nq = wl.Q.shape[0]
    order = np.arange(nq)[::-1]
    offs = np.zeros(nq, np.int64)
    run = 3                                           # a gap before the first slice
    for q in order:
        offs[q] = run
        run += Ks[q]
    ids, d2 = adsx.search_batched(ix, wl.Q, Ks, nps, eps0=math.inf, out_offsets=offs,
                                  out_total=run + 5)
    ref_ids, ref_d = adsx.search_batched(ix, wl.Q, Ks, nps, eps0=math.inf)
    for q, (a, b) in enumerate(zip(_split(ref_ids, Ks), _split(ref_d, Ks))):
        assert np.array_equal(ids[offs[q]:offs[q] + Ks[q]], a)
        assert np.array_equal(d2[offs[q]:offs[q] + Ks[q]], b)


def test_batched_in_a_captured_cuda_graph(c1):
    import torch
    adsx, wl, ix, Y, Cr, Qr, Ks, nps = c1
    Qd = torch.from_numpy(wl.Q).cuda()
    Kd = torch.from_numpy(Ks).cuda()
    Pd = torch.from_numpy(nps).cuda()
    total, maxK, maxP = int(Ks.sum()), int(Ks.max()), int(nps.max())
    ref_ids, ref_d = adsx.search_batched(ix, wl.Q, Ks, nps, eps0=math.inf)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        adsx.search_batched(ix, Qd, Kd, Pd, eps0=math.inf, max_K=maxK, max_nprobe=maxP,
                            out_total=total)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        g_ids, g_d = adsx.search_batched(ix, Qd, Kd, Pd, eps0=math.inf, max_K=maxK,
                                         max_nprobe=maxP, out_total=total)
    for _ in range(2):
        g_ids.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(g_ids.cpu().numpy(), ref_ids)
        assert np.array_equal(g_d.cpu().numpy(), ref_d)
    # new queries copied into the captured input buffer are searched on replay
    Qd.copy_(torch.from_numpy(np.ascontiguousarray(wl.Q[::-1])))
    g.replay()
    torch.cuda.synchronize()
    rev_ids, _ = adsx.search_batched(ix, np.ascontiguousarray(wl.Q[::-1]), Ks, nps, eps0=math.inf)
    assert np.array_equal(g_ids.cpu().numpy(), rev_ids)


def test_batched_rejects_bad_per_query_values(c1):
    import torch
    adsx, wl, ix, *_ = c1
    nq = wl.Q.shape[0]
    bad_K = np.full(nq, 10)
    bad_K[5] = 0
    with pytest.raises(adsx.AdsxError) as e:
        adsx.search_batched(ix, wl.Q, bad_K, np.full(nq, 10), max_K=10, max_nprobe=10)
    assert e.value.code == adsx.EINVAL
    # device arrays: checked on the device, reported through the error word
    Qd = torch.from_numpy(wl.Q).cuda()
    adsx.search_batched(ix, Qd, torch.from_numpy(bad_K).cuda(), torch.full((nq,), 10).cuda(),
                        max_K=10, max_nprobe=10, out_total=10 * nq)
    with pytest.raises(adsx.AdsxError) as e:
        adsx.stream_status(ix, torch.cuda.current_stream())
    assert e.value.code == adsx.EINVAL
    adsx.stream_status(ix, torch.cuda.current_stream())     # cleared


def test_autotune_picks_a_supported_step_and_delta_d_zero_uses_it(c1):
    adsx, wl, ix, Y, Cr, Qr, Ks, nps = c1
    dd, ip, ms = adsx.autotune(ix, wl.Q, 10, 10)
    assert dd in (16, 32, 48, 64) and ip in (24, 48, 96) and ms > 0
    a_ids, a_d = ix.search(wl.Q, 10, 10, eps0=math.inf, delta_d=0)
    b_ids, b_d = ix.search(wl.Q, 10, 10, eps0=math.inf, delta_d=dd)
    assert np.array_equal(a_ids, b_ids)
    ids, d2 = ix.search(wl.Q, 10, 10, eps0=2.1, delta_d=0)
    for q in range(0, 100, 7):
        for i, d in zip(ids[q], d2[q]):
            if i >= 0:
                ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                assert abs(d - ex) <= REL * ex + 1e-6
