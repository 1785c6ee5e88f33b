"""Serving form: the continuous-batching request loop.

Requests submitted concurrently from several host threads are batched as
they arrive, with several batches in flight on different streams; each
result must be the same alone (a one-query adsx_search) and in the mix:
bit-identical under FDScanning, and under ADSampling every returned
distance exact, the bracket invariant kept, and at least 99% of returned ids
shared with the alone result (which ids near the decision boundary survive
depends on the order in which the warps tighten r).  Admission by memory,
cancellation and bounded waits are checked on the host side."""
import math
import threading

import numpy as np
import pytest

import oracle
from paper_2303_09855_gb300 import workloads as W
from gpu_helpers import REL, near_tie_queries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    wl = W.gen_gaussian_mixture()
    ix = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
    yield adsx, wl, ix, Y, Cr, Qr
    ix.close()


def _requests(n, nq, seed):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, nq)), int([1, 10, 100][rng.integers(0, 3)]),
             int([5, 10, 20][rng.integers(0, 3)])) for _ in range(n)]


def _run_mix(adsx, srv, wl, reqs, eps0, nthreads=6):
    out = [None] * len(reqs)

    def client(k):
        tickets = []
        for i in range(k, len(reqs), nthreads):
            q, K, npb = reqs[i]
            tickets.append((i, srv.submit(wl.Q[q], K, npb, eps0=eps0, delta_d=16)))
        for i, t in tickets:
            out[i] = srv.wait(t, timeout_ms=60000)

    th = [threading.Thread(target=client, args=(k,)) for k in range(nthreads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return out


def test_mix_equals_alone(c1):
    adsx, wl, ix, Y, Cr, Qr = c1
    srv = adsx.Server(ix, max_slots=96, max_batch=24, n_streams=4, mem_budget_bytes=1 << 28,
                      max_K=100, max_nprobe=20)
    try:
        reqs = _requests(300, wl.Q.shape[0], 3)
        for eps0 in (math.inf, 2.1):
            mix = _run_mix(adsx, srv, wl, reqs, eps0)
            shared = total = 0
            for (q, K, npb), (ids, d2, dims) in zip(reqs, mix):
                a_ids, a_d = ix.search(wl.Q[q:q + 1], K, npb, eps0=eps0, delta_d=16)
                if math.isinf(eps0):
                    assert np.array_equal(ids, a_ids[0]) and np.array_equal(d2, a_d[0])
                    continue
                for i, d in zip(ids, d2):
                    if i >= 0:
                        ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                        assert abs(d - ex) <= REL * ex + 1e-6
                if not near_tie_queries(Cr, Qr[q:q + 1], npb)[0]:
                    eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Qr[q:q + 1], K, npb)
                    top = eids[0][eids[0] >= 0]
                    dec, _, mar = oracle.dco_fixed_r(Y[top], Qr[q:q + 1],
                                                     np.array([ed2[0, K - 1]]), eps0, 16)
                    must = set(top[(dec[0] == oracle.POSITIVE) & (mar[0] >= REL)].tolist())
                    assert must <= set(ids.tolist())
                v = a_ids[0] >= 0
                shared += len(set(ids.tolist()) & set(a_ids[0][v].tolist()))
                total += int(v.sum())
            if total:
                assert shared >= 0.99 * total
        st = srv.stats()
        assert st["completed"] == 600 and st["max_inflight_batches"] >= 2
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    finally:
        srv.close()


def test_admission_by_memory_and_rejection(c1):
    adsx, wl, ix, *_ = c1
    # budget for two requests: never more than two in flight
    one = 12 * 128 + 4 * 100 + 16 * 1 + 4 * 10 + 8 * 16 + 8 * 16 * 10 + 12 * 10 + 64
    srv = adsx.Server(ix, max_slots=64, max_batch=64, n_streams=4, mem_budget_bytes=2 * one + 10,
                      max_K=10, max_nprobe=10)
    try:
        ts = [srv.submit(wl.Q[i % 100], 10, 10, eps0=math.inf) for i in range(40)]
        for t in ts:
            srv.wait(t)
        assert srv.stats()["max_inflight_queries"] <= 2
    finally:
        srv.close()
    tiny = adsx.Server(ix, max_slots=4, max_batch=4, n_streams=1, mem_budget_bytes=one - 1,
                       max_K=10, max_nprobe=10)
    try:
        with pytest.raises(adsx.AdsxError) as e:
            tiny.submit(wl.Q[0], 10, 10)
        assert e.value.code == adsx.ENOMEM
    finally:
        tiny.close()


def test_cancel_and_bounded_wait(c1):
    adsx, wl, ix, *_ = c1
    one = 12 * 128 + 4 * 100 + 16 * 1 + 4 * 10 + 8 * 16 + 8 * 16 * 10 + 12 * 10 + 64
    # one request at a time, so later submissions are still queued
    srv = adsx.Server(ix, max_slots=1, max_batch=1, n_streams=1, mem_budget_bytes=one,
                      max_K=10, max_nprobe=10)
    try:
        ts = [srv.submit(wl.Q[i], 10, 10) for i in range(30)]
        cancelled = None
        for t in reversed(ts):
            try:
                srv.cancel(t)
                cancelled = t
                break
            except adsx.AdsxError:
                continue
        assert cancelled is not None
        with pytest.raises(adsx.AdsxError):
            srv.wait(cancelled)
        for t in ts:
            if t is cancelled:
                continue
            try:
                srv.wait(t, timeout_ms=0)          # may or may not be done yet
            except adsx.AdsxError as e:
                assert e.code == adsx.ETIMEOUT
                srv.wait(t, timeout_ms=60000)
    finally:
        srv.close()
