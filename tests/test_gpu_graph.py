"""Graph search with ADSampling DCOs (HNSW+, Sec. 4; the base-layer greedy
beam search of Sec. 2.2.1) through the C ABI, against the FP64 oracle running
the same algorithm on the same (exported) graph and start vertices:
  - the kNN graph: every vertex's neighbour list equals the oracle's exact
    IVF list (self excluded) except near-ties; a cluster's entry vertices
    equal the oracle's farthest-point samples, and where an FP32 near-tie
    let them part, each GPU entry is still a valid farthest-point step given
    the GPU's earlier ones;
  - eps0 = inf (exact DCOs: HNSW's own search), eps0 = 2.1 and 1.0, for
    HNSW+ and HNSW++ (Sec. 5.1), against the oracle's search in the paper's
    sequential order (one vertex at a time, the threshold updated after
    every vertex): the GPU tests a batch of 32 vertices side by side and then
    replays the decisions in list order, so every query whose oracle run has
    no comparison closer than 1e-5 relative returns the oracle's ids and
    samples the oracle's dims exactly (the others, counted, are a small
    minority); returned distances exact to 1e-5, no duplicates; HNSW++ with
    exact DCOs equals HNSW bit for bit;
  - many entries per cluster (a small upper layer: 72 start vertices, more
    than ef) against the oracle given the same starts;
  - maximum sizes: ef = K = 512, 1024 start vertices (16 clusters x 64);
  - edge cases: fewer vertices than degree + 1 (padded neighbour lists),
    D not a multiple of 16, an empty cluster, more entries asked than a
    cluster has, K = ef above N (padded results), no queries;
  - a cosine index: the graph over the normalised vectors, similarities
    1 - d^2/2 of the oracle's search on normalised rows (HNSW+ and HNSW++);
  - argument checks (K > ef, entries per cluster out of range, a 16-bit
    index, an inner-product index).
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import REL, kth_near_tie, near_tie_queries, topk_row_mismatch

pytestmark = pytest.mark.gpu

K, EF, NE, EPC = 10, 64, 3, 3


def _match_sequential(ids, d2, dims, Y, Qr, oids, od2, odims, margin, ok, min_frac=0.8):
    """The GPU search replays each batch in list order, so it follows the
    paper's sequential order (the oracle) exactly up to rounding: every
    query whose probe set is not a near-tie and whose closest call in the
    oracle (smallest relative gap of any comparison that decided the search)
    is at least REL returns the oracle's ids and samples the oracle's number
    of dims (the returned ids in the oracle's order, except between keys
    within REL of each other); the others are counted and must be a small
    minority.  Every
    returned distance is exact and the ids of a query are distinct."""
    good = ok & (margin >= REL)
    for q in np.nonzero(good)[0]:
        assert not topk_row_mismatch(ids[q], d2[q], oids[q], od2[q]), (q, ids[q], oids[q])
        if dims is not None:
            assert dims[q] == odims[q], (q, dims[q], odims[q])
    for q in range(len(Qr)):
        row = ids[q][ids[q] >= 0]
        assert len(set(row.tolist())) == len(row), q
        for i, d in zip(ids[q], d2[q]):
            if i >= 0:
                ex = float(np.sum((Y[i] - Qr[q]) ** 2))
                assert abs(d - ex) <= REL * ex + 1e-6, (q, i, d, ex)
    print("graph parity: %d of %d queries checked exactly (%d near a tie)"
          % (int(good.sum()), len(good), int((~good).sum())))
    assert good.mean() >= min_frac, good.mean()


@pytest.fixture(scope="module")
def gr():
    from paper_2303_09855_gb300 import adsx, build
    from paper_2303_09855_gb300 import workloads as W
    build.build()
    wl = W.gen_gaussian_mixture()
    ix = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    g = adsx.build_graph(ix, wl.X, degree=32, nprobe=10, entries_per_cluster=EPC)
    Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
    nbr, ent = adsx.graph_export(g)
    yield adsx, wl, ix, g, Y, Cr, Qr, nbr, ent
    g.close()
    ix.close()


def test_graph_lists_and_entries_match_oracle(gr):
    adsx, wl, ix, g, Y, Cr, Qr, nbr, ent = gr
    assert nbr.shape == (wl.N, 32)
    rows = np.random.default_rng(7).choice(wl.N, 300, replace=False)
    eids, ed2 = oracle.ivf_exact(Y, Cr, wl.assign, Y[rows], 34, 10)
    skip = near_tie_queries(Cr, Y[rows], 10) | kth_near_tie(ed2, 33)
    checked = 0
    for j, r in enumerate(rows):
        if skip[j]:
            continue
        want = [v for v in eids[j] if v != r][:32]
        assert set(nbr[r].tolist()) == set(want), r
        checked += 1
    assert checked >= 250
    assert ent.shape == (wl.nlist, EPC)
    want = oracle.cluster_entries(Y, Cr, wl.assign, EPC)
    same = 0
    for c in range(wl.nlist):
        mem = np.nonzero(wl.assign == c)[0]
        if len(mem) == 0:
            assert np.all(ent[c] == -1)
            continue
        same += np.array_equal(ent[c], want[c])
        assert set(ent[c][ent[c] >= 0].tolist()) <= set(mem.tolist()), c
        d = np.sum((Y[mem] - Cr[c]) ** 2, axis=1)
        e0 = float(np.sum((Y[ent[c, 0]] - Cr[c]) ** 2))
        assert e0 <= d.min() * (1 + REL) + 1e-6, c
        nearest = np.full(len(mem), np.inf)
        for e in range(1, EPC):
            nearest = np.minimum(nearest, np.sum((Y[mem] - Y[ent[c, e - 1]]) ** 2, axis=1))
            if ent[c, e] < 0:
                assert nearest.max() <= 1e-6 and np.all(ent[c, e:] == -1), c
                break
            got = nearest[np.searchsorted(mem, ent[c, e])]
            assert got >= nearest.max() * (1 - REL) - 1e-6, (c, e)
    assert same >= 0.9 * wl.nlist


@pytest.mark.parametrize("eps0,dd,pp", [(math.inf, 32, False), (2.1, 32, False), (2.1, 16, False),
                                         (math.inf, 32, True), (2.1, 32, True), (1.0, 16, True)])
def test_graph_search_matches_oracle(gr, eps0, dd, pp):
    adsx, wl, ix, g, Y, Cr, Qr, nbr, ent = gr
    ids, d2, dims = g.search(wl.Q, K, EF, eps0=eps0, delta_d=dd, return_dims=True, n_entry=NE,
                             decoupled=pp)
    probes, _ = oracle.probe(Cr, Qr, NE)
    starts = ent[probes].reshape(len(Qr), -1)
    oids, od2, odims, iters, margin = oracle.graph_search(Y, nbr, starts, Qr, K, EF, eps0, dd,
                                                          max_iter=4 * EF, pp=pp,
                                                          return_margin=True)
    ok = ~near_tie_queries(Cr, Qr, NE)
    _match_sequential(ids, d2, dims, Y, Qr, oids, od2, odims, margin, ok)
    assert np.all(np.diff(np.where(ids >= 0, d2, np.inf), axis=1) >= -1e-6 * (1 + d2[:, :1]))
    if math.isfinite(eps0):
        _, _, fdims = g.search(wl.Q, K, EF, eps0=math.inf, return_dims=True, n_entry=NE)
        assert dims.sum() < fdims.sum()                      # early rejections happen
    if pp and not math.isfinite(eps0):                       # HNSW++ with exact DCOs is HNSW
        h_ids, h_d2 = g.search(wl.Q, K, EF, eps0=math.inf, n_entry=NE)
        assert np.array_equal(ids, h_ids) and np.array_equal(d2, h_d2)


@pytest.mark.parametrize("pp", [False, True])
def test_graph_many_entries_match_oracle(gr, pp):
    adsx, wl, ix, g, Y, Cr, Qr, nbr, ent = gr
    g24 = adsx.build_graph(ix, wl.X, degree=32, nprobe=10, entries_per_cluster=24)
    try:
        nbr24, ent24 = adsx.graph_export(g24)
        assert np.array_equal(nbr24, nbr)                    # same kNN lists
        assert np.array_equal(ent24[:, :EPC], ent)           # sampling extends the shorter one
        ef = 48                                              # < 3 x 24 start vertices
        ids, d2, dims = g24.search(wl.Q, K, ef, eps0=2.1, delta_d=32, return_dims=True,
                                   n_entry=NE, decoupled=pp)
        probes, _ = oracle.probe(Cr, Qr, NE)
        starts = ent24[probes].reshape(len(Qr), -1)
        oids, od2, odims, _, margin = oracle.graph_search(Y, nbr24, starts, Qr, K, ef, 2.1, 32,
                                                          max_iter=4 * ef, pp=pp,
                                                          return_margin=True)
        ok = ~near_tie_queries(Cr, Qr, NE)
        _match_sequential(ids, d2, dims, Y, Qr, oids, od2, odims, margin, ok)
        # exact DCOs: every distinct start vertex costs D dims; ADSampling
        # rejects some of the later start batches early
        _, _, xdims = g24.search(wl.Q, K, ef, eps0=math.inf, return_dims=True, n_entry=NE,
                                 decoupled=pp)
        nstart = np.array([len(set(s[s >= 0].tolist())) for s in starts])
        assert np.all(xdims >= nstart * wl.D) and dims.sum() < xdims.sum()
    finally:
        g24.close()


def test_graph_argument_checks(gr):
    adsx, wl, ix, g, Y, Cr, Qr, nbr, ent = gr
    with pytest.raises(adsx.AdsxError):
        g.search(wl.Q, 65, 64)                               # K > ef
    with pytest.raises(adsx.AdsxError):
        g.search(wl.Q, 10, 10_000)                           # ef > ADSX_MAX_EF
    with pytest.raises(adsx.AdsxError):
        g.search(wl.Q, 10, 64, n_entry=17)                   # n_entry > ADSX_MAX_GRAPH_ENTRIES
    for bad in (0, 65):                                      # 1..ADSX_MAX_CLUSTER_ENTRIES
        with pytest.raises(adsx.AdsxError):
            adsx.build_graph(ix, wl.X, entries_per_cluster=bad)
    ix16 = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign, storage=adsx.BF16)
    try:
        with pytest.raises(adsx.AdsxError):
            adsx.build_graph(ix16, wl.X)
    finally:
        ix16.close()
    ixip = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign, metric=adsx.IP)
    try:
        with pytest.raises(adsx.AdsxError):
            adsx.build_graph(ixip, wl.X)
    finally:
        ixip.close()


@pytest.mark.parametrize("pp", [False, True])
def test_graph_tiny_edge_cases(pp):
    from paper_2303_09855_gb300 import adsx
    from paper_2303_09855_gb300 import workloads as W
    rng = np.random.default_rng(21)
    N, D, nlist = 20, 20, 3                               # Dp = 32; 19 others < degree 32
    X = rng.normal(size=(N, D)).astype(np.float32)
    assign = (np.arange(N) % 2).astype(np.int32)         # 10 members each, cluster 2 empty
    C = np.stack([X[assign == 0].mean(0), X[assign == 1].mean(0), X[0] + 50.0]).astype(np.float32)
    P = W.make_P(D, 22).astype(np.float32)
    ix = adsx.build_index(X, P, C, assign)
    g = adsx.build_graph(ix, X, degree=32, nprobe=3, entries_per_cluster=30)
    try:
        nbr, ent = adsx.graph_export(g)
        Y, Cr = oracle.rotate(P, X), oracle.rotate(P, C)
        assert nbr.shape == (N, 32)
        assert np.all((nbr >= 0).sum(1) == N - 1) and np.all(nbr[:, N - 1:] == -1)
        for v in range(N):
            assert sorted(nbr[v, :N - 1].tolist()) == [u for u in range(N) if u != v]
        assert ent.shape == (nlist, 30) and np.all(ent[2] == -1) and np.all(ent[:2, 10:] == -1)
        for c in range(2):                               # distinct points: every member once
            assert sorted(ent[c, :10].tolist()) == np.nonzero(assign == c)[0].tolist()
        Q = rng.normal(size=(6, D)).astype(np.float32)
        Qr = oracle.rotate(P, Q)
        K = ef = 50                                      # above N: padded results
        ids, d2 = g.search(Q, K, ef, eps0=math.inf, n_entry=3, decoupled=pp)
        probes, _ = oracle.probe(Cr, Qr, 3)
        oids, od2, _, _ = oracle.graph_search(Y, nbr, ent[probes].reshape(6, -1), Qr, K, ef,
                                              math.inf, 32, max_iter=4 * ef, pp=pp)
        assert np.array_equal(ids, oids)
        assert np.all(ids[:, N:] == -1) and np.all(np.isinf(d2[:, N:]))
        assert np.array_equal(np.sort(ids[:, :N], axis=1), np.tile(np.arange(N), (6, 1)))
        fin = ids >= 0
        assert np.allclose(d2[fin], od2[fin], rtol=1e-5, atol=1e-6)
        e_ids, e_d2 = g.search(Q[:0], 10, 16, n_entry=2)
        assert e_ids.shape == (0, 10) and e_d2.shape == (0, 10)
    finally:
        g.close()
        ix.close()


@pytest.mark.parametrize("pp", [False, True])
def test_graph_cosine_matches_oracle(gr, pp):
    adsx, wl, ix, g, Y, Cr, Qr, nbr, ent = gr
    Yn, Cn, Qn = oracle.normalize_rows(Y), oracle.normalize_rows(Cr), oracle.normalize_rows(Qr)
    ixc = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign, metric=adsx.COSINE)
    gc = adsx.build_graph(ixc, wl.X, degree=32, nprobe=10, entries_per_cluster=8)
    try:
        nbrc, entc = adsx.graph_export(gc)
        ef = 64
        ids, cs, dims = gc.search(wl.Q, K, ef, eps0=2.1, delta_d=32, return_dims=True,
                                  n_entry=NE, decoupled=pp)
        probes, _ = oracle.probe(Cn, Qn, NE)
        starts = entc[probes].reshape(len(Qn), -1)
        oids, od2, odims, _, margin = oracle.graph_search(Yn, nbrc, starts, Qn, K, ef, 2.1, 32,
                                                          max_iter=4 * ef, pp=pp,
                                                          return_margin=True)
        ok = ~near_tie_queries(Cn, Qn, NE)
        good = ok & (margin >= REL)
        for q in np.nonzero(good)[0]:
            # similarities 1 - d^2/2 against the oracle's squared distances
            assert not topk_row_mismatch(ids[q], 2.0 - 2.0 * cs[q], oids[q], od2[q]), q
            assert dims[q] == odims[q], q
        assert good.mean() >= 0.8, good.mean()
        for q in range(len(Qn)):
            row = ids[q][ids[q] >= 0]
            assert len(set(row.tolist())) == len(row)
            for i, v in zip(ids[q], cs[q]):
                if i >= 0:
                    assert abs(v - float(Yn[i] @ Qn[q])) <= 1e-5, (q, i, v)
            assert np.all(np.diff(cs[q][ids[q] >= 0]) <= 1e-6)      # largest first
    finally:
        gc.close()
        ixc.close()


def test_graph_maximum_sizes(gr):
    """ef = K = ADSX_MAX_EF, 16 start clusters x 64 entries (1024 start
    vertices, 32 start batches), exact DCOs, against the oracle on the same
    graph and starts."""
    adsx, wl, ix, g, Y, Cr, Qr, nbr, ent = gr
    g64 = adsx.build_graph(ix, wl.X, degree=32, nprobe=10, entries_per_cluster=64)
    try:
        nbr64, ent64 = adsx.graph_export(g64)
        nq = 40
        ids, d2 = g64.search(wl.Q[:nq], 512, 512, eps0=math.inf, n_entry=16)
        probes, _ = oracle.probe(Cr, Qr[:nq], 16)
        starts = ent64[probes].reshape(nq, -1)
        assert starts.shape[1] == 1024
        oids, od2, _, _, margin = oracle.graph_search(Y, nbr64, starts, Qr[:nq], 512, 512,
                                                      math.inf, 32, max_iter=4 * 512,
                                                      return_margin=True)
        ok = ~near_tie_queries(Cr, Qr[:nq], 16)
        # 512 results and hundreds of expansions: nearly every query has some
        # comparison closer than REL, so besides the exact match of the
        # queries without one, the result sets must overlap almost entirely
        _match_sequential(ids, d2, None, Y, Qr[:nq], oids, od2, None, margin, ok, min_frac=0.0)
        overlap = np.mean([len(set(ids[q].tolist()) & set(oids[q].tolist())) / 512.0
                           for q in range(nq)])
        assert overlap >= 0.99, overlap
    finally:
        g64.close()
