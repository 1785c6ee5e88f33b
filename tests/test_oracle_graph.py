"""Pins of the oracle's greedy beam search with ADSampling DCOs (HNSW+, the
base-layer search of Sec. 2.2.1 with Algorithm 1 as its DCO, Sec. 4):

  - a hand-worked chain graph (points on a line, ef = 1) walks greedily to
    the nearest point and stops there; with two start vertices it keeps the
    nearer one;
  - on a complete graph one expansion sees every vertex, so the result is the
    exact KNN (brute force) for any ef >= K;
  - eps0 = inf and delta_d >= D give identical results (exact DCOs);
  - with ADSampling every returned distance is the exact distance of that id
    and the result has no duplicates;
  - the start vertices per cluster (farthest-point sampling): a hand-worked
    line example whose third step tells the min-distance rule from a
    max-distance one, duplicates and empty clusters, every member chosen once
    when E reaches the cluster size, and the 2-approximation bound of greedy
    k-center against brute force over all E-subsets;
  - a cluster holding two blobs that no kNN edge joins: one entry reaches one
    blob only, two entries give the exact KNN;
  - vertices are tested one at a time in the paper's order: a hand-worked
    start list where the third vertex is rejected early only because the
    second has already tightened R (sequential dims 208 against 256 for a
    threshold fixed at the start), and the closest-call margin the oracle
    reports;
  - HNSW++ (Sec. 5.1) on a hand-worked graph: rejected vertices enter the
    beam by their observed distance (D/d) S_d, which decides which branch is
    expanded (result, expansions and dims fixed by hand), where HNSW+ on the
    same graph takes the other branch.
"""
import itertools
import math

import numpy as np

import oracle


def test_chain_graph_greedy_walk():
    N = 20
    Y = np.arange(N, dtype=np.float64)[:, None]            # points 0, 1, ..., 19 on a line
    graph = np.full((N, 2), -1, np.int32)
    for i in range(N):
        graph[i, 0] = i - 1 if i > 0 else -1
        graph[i, 1] = i + 1 if i < N - 1 else -1
    Q = np.array([[10.3], [0.2], [25.0]])
    ids, d2, dims, iters = oracle.graph_search(Y, graph, np.zeros(3, np.int64), Q, 1, 1,
                                               math.inf, 16, max_iter=100)
    assert ids[:, 0].tolist() == [10, 0, 19]
    assert np.allclose(d2[:, 0], [0.3 ** 2, 0.2 ** 2, 36.0])
    # ef = 1 expands exactly the vertices on the walk 0 -> 1 -> ... -> 10
    assert iters[0] == 11 and iters[1] == 1 and iters[2] == 20
    # several start vertices: R starts as the ef nearest of them (here 19 of
    # {0, 19}); 19's other neighbour 18 is farther, so one expansion ends it
    ids, _, _, iters = oracle.graph_search(Y, graph, np.array([[0, 19]], np.int64),
                                           np.array([[18.6]]), 1, 1, math.inf, 16)
    assert ids[0, 0] == 19 and iters[0] == 1
    # the expansion cap stops the walk where it is (default 16 ef = 16 here)
    ids, _, _, iters = oracle.graph_search(Y, graph, np.zeros(1, np.int64), Q[2:], 1, 1,
                                           math.inf, 16)
    assert ids[0, 0] == 16 and iters[0] == 16


def test_complete_graph_is_exact_knn():
    rng = np.random.default_rng(3)
    N, D = 300, 12
    Y = rng.normal(size=(N, D))
    Q = rng.normal(size=(7, D))
    graph = np.array([[j for j in range(N) if j != i] for i in range(N)], np.int32)
    eids, ed2 = oracle.knn_exact(Y, Q, 10)
    for ef in (10, 25):
        ids, d2, _, _ = oracle.graph_search(Y, graph, np.arange(7, dtype=np.int64), Q, 10, ef,
                                            math.inf, 4)
        assert np.array_equal(ids, eids) and np.allclose(d2, ed2, rtol=1e-12)


def _knn_graph(Y, R):
    ids, _ = oracle.knn_exact(Y, Y, R + 1)
    return np.array([[j for j in row if j != i][:R] for i, row in enumerate(ids)], np.int32)


def test_exact_modes_agree_and_adsampling_is_exact():
    rng = np.random.default_rng(4)
    N, D = 2000, 32
    C = rng.normal(0, 3, size=(20, D))
    Y = C[rng.integers(0, 20, N)] + rng.normal(size=(N, D))
    Q = C[rng.integers(0, 20, 15)] + rng.normal(size=(15, D))
    graph = _knn_graph(Y, 12)
    ent = np.zeros(15, np.int64)
    a = oracle.graph_search(Y, graph, ent, Q, 10, 40, math.inf, 8)
    b = oracle.graph_search(Y, graph, ent, Q, 10, 40, 2.1, 32)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ids, d2, dims, iters = oracle.graph_search(Y, graph, ent, Q, 10, 40, 1.0, 8)
    assert dims.sum() < a[2].sum()                             # early rejections happen
    for q in range(15):
        row = ids[q][ids[q] >= 0]
        assert len(set(row.tolist())) == len(row)
        for i, d in zip(ids[q], d2[q]):
            if i >= 0:
                assert abs(d - float(np.sum((Y[i] - Q[q]) ** 2))) <= 1e-12 * (1 + d)


def test_hnsw_pp_reduces_to_hnsw_and_samples_fewer_dims():
    """Sec. 5.1 (HNSW++): with exact DCOs every observed distance is exact, so
    the beam evolves exactly as HNSW's and R1 is its first K: identical
    results.  With ADSampling, R1's K-th distance is a tighter threshold than
    the beam's N_ef-th, so fewer dimensions are sampled than by HNSW+;
    returned distances stay exact and distinct."""
    rng = np.random.default_rng(5)
    N, D = 2000, 32
    C = rng.normal(0, 3, size=(20, D))
    Y = C[rng.integers(0, 20, N)] + rng.normal(size=(N, D))
    Q = C[rng.integers(0, 20, 15)] + rng.normal(size=(15, D))
    graph = _knn_graph(Y, 12)
    ent = np.stack([np.zeros(15, np.int64), np.full(15, 7, np.int64)], axis=1)
    a = oracle.graph_search(Y, graph, ent, Q, 10, 40, math.inf, 8)
    b = oracle.graph_search(Y, graph, ent, Q, 10, 40, math.inf, 8, pp=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])
    plus = oracle.graph_search(Y, graph, ent, Q, 10, 40, 2.1, 8)
    ids, d2, dims, _ = oracle.graph_search(Y, graph, ent, Q, 10, 40, 2.1, 8, pp=True)
    assert dims.sum() < plus[2].sum()
    for q in range(15):
        row = ids[q][ids[q] >= 0]
        assert len(set(row.tolist())) == len(row)
        for i, d in zip(ids[q], d2[q]):
            if i >= 0:
                assert abs(d - float(np.sum((Y[i] - Q[q]) ** 2))) <= 1e-12 * (1 + d)


def test_cluster_entries_hand_worked_line():
    # members of cluster 0 at 0, 4, 5, 10, 11 (ids 0..4), centroid at 5.9:
    # entry 0 = 5 (id 2); farthest from it 11 (id 4); then 0 (id 0, at 5 from
    # {5, 11}); then 4 and 10 both sit at 1 from the chosen set: the tie goes
    # to id 1 (with max instead of min distances it would be 10, id 3); last
    # id 3; nothing is left for the sixth entry.
    Y = np.array([0.0, 4.0, 5.0, 10.0, 11.0, 3.0])[:, None]
    assign = np.array([0, 0, 0, 0, 0, 1])
    Cr = np.array([[5.9], [100.0]])
    ent = oracle.cluster_entries(Y, Cr, assign, 6)
    assert ent[0].tolist() == [2, 4, 0, 1, 3, -1]
    assert ent[1].tolist() == [5, -1, -1, -1, -1, -1]
    assert oracle.cluster_entries(Y, Cr, assign, 1).tolist() == [[2], [5]]


def test_cluster_entries_duplicates_empty_and_full():
    Y = np.zeros((4, 3))
    Y[3] = 1.0
    assign = np.array([1, 1, 1, 2])                      # cluster 0 empty
    ent = oracle.cluster_entries(Y, np.zeros((3, 3)), assign, 3)
    assert ent[0].tolist() == [-1, -1, -1]
    assert ent[1].tolist() == [0, -1, -1]                # three equal points: lowest id, then none
    assert ent[2].tolist() == [3, -1, -1]
    rng = np.random.default_rng(11)
    Y = rng.normal(size=(12, 5))
    ent = oracle.cluster_entries(Y, Y.mean(0, keepdims=True), np.zeros(12, int), 12)
    assert sorted(ent[0].tolist()) == list(range(12))


def test_cluster_entries_greedy_k_center_bound():
    """Farthest-point sampling is greedy k-center: its covering radius
    max_m min_e ||y_m - y_e|| is at most twice the best over all E-subsets."""
    rng = np.random.default_rng(12)
    for trial in range(6):
        n, E = 10, 3
        Y = rng.normal(size=(n, 4)) * rng.uniform(0.5, 3.0, size=4)
        ent = oracle.cluster_entries(Y, rng.normal(size=(1, 4)), np.zeros(n, int), E)[0]
        dist = np.sqrt(np.sum((Y[:, None, :] - Y[None, :, :]) ** 2, axis=2))
        greedy = dist[:, ent].min(axis=1).max()
        best = min(dist[:, list(sub)].min(axis=1).max() for sub in itertools.combinations(range(n), E))
        assert best <= greedy <= 2 * best + 1e-12, (trial, greedy, best)
        # each step takes a point at the largest distance from the earlier ones
        for e in range(1, E):
            nearest = dist[:, ent[:e]].min(axis=1) ** 2
            assert nearest[ent[e]] == nearest.max()


def test_two_blobs_in_one_cluster_need_two_entries():
    rng = np.random.default_rng(13)
    D = 8
    a = rng.normal(size=(60, D))
    b = rng.normal(size=(60, D)) + 40.0                   # far apart: no kNN edge between them
    Y = np.concatenate([a, b])
    assign = np.zeros(120, int)                           # one cluster holds both
    Cr = Y.mean(0, keepdims=True)
    graph = _knn_graph(Y, 8)
    assert not np.any((graph[:60] >= 60)) and not np.any((graph[60:] < 60))
    Q = np.concatenate([a[:3] + 0.1, b[:3] + 0.1])
    gt, gd = oracle.knn_exact(Y, Q, 5)
    one = oracle.cluster_entries(Y, Cr, assign, 1)
    two = oracle.cluster_entries(Y, Cr, assign, 2)
    assert (one[0, 0] < 60) != (two[0, 1] < 60)          # the second entry is in the other blob
    ids1, _, _, _ = oracle.graph_search(Y, graph, np.repeat(one, 6, axis=0), Q, 5, 20, math.inf, 8)
    ids2, d2, _, _ = oracle.graph_search(Y, graph, np.repeat(two, 6, axis=0), Q, 5, 20, math.inf, 8)
    assert oracle.recall_at(ids1, gt, 5) == 0.5
    assert np.array_equal(ids2, gt) and np.allclose(d2, gd, rtol=1e-12)


def test_vertices_are_tested_one_at_a_time_hand_worked():
    """The paper's order (Sec. 2.2.1): each vertex's DCO faces R's largest
    distance as it stands after the vertices before it.  q = 0, D = 64,
    delta_d = 16, eps0 = 0 (a DCO rejects at d < D iff (D/d) S_d > r^2),
    K = ef = 1, four start vertices and no edges:
      v0  distance^2 4, R empty (r = inf): exact, 64 dims, R = {v0};
      v1  distance^2 1 against r^2 = 4: S_d = 0 until d = 64, positive,
          64 dims, R = {v1};
      v2  S_16 = 0.5 (distance^2 1) against r^2 = 1: 4 x 0.5 = 2 > 1,
          rejected at d = 16 (16 dims) -- had the four been tested against the
          threshold at the start (r = inf) it would cost 64;
      v3  distance^2 0.81 against r^2 = 1: positive, 64 dims, R = {v3}.
    Result v3, 208 dims, one expansion (v3, no neighbours); with exact DCOs
    4 x 64 dims.  HNSW++ gives the same (R1 = R here)."""
    D = 64
    Y = np.zeros((4, D))
    Y[0, 63] = 2.0
    Y[1, 63] = 1.0
    Y[2, 0], Y[2, 63] = np.sqrt(0.5), np.sqrt(0.5)
    Y[3, 63] = 0.9
    graph = np.full((4, 1), -1, np.int32)
    starts = np.arange(4, dtype=np.int64)[None, :]
    q = np.zeros((1, D))
    for pp in (False, True):
        ids, d2, dims, iters = oracle.graph_search(Y, graph, starts, q, 1, 1, 0.0, 16, pp=pp)
        assert ids[0].tolist() == [3] and abs(d2[0, 0] - 0.81) < 1e-12
        assert dims[0] == 64 + 64 + 16 + 64 and iters[0] == 1
        _, _, dims_exact, _ = oracle.graph_search(Y, graph, starts, q, 1, 1, math.inf, 16, pp=pp)
        assert dims_exact[0] == 4 * D
    # with exact DCOs R is the ef nearest of all starts, whatever their order
    rng = np.random.default_rng(14)
    Yr = rng.normal(size=(40, 16))
    qr = rng.normal(size=(1, 16))
    g0 = np.full((40, 1), -1, np.int32)
    st = np.arange(40, dtype=np.int64)[None, :]
    a = oracle.graph_search(Yr, g0, st, qr, 5, 5, math.inf, 16)
    b = oracle.graph_search(Yr, g0, st[:, ::-1].copy(), qr, 5, 5, math.inf, 16)
    order = np.argsort(np.sum((Yr - qr) ** 2, axis=1))[:5]
    assert np.array_equal(a[0][0], order) and np.array_equal(b[0][0], order)


def test_closest_call_margin():
    """The margin the oracle reports per query is the smallest relative gap of
    any comparison that steered the search: with exact DCOs and ef = 1, start
    vertices at squared distances 1 and 1 + 1e-7 give about 1e-7 (the second
    DCO's S_D against r^2 = 1); 1 and 2 give |2/1 - 1| = 1."""
    D = 8
    for d_b, want in ((1.0 + 1e-7, 1e-7), (2.0, 1.0)):
        Y = np.zeros((2, D))
        Y[0, 0] = 1.0
        Y[1, 0] = np.sqrt(d_b)
        *_, margin = oracle.graph_search(Y, np.full((2, 1), -1, np.int32),
                                         np.array([[0, 1]], np.int64), np.zeros((1, D)), 1, 1,
                                         math.inf, 8, return_margin=True)
        assert abs(margin[0] - want) <= 1e-3 * want


def test_hnsw_pp_beam_keeps_observed_distances_hand_worked():
    """Sec. 5.1 on a hand-worked graph (q = 0, D = 64, delta_d = 16, eps0 = 0,
    so a DCO rejects at d iff (D/d) S_d > r^2; K = 1, ef = 2).  The start a
    (distance 1) fills R1, r^2 = 1.  a's neighbours: v1 has S_16 = 0.3, rejected
    at d = 16, observed distance 4 x 0.3 = 1.2; v2 has S_16 = 0.1, S_32 = 0.55,
    rejected at d = 32, observed 2 x 0.55 = 1.1.  Both enter the beam by their
    observed distances, which keeps a and v2 (ef = 2).  Expanding v2 finds w2
    (0.5 < r^2: exact, into R1); w1 behind v1 is never visited.  Expansions:
    a, v2, w2; dims 64 (a) + 16 (v1) + 32 (v2) + 64 (w2)."""
    D = 64
    Y = np.zeros((5, D))
    Y[0, 63] = 1.0                                        # a: distance^2 1
    Y[1, 0], Y[1, 63] = np.sqrt(0.3), np.sqrt(1.7)        # v1: S_16 = 0.3, total 2
    Y[2, 0], Y[2, 16], Y[2, 63] = np.sqrt(0.1), np.sqrt(0.45), np.sqrt(1.45)   # v2
    Y[3, 62] = np.sqrt(0.9)                               # w1 (behind v1)
    Y[4, 62] = np.sqrt(0.5)                               # w2 (behind v2)
    graph = np.full((5, 2), -1, np.int32)
    graph[0] = [1, 2]
    graph[1, 0] = 3
    graph[2, 0] = 4
    q = np.zeros((1, D))
    ids, d2, dims, iters = oracle.graph_search(Y, graph, np.zeros(1, np.int64), q, 1, 2, 0.0, 16,
                                               pp=True)
    assert ids[0].tolist() == [4] and abs(d2[0, 0] - 0.5) < 1e-12
    assert iters[0] == 3 and dims[0] == 64 + 16 + 32 + 64
    # HNSW+ on the same graph: R is not full while a's neighbours are tested
    # (r = +inf), so v1 and v2 get exact distances 2 and the beam {a, v1}
    # (ties by id) expands v1 and finds w1 (0.9 < 1); w2 is never reached.
    ids, d2, dims, iters = oracle.graph_search(Y, graph, np.zeros(1, np.int64), q, 1, 2, 0.0, 16)
    assert ids[0].tolist() == [3] and abs(d2[0, 0] - 0.9) < 1e-12
