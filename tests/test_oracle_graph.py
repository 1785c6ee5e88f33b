"""Pins of the oracle's greedy beam search with ADSampling DCOs (HNSW+, the
base-layer search of Sec. 2.2.1 with Algorithm 1 as its DCO, Sec. 4):

  - a hand-worked chain graph (points on a line, ef = 1) walks greedily to
    the nearest point and stops there; with two start vertices it keeps the
    nearer one;
  - on a complete graph one expansion sees every vertex, so the result is the
    exact KNN (brute force) for any ef >= K;
  - eps0 = inf and delta_d >= D give identical results (exact DCOs);
  - with ADSampling every returned distance is the exact distance of that id
    and the result has no duplicates.
"""
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
