"""CPU checks of the seeded synthetic inputs (the stand-ins for the paper's
datasets): each generator is deterministic in its seeds, gives the shapes,
value ranges and structure its recipe states, and its k-means assignment is
the nearest-centroid one (ties to the lower id).  Small sizes only."""
import numpy as np
import pytest

from paper_2303_09855_gb300 import workloads as W


def _same(a, b):
    return (np.array_equal(a.X, b.X) and np.array_equal(a.Q, b.Q) and np.array_equal(a.P, b.P)
            and np.array_equal(a.centroids, b.centroids) and np.array_equal(a.assign, b.assign))


def _nearest_centroid_assignment(wl):
    X = wl.X.astype(np.float64)
    C = wl.centroids.astype(np.float64)
    d = (C * C).sum(1)[None, :] - 2.0 * X @ C.T
    best = d.min(axis=1, keepdims=True)
    # FP32 k-means may settle a near-tie either way: only clear winners are checked
    clear = np.sort(d, axis=1)[:, 1] - best[:, 0] > 1e-3 * (1.0 + np.abs(best[:, 0]))
    return np.all(wl.assign[clear] == np.argmin(d, axis=1)[clear])


def test_gaussian_mixture_shapes_determinism_and_assignment():
    a = W.gen_gaussian_mixture(N=1500, D=24, nq=20, ncomp=6, nlist=8, kmeans_iters=3)
    b = W.gen_gaussian_mixture(N=1500, D=24, nq=20, ncomp=6, nlist=8, kmeans_iters=3)
    assert _same(a, b)
    assert a.X.shape == (1500, 24) and a.Q.shape == (20, 24) and a.P.shape == (24, 24)
    assert a.centroids.shape == (8, 24) and a.assign.shape == (1500,)
    assert a.X.dtype == np.float32 and a.assign.dtype == np.int32
    assert a.assign.min() >= 0 and a.assign.max() < 8
    assert _nearest_centroid_assignment(a)
    c = W.gen_gaussian_mixture(N=1500, D=24, nq=20, ncomp=6, nlist=8, kmeans_iters=3, cfg=5)
    assert not np.array_equal(a.X, c.X)                  # another config, other seeds


def test_sift_like_is_integer_valued_in_0_255_and_sparse_centred():
    wl = W.gen_sift_like(N=3000, nq=30, ncomp=16, nlist=12, kmeans_iters=2)
    assert wl.X.shape == (3000, 128)
    for A in (wl.X, wl.Q):
        assert A.min() >= 0.0 and A.max() <= 255.0
        assert np.array_equal(A, np.rint(A))
    # a quarter of the centre dims are active: many coordinates sit at the clip
    assert 0.05 < np.mean(wl.X == 0.0) < 0.9
    assert _nearest_centroid_assignment(wl)


def test_gist_like_lies_in_the_unit_interval():
    wl = W.gen_gist_like(N=1200, D=96, nq=10, ncomp=8, nlist=8, rank=8, kmeans_iters=2)
    assert wl.X.shape == (1200, 96) and wl.Q.shape == (10, 96)
    assert wl.X.min() > 0.0 and wl.X.max() < 1.0
    # correlated dims through the shared low-rank factor: the leading
    # principal component of within-data covariance dominates a white one
    Xc = wl.X - wl.X.mean(0)
    ev = np.linalg.eigvalsh(np.cov(Xc.T))
    assert ev[-1] > 5 * np.median(ev)


def test_uneven_per_query_K_and_nprobe_ranges():
    wl = W.gen_uneven(N=4000, D=32, nq=400, ncomp=50, nlist=40, kmeans_iters=2)
    K, npb = wl.params["K"], wl.params["nprobe"]
    assert set(np.unique(K).tolist()) <= {1, 10, 100} and len(np.unique(K)) == 3
    assert npb.min() >= 8 and npb.max() <= 512
    # log-uniform: about as many below 64 (the geometric midpoint) as above
    assert 0.35 < np.mean(npb < 64) < 0.65
    assert _nearest_centroid_assignment(wl)


def test_serving_rows_are_unit_norm_with_nprobe_choices():
    wl = W.gen_serving(N=3000, D=96, nq=300, ncomp=20, nlist=16, kmeans_iters=2)
    assert np.allclose(np.linalg.norm(wl.X, axis=1), 1.0, atol=1e-5)
    assert np.allclose(np.linalg.norm(wl.Q, axis=1), 1.0, atol=1e-5)
    assert set(np.unique(wl.params["nprobe"]).tolist()) == {16, 32, 64}


def test_kac_walk_layers_are_disjoint_rotations():
    pairs, cs = W.make_kac_walk(37, 9, 4)
    assert pairs.shape == cs.shape == (9, 36)
    for l in range(9):
        assert len(set(pairs[l].tolist())) == 36 and pairs[l].min() >= 0 and pairs[l].max() < 37
        c, s = cs[l, 0::2].astype(np.float64), cs[l, 1::2].astype(np.float64)
        assert np.allclose(c * c + s * s, 1.0, atol=1e-6)
    p2, c2 = W.make_kac_walk(37, 9, 4)
    assert np.array_equal(pairs, p2) and np.array_equal(cs, c2)


@pytest.mark.parametrize("D", [1, 5, 64])
def test_make_P_is_the_positive_diagonal_QR_factor_of_its_gaussian_draw(D):
    """P is the unique Q of G = Q R with diag(R) > 0 (the Haar convention):
    then P^T G is upper triangular with a positive diagonal."""
    P = W.make_P(D, 3)
    G = np.random.default_rng(3).standard_normal((D, D))
    T = P.T @ G
    assert np.allclose(P.T @ P, np.eye(D), atol=1e-12)
    assert np.allclose(np.tril(T, -1), 0.0, atol=1e-10)
    assert np.all(np.diag(T) > 0)
