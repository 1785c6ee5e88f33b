"""Pins of the oracle's Kac-walk rotation (Sec. 6.2.3: the random rotation in
O(D log D) by Kac's walk instead of a dense matrix product):

  - a hand-worked layer (a quarter turn on one pair, identity on the other);
  - layers apply in order (two layers equal the second applied to the
    first's output);
  - with D odd, the coordinate a layer leaves unpaired passes through it
    unchanged, and each pair's 2-vector keeps its length;
  - the walk is orthogonal to within the rounding of its FP32 cosines and
    sines, and the dense matrix equals the walk applied to each vector;
  - after 3 log2(D) layers the walk mixes like a Haar rotation for the
    statistic ADSampling relies on (Lemma 3.1): the squared mass that a unit
    basis vector puts on the first d coordinates has the Beta(d/2, (D-d)/2)
    mean d/D and variance 2 d (D-d) / (D^2 (D+2)), within sampling error.
"""
import numpy as np

import oracle
from paper_2303_09855_gb300 import workloads as W


def test_hand_worked_layer():
    pairs = np.array([[0, 1, 2, 3]], np.int32)
    cs = np.array([[0.0, 1.0, 1.0, 0.0]], np.float32)   # (0,1): 90 degrees, (2,3): 0 degrees
    y = oracle.kac_apply(pairs, cs, np.array([[1.0, 2.0, 3.0, 4.0]]))
    assert np.array_equal(y, [[-2.0, 1.0, 3.0, 4.0]])
    # the pair order matters: (i, j) = (1, 0) gives y1 = -x0, y0 = x1
    y2 = oracle.kac_apply(np.array([[1, 0, 2, 3]], np.int32), cs, np.array([[1.0, 2.0, 3.0, 4.0]]))
    assert np.array_equal(y2, [[2.0, -1.0, 3.0, 4.0]])


def test_layers_apply_in_order():
    pairs, cs = W.make_kac_walk(10, 2, 5)
    X = np.random.default_rng(0).normal(size=(3, 10))
    both = oracle.kac_apply(pairs, cs, X)
    one_then_two = oracle.kac_apply(pairs[1:], cs[1:], oracle.kac_apply(pairs[:1], cs[:1], X))
    assert np.allclose(both, one_then_two, atol=0, rtol=0)
    other_order = oracle.kac_apply(pairs[:1], cs[:1], oracle.kac_apply(pairs[1:], cs[1:], X))
    assert not np.allclose(both, other_order)


def test_odd_dimension_rests_one_coordinate_per_layer():
    D = 9
    pairs, cs = W.make_kac_walk(D, 5, 8)
    X = np.random.default_rng(1).normal(size=(4, D))
    for l in range(5):
        y = oracle.kac_apply(pairs[l:l + 1], cs[l:l + 1], X)
        rest = sorted(set(range(D)) - set(pairs[l].tolist()))
        assert len(rest) == 1
        assert np.array_equal(y[:, rest[0]], X[:, rest[0]])
        for t in range(D // 2):
            i, j = pairs[l, 2 * t], pairs[l, 2 * t + 1]
            assert np.allclose(y[:, i] ** 2 + y[:, j] ** 2, X[:, i] ** 2 + X[:, j] ** 2,
                               rtol=1e-6)


def test_walk_is_orthogonal_and_matrix_matches():
    for D, L in ((16, 8), (37, 12), (128, 14)):
        pairs, cs = W.make_kac_walk(D, L, 7)
        Wm = oracle.kac_matrix(pairs, cs, D)
        err = np.max(np.abs(Wm.T @ Wm - np.eye(D)))
        assert err <= L * 2.5e-7, (D, err)
        X = np.random.default_rng(1).normal(size=(5, D))
        assert np.allclose(oracle.kac_apply(pairs, cs, X), X @ Wm.T, rtol=1e-12, atol=1e-12)


def test_walk_mixes_like_haar_for_the_sampled_mass():
    D, L, n = 64, 18, 3000
    d = 16
    mass = np.empty(n)
    for k in range(n):
        pairs, cs = W.make_kac_walk(D, L, 1000 + k)
        e = np.zeros((1, D))
        e[0, k % D] = 1.0
        y = oracle.kac_apply(pairs, cs, e)[0]
        mass[k] = np.sum(y[:d] ** 2)
    mean, var = d / D, 2.0 * d * (D - d) / (D * D * (D + 2))
    assert abs(mass.mean() - mean) <= 4.0 * np.sqrt(var / n), (mass.mean(), mean)
    assert 0.8 <= mass.var() / var <= 1.25, (mass.var(), var)
