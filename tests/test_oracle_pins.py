"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(not against the oracle itself): brute force on tiny inputs, exact rotations,
hand-worked cases of Algorithm 1, exact reductions of IVF+ to IVF, and the
probability law of a rejection step."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2303_09855_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _f(v):
    return math.inf if v == "inf" else float(v)


# ------------------------------------------------------------ Sec. 3.1
def test_rotate_permutation_matrix_is_not_transposed():
    """A cyclic permutation P with P[i, pi(i)] = 1 must give y_i = x_pi(i);
    the transpose would give the inverse permutation."""
    D = 7
    pi = np.array([3, 0, 6, 1, 5, 2, 4])
    P = np.zeros((D, D), np.float32)
    P[np.arange(D), pi] = 1.0
    X = np.random.default_rng(0).standard_normal((5, D)).astype(np.float32)
    Y = oracle.rotate(P, X)
    assert np.array_equal(Y, X[:, pi].astype(np.float64))


def test_rotate_exact_hadamard_preserves_norms():
    """H_16 / 4 has entries +-1/4 (exact in float32) and is exactly
    orthogonal, so ||P x|| = ||x|| to FP64 rounding (Sec. 3.1: rotation
    preserves distances)."""
    H = np.array([[1.0]])
    for _ in range(4):
        H = np.block([[H, H], [H, -H]])
    P = (H / 4.0).astype(np.float32)
    X = np.random.default_rng(1).standard_normal((50, 16)).astype(np.float32)
    Y = oracle.rotate(P, X)
    n0 = (X.astype(np.float64) ** 2).sum(1)
    n1 = (Y ** 2).sum(1)
    assert np.max(np.abs(n1 - n0) / n0) < 1e-13


def test_make_P_is_orthogonal_to_1e12():
    for D in (16, 128, 960):
        P = W.make_P(D, 3)
        assert np.max(np.abs(P.T @ P - np.eye(D))) < 1e-12
        x = np.random.default_rng(D).standard_normal(D)
        assert abs(np.sum((P @ x) ** 2) - np.sum(x ** 2)) <= 1e-12 * np.sum(x ** 2)


def test_rotate_matches_haar_distance_preservation():
    wl = W.random_small(300, 32, 20, 8, seed=5)
    Y = oracle.rotate(wl.P, wl.X)
    Qr = oracle.rotate(wl.P, wl.Q)
    d_raw = ((wl.X[:, None, :].astype(np.float64) - wl.Q[None, :, :]) ** 2).sum(-1)
    d_rot = ((Y[:, None, :] - Qr[None, :, :]) ** 2).sum(-1)
    # P is float32-rounded: orthogonal to ~1e-7, distances agree to that order
    assert np.max(np.abs(d_rot - d_raw) / d_raw) < 2e-6


# ------------------------------------------------------------ Sec. 2.1 / 2.2.2
def _np_topk(d2, K):
    ids = np.lexsort((np.arange(d2.shape[0]), d2))[:K]
    return ids, d2[ids]


def test_knn_exact_matches_numpy_brute_force_with_ties():
    rng = np.random.default_rng(2)
    Y = rng.integers(0, 4, size=(400, 6)).astype(np.float64)   # many exact ties
    Qr = rng.integers(0, 4, size=(13, 6)).astype(np.float64)
    K = 17
    ids, d2 = oracle.knn_exact(Y, Qr, K)
    for q in range(Qr.shape[0]):
        dd = ((Y - Qr[q]) ** 2).sum(1)
        e_ids, e_d = _np_topk(dd, K)
        assert np.array_equal(ids[q], e_ids)
        assert np.array_equal(d2[q], e_d)


def test_knn_exact_pads_when_K_exceeds_N():
    Y = np.eye(3)
    ids, d2 = oracle.knn_exact(Y, np.zeros((1, 3)), 5)
    assert list(ids[0, :3]) == [0, 1, 2] and list(ids[0, 3:]) == [-1, -1]
    assert np.all(np.isinf(d2[0, 3:]))


def test_probe_matches_numpy_and_breaks_ties_by_cluster_id():
    Cr = np.array([[0, 0], [2, 0], [0, 2], [-2, 0], [0, -2], [5, 5]], np.float64)
    Qr = np.array([[0, 0], [1, 1]], np.float64)
    probes, pd2 = oracle.probe(Cr, Qr, 4)
    assert list(probes[0]) == [0, 1, 2, 3]          # four-way tie at 4 -> ids 1,2,3
    assert list(pd2[0]) == [0, 4, 4, 4]
    assert list(probes[1]) == [0, 1, 2, 3]          # (1,1): d=2,2,2 then a 3/4 tie at 10
    assert list(pd2[1]) == [2, 2, 2, 10]
    # recompute exactly
    for q in range(2):
        dd = ((Cr - Qr[q]) ** 2).sum(1)
        e, ed = _np_topk(dd, 4)
        assert np.array_equal(probes[q], e) and np.array_equal(pd2[q], ed)


def _np_ivf(Y, Cr, assign, Qr, K, nprobe):
    out = []
    for q in range(Qr.shape[0]):
        dc = ((Cr - Qr[q]) ** 2).sum(1)
        pr, _ = _np_topk(dc, nprobe)
        cand = np.nonzero(np.isin(assign, pr))[0]
        dd = ((Y[cand] - Qr[q]) ** 2).sum(1)
        order = np.lexsort((cand, dd))[:K]
        ids = np.full(K, -1, np.int64)
        ids[:len(order)] = cand[order]
        out.append(ids)
    return np.array(out)


def test_ivf_exact_matches_numpy_ivf_on_tiny_inputs():
    wl = W.random_small(500, 24, 30, 12, seed=9)
    Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
    for nprobe in (1, 3, 12):
        ids, _ = oracle.ivf_exact(Y, Cr, wl.assign, Qr, 10, nprobe)
        assert np.array_equal(ids, _np_ivf(Y, Cr, wl.assign, Qr, 10, nprobe))


def test_ivf_exact_with_all_clusters_is_exact_knn():
    wl = W.random_small(800, 16, 25, 10, seed=4)
    Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
    a_ids, a_d = oracle.ivf_exact(Y, Cr, wl.assign, Qr, 20, wl.nlist)
    b_ids, b_d = oracle.knn_exact(Y, Qr, 20)
    assert np.array_equal(a_ids, b_ids) and np.array_equal(a_d, b_d)


# ------------------------------------------------------------ Algorithm 1
def test_dco_hand_worked_cases():
    with open(os.path.join(GOLDEN, "dco_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        dec, dims, S, _ = oracle.dco(np.array(c["o"], float), np.array(c["q"], float),
                                     _f(c["r2"]), _f(c["eps0"]), c["delta_d"])
        assert (dec, dims, S) == (c["decision"], c["dims"], c["S"]), c["name"]


def test_dco_margin_is_the_closest_comparison_hand_worked():
    """The margin the GPU tests use to set boundary cases aside: the smallest
    |lhs / rhs - 1| over every comparison Algorithm 1 made (D S_d against
    r^2 d (1 + eps0/sqrt(d))^2 at each d < D, then S_D against r^2)."""
    q = np.zeros(4)
    o = np.array([1.0, 1.0, 1.0, 0.0])                   # S_2 = 2, S_4 = 3
    # eps0 = 0, r^2 = 5: d = 2: 8 vs 10 (0.2); d = 4: 3 vs 5 (0.4) -> 0.2
    assert oracle.dco(o, q, 5.0, 0.0, 2) == (oracle.POSITIVE, 4, 3.0, pytest.approx(0.2))
    # r^2 = 4: d = 2 sits on the boundary (8 vs 8, not rejected) -> margin 0
    assert oracle.dco(o, q, 4.0, 0.0, 2) == (oracle.POSITIVE, 4, 3.0, 0.0)
    # r^2 = 2.5: d = 2: 8 > 5, rejected there with margin 0.6
    assert oracle.dco(o, q, 2.5, 0.0, 2) == (oracle.REJECTED, 2, 2.0, pytest.approx(0.6))
    # eps0 = 1, r^2 = 5: d = 2: 8 vs 10 (1 + 1/sqrt 2)^2 = 29.14.. (0.7255..); d = 4: 0.4
    g2 = (1.0 + 1.0 / np.sqrt(2.0)) ** 2
    res, dims, S, m = oracle.dco(o, q, 5.0, 1.0, 2)
    assert (res, dims, S) == (oracle.POSITIVE, 4, 3.0)
    assert m == pytest.approx(min(abs(8.0 / (10.0 * g2) - 1.0), 0.4))
    # r^2 = 2.9: no rejection (8 vs 5.8 g2), negative at d = D: 3 vs 2.9
    res, dims, S, m = oracle.dco(o, q, 2.9, 1.0, 2)
    assert (res, dims, S) == (oracle.NEGATIVE_AT_D, 4, 3.0)
    assert m == pytest.approx(min(abs(8.0 / (5.8 * g2) - 1.0), abs(3.0 / 2.9 - 1.0)))


def test_dco_full_scan_is_exact_distance():
    rng = np.random.default_rng(3)
    o, q = rng.standard_normal(37), rng.standard_normal(37)
    dec, dims, S, _ = oracle.dco(o, q, math.inf, 2.1, 8)
    assert dec == oracle.POSITIVE and dims == 37
    assert abs(S - np.sum((o - q) ** 2)) < 1e-12 * S


def test_beta_law_of_one_rejection_step():
    """Lemma 3.1 made exact: for a Haar rotation P and fixed x with
    ||x|| = r (dis = r), S_d / ||x||^2 = ||(P x)|_d||^2 / ||x||^2 follows
    Beta(d/2, (D-d)/2).  The first test (d = delta_d) rejects iff
    S_d/||x||^2 > (d/D)(1+eps0/sqrt d)^2, so its rate must equal the
    regularised incomplete beta tail.  The rotations are applied in FP64
    (float32 rounding of P would blur the law), the oracle runs Algorithm 1,
    and the expected rate comes from scipy."""
    from scipy.special import betainc
    D, dd, n = 32, 8, 12000
    x = np.random.default_rng(11).standard_normal(D).astype(np.float32)
    r2 = float(np.sum(x.astype(np.float64) ** 2))
    rng = np.random.default_rng(12)
    Ys = np.empty((n, D))
    for i in range(n):
        G = rng.standard_normal((D, D))
        Qm, R = np.linalg.qr(G)
        P = (Qm * np.sign(np.diag(R))[None, :])
        # exact rotation in FP64 so the law is not blurred by float32 rounding
        Ys[i] = P @ x.astype(np.float64)
    zero = np.zeros(D)
    for eps0 in (0.5, 1.0, 1.5):
        first, total = 0, 0
        steps = np.zeros(D // dd)
        for i in range(n):
            dec, dims, _, _ = oracle.dco(Ys[i], zero, r2, eps0, dd)
            if dec == oracle.REJECTED:
                total += 1
                steps[dims // dd - 1] += 1
                first += dims == dd
        g2 = (1.0 + eps0 / math.sqrt(dd)) ** 2
        f = dd / D * g2
        p = 1.0 - betainc(dd / 2.0, (D - dd) / 2.0, f) if f < 1 else 0.0
        sig = math.sqrt(max(p * (1 - p), 1e-12) / n)
        assert abs(first / n - p) < 4.0 * sig + 1e-4, (eps0, first / n, p)
        # Eq. 4-6: overall failure between the largest single step and the union bound
        per_step = []
        for j in range(1, D // dd):
            d = j * dd
            fj = d / D * (1.0 + eps0 / math.sqrt(d)) ** 2
            per_step.append(1.0 - betainc(d / 2.0, (D - d) / 2.0, fj) if fj < 1 else 0.0)
        rate = total / n
        assert rate <= sum(per_step) + 4.0 * math.sqrt(sum(per_step) / n) + 1e-4
        assert rate >= max(per_step) - 4.0 * math.sqrt(max(per_step) / n) - 1e-4


# ------------------------------------------------------------ Sec. 4 IVF+
@pytest.fixture(scope="module")
def small_wl():
    wl = W.random_small(3000, 64, 40, 30, seed=21)
    Y, Cr, Qr = (oracle.rotate(wl.P, a) for a in (wl.X, wl.centroids, wl.Q))
    return wl, Y, Cr, Qr


def test_ivf_ads_visit_order_hand_worked():
    """Sequential IVF+ visits clusters by (centroid distance, id) and members
    by ascending id; r^2 tightens along that order, so the dims it samples
    pin the order.  eps0 = 0 (reject at d iff (D/d) S_d > r^2), K = 1, q = 0."""
    q = np.zeros((1, 4))
    # A: cluster 0 (nearer centroid) holds id 0 at distance 1; cluster 1 holds
    # id 1 (S_2 = 4, distance 4) and id 2 (distance 0.25).  Cluster 0 first:
    # id 0 exact (4 dims, r^2 = 1), id 1 rejected at d = 2, id 2 exact -> 10.
    # (Cluster 1 first would sample 4 + 4 + 4 = 12.)
    Y = np.array([[0, 0, 0, 1.0], [2.0, 0, 0, 0], [0, 0, 0, 0.5]])
    C = np.array([[0, 0, 0, 0.9], [1.0, 0, 0, 0.3]])
    ids, d2, dims, ncand = oracle.ivf_ads(Y, C, np.array([0, 1, 1]), q, 1, 2, 0.0, 2)
    assert ids[0, 0] == 2 and d2[0, 0] == 0.25 and ncand[0] == 3 and dims[0] == 10
    # B: one cluster, id 0 at distance 0.25, id 1 with S_2 = 0.36 (distance
    # 0.36).  Ascending ids: id 0 exact (r^2 = 0.25), id 1 rejected at d = 2
    # (2 x 0.36 > 0.25) -> 6 dims.  (Id 1 first would sample 8.)
    Y = np.array([[0, 0, 0, 0.5], [0.6, 0, 0, 0]])
    ids, d2, dims, ncand = oracle.ivf_ads(Y, np.zeros((1, 4)), np.array([0, 0]), q, 1, 1, 0.0, 2)
    assert ids[0, 0] == 0 and dims[0] == 6


def test_ivf_ads_with_infinite_eps0_is_ivf(small_wl):
    wl, Y, Cr, Qr = small_wl
    e_ids, e_d = oracle.ivf_exact(Y, Cr, wl.assign, Qr, 10, 6)
    for eps0, dd in ((math.inf, 16), (math.inf, 1), (2.1, 64), (0.5, 1000)):
        ids, d2, dims, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, 10, 6, eps0, dd)
        assert np.array_equal(ids, e_ids) and np.array_equal(d2, e_d), (eps0, dd)
        assert np.array_equal(dims, ncand * 64)


def test_ivf_ads_all_candidates_when_K_is_large(small_wl):
    """r stays +inf while the KNN set is not full (Sec. 2.2.2), so with K at
    least the number of candidates nothing is rejected."""
    wl, Y, Cr, Qr = small_wl
    ids, d2, dims, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, 3000, 2, 0.1, 16)
    e_ids, e_d = oracle.ivf_exact(Y, Cr, wl.assign, Qr, 3000, 2)
    assert np.array_equal(ids, e_ids) and np.array_equal(dims, ncand * 64)


def test_ivf_ads_returns_only_exact_distances_and_brackets_ivf(small_wl):
    """No false positives (Lemma 3.2: failure prob 0 if dis > r) and the
    bracket: every true IVF top-K member whose DCO at r* (the exact K-th
    candidate distance) is not rejected must be returned, for any visit
    order, because the live r is always >= r* (Sec. 4 corollaries)."""
    wl, Y, Cr, Qr = small_wl
    K, nprobe = 10, 6
    e_ids, e_d = oracle.ivf_exact(Y, Cr, wl.assign, Qr, K, nprobe)
    for eps0 in (0.3, 1.0, 2.1):
        ids, d2, _, _ = oracle.ivf_ads(Y, Cr, wl.assign, Qr, K, nprobe, eps0, 16)
        for q in range(Qr.shape[0]):
            for i, d in zip(ids[q], d2[q]):
                if i >= 0:
                    exact = np.sum((Y[i] - Qr[q]) ** 2)
                    assert abs(d - exact) <= 1e-12 * exact
            rstar = e_d[q, K - 1]
            dec, _, _ = oracle.dco_fixed_r(Y[e_ids[q]], Qr[q:q + 1], np.array([rstar]), eps0, 16)
            must = set(e_ids[q][dec[0] == oracle.POSITIVE])
            assert must <= set(ids[q]), (eps0, q)


def test_fixed_r_rejections_are_nested_in_r_and_eps0(small_wl):
    wl, Y, Cr, Qr = small_wl
    Qs = Qr[:8]
    _, kd = oracle.knn_exact(Y, Qs, 10)
    base = kd[:, -1]
    prev = None
    for s in (0.8, 1.0, 1.3):
        dec, _, _ = oracle.dco_fixed_r(Y, Qs, base * s, 1.5, 16)
        rej = dec == oracle.REJECTED
        if prev is not None:
            assert np.all(rej <= prev)          # rejected set shrinks as r grows
        prev = rej
    prev = None
    for eps0 in (0.5, 1.0, 2.0, 3.0):
        dec, _, _ = oracle.dco_fixed_r(Y, Qs, base, eps0, 16)
        rej = dec == oracle.REJECTED
        if prev is not None:
            assert np.all(rej <= prev)          # and as eps0 grows
        prev = rej


def test_lemma_3_2_and_3_3_trends():
    """Sec. 6.2.5 protocol: linear scan, fixed r = exact K-th NN distance,
    delta_d = 1.  Failure rate on positives falls quadratic-exponentially in
    eps0 (Lemma 3.2: log-failure against eps0^2 has a negative slope), and
    the dims sampled on negatives fall as the gap alpha grows (Lemma 3.3)."""
    wl = W.random_small(2000, 96, 24, 10, seed=31, spread=1.0)
    Y, Qr = oracle.rotate(wl.P, wl.X), oracle.rotate(wl.P, wl.Q)
    K = 20
    _, kd = oracle.knn_exact(Y, Qr, K)
    r2 = kd[:, -1]
    d_all = ((Y[None, :, :] - Qr[:, None, :]) ** 2).sum(-1)
    near = np.abs(d_all - r2[:, None]) <= 1e-12 * r2[:, None]   # summation-order ulps
    pos = (d_all <= r2[:, None]) & ~near
    neg = (d_all > r2[:, None]) & ~near
    eps_grid = [0.5, 1.0, 1.5, 2.0, 2.5]
    fails = []
    for eps0 in eps_grid:
        dec, dims, _ = oracle.dco_fixed_r(Y, Qr, r2, eps0, 1)
        fails.append(np.mean(dec[pos] == oracle.REJECTED))
        assert np.all(dec[neg] != oracle.POSITIVE)     # negatives never fail
        if eps0 == 2.0:
            alpha = np.sqrt(d_all[neg]) / np.sqrt(np.repeat(r2[:, None], Y.shape[0], 1)[neg]) - 1
            dn = dims[neg]
            lo = dn[alpha < np.quantile(alpha, 0.2)].mean()
            hi = dn[alpha > np.quantile(alpha, 0.8)].mean()
            assert lo > hi
            assert np.mean(dn) < 0.4 * 96
    fails = np.array(fails)
    assert np.all(np.diff(fails) <= 0)
    assert fails[0] > 0.05 and fails[-1] < 0.01
    ok = fails > 0
    slope = np.polyfit(np.square(eps_grid)[ok], np.log(fails[ok]), 1)[0]
    assert slope < 0


def test_recall_and_ratio_metrics():
    assert oracle.recall_at([[1, 2, 3]], [[3, 2, 9]], 3) == pytest.approx(2 / 3)
    assert oracle.recall_at([[1, -1, -1]], [[1, 2, 3]], 3) == pytest.approx(1 / 3)
    assert oracle.avg_dist_ratio([[4.0, 16.0]], [[1.0, 16.0]]) == pytest.approx(1.5)


# ------------------------------------------------------------ Sec. 6.1 PDScanning
def test_pdscanning_hand_cases_and_exactness(small_wl):
    """PDScanning stops when the partial squared distance exceeds r^2
    (strictly): o - q = (2, 1, 1, 0), delta_d 1, r2 = 4: S_1 = 4 (not > 4),
    S_2 = 5 > 4 -> stopped with 2 dims; r2 = 6: S = 4, 5, 6, 6 -> positive."""
    o, q = np.array([2.0, 1, 1, 0]), np.zeros(4)
    assert oracle.dco_pd(o, q, 4.0, 1)[:2] == (oracle.REJECTED, 2)
    assert oracle.dco_pd(o, q, 6.0, 1)[:2] == (oracle.POSITIVE, 4)
    assert oracle.dco_pd(o, q, 5.5, 2)[:2] == (oracle.NEGATIVE_AT_D, 4)
    wl, Y, Cr, Qr = small_wl
    e_ids, e_d = oracle.ivf_exact(Y, Cr, wl.assign, Qr, 10, 6)
    ids, d2, dims = oracle.ivf_pd(Y, Cr, wl.assign, Qr, 10, 6, 16)
    assert np.array_equal(ids, e_ids) and np.array_equal(d2, e_d)   # exact DCO
    _, _, full, ncand = oracle.ivf_ads(Y, Cr, wl.assign, Qr, 10, 6, math.inf, 16)
    assert np.all(dims <= full) and np.any(dims < full)
