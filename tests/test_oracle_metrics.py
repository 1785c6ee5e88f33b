"""Pins of the oracle's cosine and inner-product reductions (Sec. 8,
extension (1)) against definitions computed independently with numpy:

  - the inner-product DCO in exact mode (eps0 = inf) decides <o, q> >= r
    exactly as the direct comparison does, including thresholds beyond
    ||o|| ||q|| (Cauchy-Schwarz) and far below -||o|| ||q||;
  - with any eps0 it never accepts an object whose inner product is below r;
  - IVF for inner products with nprobe = nlist is brute-force maximum inner
    product search; with fewer probes it searches the clusters of largest
    <c, q>;
  - IVF+ for inner products reduces to exact IVF with eps0 = inf or
    delta_d >= D, returns exact inner products, and keeps every true top-K
    member that passes its DCO at the exact K-th inner product;
  - cosine-similarity top-K equals Euclidean top-K of the normalised rows.
"""
import math

import numpy as np
import pytest

import oracle


def _data(seed, N=3000, D=48, nq=12, nlist=20):
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, 1.5, size=(nlist, D))
    lab = rng.integers(0, nlist, size=N)
    scale = rng.uniform(0.3, 3.0, size=(N, 1))         # varying norms matter for IP
    Y = (centres[lab] + rng.standard_normal((N, D))) * scale
    Q = centres[rng.integers(0, nlist, size=nq)] + rng.standard_normal((nq, D))
    C = np.stack([Y[lab == c].mean(0) for c in range(nlist)])
    return Y, Q, C, lab.astype(np.int32)


def _mips_topk(Y, q, K, members=None):
    """Brute force: the K largest <y, q>, ties by ascending id."""
    idx = np.arange(Y.shape[0]) if members is None else np.sort(members)
    ip = Y[idx] @ q
    order = np.lexsort((idx, -ip))[:K]
    return idx[order], ip[order]


def test_dco_ip_exact_mode_is_the_inner_product_comparison():
    rng = np.random.default_rng(5)
    for _ in range(300):
        D = int(rng.integers(8, 100))
        o, q = rng.normal(size=D) * rng.uniform(0.1, 5), rng.normal(size=D) * rng.uniform(0.1, 5)
        ip, bound = float(o @ q), float(np.linalg.norm(o) * np.linalg.norm(q))
        for r in (ip - 0.3 * abs(ip) - 1e-3, ip + 0.3 * abs(ip) + 1e-3, -2 * bound, bound * 1.01,
                  float(rng.uniform(-bound, bound))):
            if abs(ip - r) <= 1e-9 * bound:
                continue
            dec, dims, got_ip, _ = oracle.dco_ip(o, q, r, math.inf, 16)
            assert abs(got_ip - ip) <= 1e-12 * bound
            assert (dec == oracle.POSITIVE) == (ip >= r), (D, ip, r, dec)
            if r > bound:
                assert dec == oracle.REJECTED and dims == 0   # no real threshold exists
            else:
                assert dims == D
            # with sampling, never a false positive
            dec2, _, _, _ = oracle.dco_ip(o, q, r, 1.0, 16)
            if ip < r:
                assert dec2 != oracle.POSITIVE


def test_ivf_exact_ip_full_probe_is_brute_force_mips():
    Y, Q, C, lab = _data(11)
    ids, ips = oracle.ivf_exact_ip(Y, C, lab, Q, 15, C.shape[0])
    for q in range(Q.shape[0]):
        eids, eip = _mips_topk(Y, Q[q], 15)
        assert np.array_equal(ids[q], eids)
        assert np.allclose(ips[q], eip, rtol=1e-12, atol=1e-12)


def test_ivf_exact_ip_searches_the_clusters_of_largest_inner_product():
    Y, Q, C, lab = _data(12)
    nprobe = 4
    ids, ips = oracle.ivf_exact_ip(Y, C, lab, Q, 10, nprobe)
    for q in range(Q.shape[0]):
        cip = C @ Q[q]
        probes = np.lexsort((np.arange(C.shape[0]), -cip))[:nprobe]
        members = np.nonzero(np.isin(lab, probes))[0]
        eids, eip = _mips_topk(Y, Q[q], 10, members)
        assert np.array_equal(ids[q], eids)


@pytest.mark.parametrize("eps0,dd", [(math.inf, 16), (2.1, 48), (2.1, 64)])
def test_ivf_ads_ip_reduces_to_exact_ivf(eps0, dd):
    Y, Q, C, lab = _data(13)
    eids, eip = oracle.ivf_exact_ip(Y, C, lab, Q, 10, 5)
    ids, ips, dims, ncand = oracle.ivf_ads_ip(Y, C, lab, Q, 10, 5, eps0, dd)
    assert np.array_equal(ids, eids) and np.array_equal(ips, eip)


def test_ivf_ads_ip_exact_values_and_bracket():
    Y, Q, C, lab = _data(14)
    K, nprobe, eps0, dd = 10, 6, 2.1, 8
    ids, ips, dims, ncand = oracle.ivf_ads_ip(Y, C, lab, Q, K, nprobe, eps0, dd)
    eids, eip = oracle.ivf_exact_ip(Y, C, lab, Q, K, nprobe)
    assert np.all(dims < ncand * Y.shape[1])                 # early decisions happen
    for q in range(Q.shape[0]):
        for i, v in zip(ids[q], ips[q]):
            assert i >= 0 and abs(v - float(Y[i] @ Q[q])) <= 1e-10 * (1 + abs(v))
        rstar = eip[q, K - 1]
        must = [i for i in eids[q]
                if oracle.dco_ip(Y[i], Q[q], rstar, eps0, dd)[0] == oracle.POSITIVE]
        assert set(must) <= set(ids[q].tolist()), q


def test_cosine_top_k_is_euclidean_top_k_of_normalised_rows():
    Y, Q, C, lab = _data(15)
    Yn, Qn = oracle.normalize_rows(Y), oracle.normalize_rows(Q)
    assert np.allclose(np.linalg.norm(Yn, axis=1), 1.0, atol=1e-14)
    ids, d2 = oracle.knn_exact(Yn, Qn, 12)
    for q in range(Q.shape[0]):
        cos = (Y @ Q[q]) / (np.linalg.norm(Y, axis=1) * np.linalg.norm(Q[q]))
        order = np.lexsort((np.arange(Y.shape[0]), -cos))[:12]
        assert np.array_equal(ids[q], order)
        assert np.allclose(1.0 - d2[q] / 2.0, cos[order], atol=1e-12)
    z = oracle.normalize_rows(np.zeros((2, 5)))
    assert np.array_equal(z, np.zeros((2, 5)))
