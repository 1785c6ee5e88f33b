"""Seeded synthetic workloads shaped like the paper's benchmarks.

This module only makes inputs: data vectors, query vectors, the random
orthogonal matrix P, and IVF centroids/assignments (k-means, the index-phase
clustering the paper takes from Faiss, Sec. 6.1).  It holds none of the
search method's arithmetic, and both the CUDA library's tests and the FP64
oracle's tests draw their inputs from it.

The paper's datasets (Table 1: Msong, DEEP, Word2Vec, GIST, GloVe, Tiny5M)
are not available here; the generators below stand in for them with the same
sizes, dimensionalities and value ranges (SIFT-like non-negative integer
values, GIST-like [0,1] sigmoid features, ...).

Seeds: numpy ``default_rng`` with data = 1, queries = 2, P = 3, k-means = 4,
each plus 1000 * (config number).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    X: np.ndarray            # N x D float32, raw space
    Q: np.ndarray            # nq x D float32, raw space
    P: np.ndarray            # D x D float32, orthogonal (y = P x)
    centroids: np.ndarray    # nlist x D float32, raw space
    assign: np.ndarray       # N int32 in [0, nlist)
    params: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.X.shape[0]

    @property
    def D(self):
        return self.X.shape[1]

    @property
    def nlist(self):
        return self.centroids.shape[0]


def make_P(D: int, seed: int) -> np.ndarray:
    """Haar-random orthogonal D x D matrix (float64): the Q factor of the QR
    decomposition of a seeded standard Gaussian matrix, with the signs fixed so
    that R has a positive diagonal (Mezzadri 2007).  The paper generates its
    random orthogonal transform by orthonormalising a Gaussian matrix
    (Sec. 3.1 footnote)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((D, D))
    Qm, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Qm * s[None, :]


def make_kac_walk(D: int, L: int, seed: int):
    """A seeded layered Kac walk (the O(D log D) random rotation named in
    Sec. 6.2.3): L layers, each a random perfect matching of the D coordinates
    (a seeded permutation read as consecutive pairs; with D odd one coordinate
    rests) with an angle theta ~ U[0, 2 pi) per pair.  Returns pairs (L x 2m
    int32, m = D // 2) and cs (L x 2m float32: cos theta, sin theta per pair).
    Only random draws -- applying the walk is the library's and the oracle's
    business."""
    rng = np.random.default_rng(seed)
    m = D // 2
    pairs = np.empty((L, 2 * m), np.int32)
    cs = np.empty((L, 2 * m), np.float32)
    for l in range(L):
        pairs[l] = rng.permutation(D)[:2 * m]
        th = rng.uniform(0.0, 2.0 * np.pi, size=m)
        cs[l, 0::2] = np.cos(th)
        cs[l, 1::2] = np.sin(th)
    return pairs, cs


def kmeans(X: np.ndarray, nlist: int, iters: int, seed: int, device: str = "cpu",
           sample: int | None = None):
    """Lloyd's k-means in float32 (index phase; the paper uses Faiss).

    Init: a seeded sample of nlist points.  Empty clusters keep their previous
    centroid.  Training runs on a seeded subsample of ``sample`` points (all
    points when None); the returned assignment is one nearest-centroid pass
    over all of X (ties to the lower cluster id).  Runs through torch on
    ``device`` so the million-point workloads stay quick."""
    import torch

    rng = np.random.default_rng(seed)
    N = X.shape[0]
    init = rng.choice(N, size=nlist, replace=False)
    train_idx = np.arange(N) if (sample is None or sample >= N) else np.sort(
        rng.choice(N, size=sample, replace=False))
    dev = torch.device(device)
    Xt = torch.from_numpy(np.ascontiguousarray(X[train_idx], np.float32)).to(dev)
    C = torch.from_numpy(np.ascontiguousarray(X[init], np.float32)).to(dev)

    def assign_of(A, C):
        out = torch.empty(A.shape[0], dtype=torch.int64, device=dev)
        cn = (C * C).sum(1)
        step = max(1, (1 << 26) // max(1, C.shape[0]))
        for s in range(0, A.shape[0], step):
            a = A[s:s + step]
            d = cn[None, :] - 2.0 * (a @ C.T)
            out[s:s + step] = torch.argmin(d, dim=1)
        return out

    for _ in range(iters):
        a = assign_of(Xt, C)
        sums = torch.zeros_like(C)
        sums.index_add_(0, a, Xt)
        cnt = torch.bincount(a, minlength=nlist).to(C.dtype)
        nz = cnt > 0
        C[nz] = sums[nz] / cnt[nz, None]
    Xall = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    a = assign_of(Xall, C)
    return C.cpu().numpy().astype(np.float32), a.cpu().numpy().astype(np.int32)


def _mixture_draw(rng, centres, n, noise_fn, weights=None):
    comp = rng.choice(centres.shape[0], size=n, p=weights)
    return comp, centres[comp] + noise_fn(comp)


# ------------------------------------------------------------------ configs
def gen_gaussian_mixture(N=10_000, D=128, nq=100, ncomp=50, nlist=100, kmeans_iters=10,
                         cfg=0, device="cpu", P_seed=None):
    """Plain FP32 IVF+ADSampling workload: N vectors from a ``ncomp``-component
    Gaussian mixture (centres ~ N(0, 4 I), unit within-component variance),
    queries from the same mixture, nlist k-means centroids (10 seeded
    iterations).  Defaults: the 10k x 128 correctness case."""
    base = 1000 * cfg
    rng = np.random.default_rng(1 + base)
    centres = rng.normal(0.0, 2.0, size=(ncomp, D))
    _, X = _mixture_draw(rng, centres, N, lambda c: rng.standard_normal((c.shape[0], D)))
    rq = np.random.default_rng(2 + base)
    _, Q = _mixture_draw(rq, centres, nq, lambda c: rq.standard_normal((c.shape[0], D)))
    X = X.astype(np.float32)
    Q = Q.astype(np.float32)
    P = make_P(D, (3 + base) if P_seed is None else P_seed).astype(np.float32)
    C, a = kmeans(X, nlist, kmeans_iters, 4 + base, device=device)
    return Workload("gauss_mix_N%d_D%d" % (N, D), X, Q, P, C, a,
                    dict(N=N, D=D, nq=nq, ncomp=ncomp, nlist=nlist, kmeans_iters=kmeans_iters))


def gen_sift_like(N=1_000_000, D=128, nq=10_000, ncomp=1024, nlist=4096, kmeans_iters=10,
                  cfg=1, device="cpu", noise_sd=6.0, inactive_sd=3.0, rank=16, amp=70.0):
    """SIFT-shaped workload: non-negative integer-valued floats in [0, 255].

    A ``ncomp``-component mixture whose centre dims are active with
    probability 0.25 with heavy-tailed magnitude |t_3| * 24 (else 0).  Each
    draw adds low-rank noise (z * s_c) W, with W a shared random rank x D
    basis of unit rows and s_c per-component scales amp * U(0.5, 1.5), plus
    isotropic noise N(0, noise_sd^2) on the component's active dims and
    N(0, inactive_sd^2) on the others; the result is clipped to [0, 255] and
    rounded.  The defaults give each component a low intrinsic dimension
    (rank 16) and make components overlap, so exact IVF over 4096 lists
    reaches recall@10 = 0.95 between nprobe 32 and 64, as SIFT1M does
    (measured: 0.937 at 32, 0.971 at 64); isotropic-only noise either
    isolates the components (nprobe 4 suffices) or concentrates distances
    (no early rejection is possible), neither of which resembles SIFT."""
    base = 1000 * cfg
    rng = np.random.default_rng(1 + base)
    active = rng.random((ncomp, D)) < 0.25
    mag = np.abs(rng.standard_t(3, size=(ncomp, D))) * 24.0
    centres = np.where(active, mag, 0.0)
    if rank > 0:
        Wb = rng.standard_normal((rank, D))
        Wb /= np.linalg.norm(Wb, axis=1, keepdims=True)
        sc = amp * rng.uniform(0.5, 1.5, size=(ncomp, rank))

    def draw(r, n):
        comp = r.integers(0, ncomp, size=n)
        out = np.empty((n, D), np.float32)
        step = 1 << 17
        for s in range(0, n, step):
            c = comp[s:s + step]
            noise = r.standard_normal((c.shape[0], D))
            v = centres[c] + noise * np.where(active[c], noise_sd, inactive_sd)
            if rank > 0:
                v += (r.standard_normal((c.shape[0], rank)) * sc[c]) @ Wb
            out[s:s + step] = np.rint(np.clip(v, 0.0, 255.0))
        return out

    X = draw(rng, N)
    Q = draw(np.random.default_rng(2 + base), nq)
    P = make_P(D, 3 + base).astype(np.float32)
    C, a = kmeans(X, nlist, kmeans_iters, 4 + base, device=device,
                  sample=min(N, 256 * nlist))
    return Workload("sift_like_N%d_D%d" % (N, D), X, Q, P, C, a,
                    dict(N=N, D=D, nq=nq, ncomp=ncomp, nlist=nlist, kmeans_iters=kmeans_iters,
                         noise_sd=noise_sd, inactive_sd=inactive_sd, rank=rank, amp=amp))


def gen_gist_like(N=1_000_000, D=960, nq=1_000, ncomp=1000, nlist=1024, rank=64,
                  kmeans_iters=10, cfg=2, device="cpu"):
    """GIST-shaped workload: floats in [0, 1] with correlated dims.

    Centres ~ N(0, I); shared covariance W W^T + 0.01 I with W in R^{D x rank},
    entries N(0, 1/rank); a logistic sigmoid maps every coordinate to (0, 1)."""
    base = 1000 * cfg
    rng = np.random.default_rng(1 + base)
    centres = rng.standard_normal((ncomp, D))
    W = rng.normal(0.0, 1.0 / np.sqrt(rank), size=(D, rank))

    def draw(r, n):
        out = np.empty((n, D), np.float32)
        step = 1 << 15
        for s in range(0, n, step):
            m = min(step, n - s)
            c = r.integers(0, ncomp, size=m)
            z = centres[c] + r.standard_normal((m, rank)) @ W.T + 0.1 * r.standard_normal((m, D))
            out[s:s + m] = 1.0 / (1.0 + np.exp(-z))
        return out

    X = draw(rng, N)
    Q = draw(np.random.default_rng(2 + base), nq)
    P = make_P(D, 3 + base).astype(np.float32)
    C, a = kmeans(X, nlist, kmeans_iters, 4 + base, device=device,
                  sample=min(N, 256 * nlist))
    return Workload("gist_like_N%d_D%d" % (N, D), X, Q, P, C, a,
                    dict(N=N, D=D, nq=nq, ncomp=ncomp, nlist=nlist, rank=rank))


def gen_uneven(N=2_000_000, D=256, nq=20_000, ncomp=4000, nlist=4096, kmeans_iters=10,
               cfg=3, device="cpu"):
    """Batched uneven workload: anisotropic mixture (per-(component, dim)
    variances log-uniform in [0.1, 10]), component weights Zipf(1.1), and
    per-query K in {1, 10, 100} and nprobe = round(exp(U[ln 8, ln 512]))."""
    base = 1000 * cfg
    rng = np.random.default_rng(1 + base)
    centres = rng.normal(0.0, 2.0, size=(ncomp, D))
    sd = np.sqrt(np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=(ncomp, D))))
    w = 1.0 / np.arange(1, ncomp + 1) ** 1.1
    w /= w.sum()

    def draw(r, n):
        out = np.empty((n, D), np.float32)
        step = 1 << 16
        for s in range(0, n, step):
            m = min(step, n - s)
            c = r.choice(ncomp, size=m, p=w)
            out[s:s + m] = centres[c] + sd[c] * r.standard_normal((m, D))
        return out

    X = draw(rng, N)
    rq = np.random.default_rng(2 + base)
    Q = draw(rq, nq)
    Ks = np.array([1, 10, 100], np.int32)[rq.integers(0, 3, size=nq)]
    nprobes = np.rint(np.exp(rq.uniform(np.log(8), np.log(512), size=nq))).astype(np.int32)
    P = make_P(D, 3 + base).astype(np.float32)
    C, a = kmeans(X, nlist, kmeans_iters, 4 + base, device=device,
                  sample=min(N, 256 * nlist))
    return Workload("uneven_N%d_D%d" % (N, D), X, Q, P, C, a,
                    dict(N=N, D=D, nq=nq, ncomp=ncomp, nlist=nlist, K=Ks, nprobe=nprobes))


def gen_serving(N=10_000_000, D=96, nq=100_000, ncomp=10_000, nlist=16384, kmeans_iters=10,
                cfg=4, device="cpu"):
    """Serving workload: unit-normalised mixture (centres ~ N(0, I), noise
    N(0, 0.25 I)), nprobe per request uniform in {16, 32, 64}."""
    base = 1000 * cfg
    rng = np.random.default_rng(1 + base)
    centres = rng.standard_normal((ncomp, D))

    def draw(r, n):
        out = np.empty((n, D), np.float32)
        step = 1 << 18
        for s in range(0, n, step):
            m = min(step, n - s)
            c = r.integers(0, ncomp, size=m)
            v = centres[c] + 0.5 * r.standard_normal((m, D))
            out[s:s + m] = v / np.linalg.norm(v, axis=1, keepdims=True)
        return out

    X = draw(rng, N)
    rq = np.random.default_rng(2 + base)
    Q = draw(rq, nq)
    nprobes = np.array([16, 32, 64], np.int32)[rq.integers(0, 3, size=nq)]
    P = make_P(D, 3 + base).astype(np.float32)
    C, a = kmeans(X, nlist, kmeans_iters, 4 + base, device=device,
                  sample=min(N, 256 * nlist))
    return Workload("serving_N%d_D%d" % (N, D), X, Q, P, C, a,
                    dict(N=N, D=D, nq=nq, ncomp=ncomp, nlist=nlist, nprobe=nprobes))


def random_small(N, D, nq, nlist, seed, spread=2.0, P_seed=None, kmeans_iters=5):
    """A quick seeded mixture of arbitrary (possibly ragged) size for tests."""
    rng = np.random.default_rng(seed)
    ncomp = max(2, nlist // 2)
    centres = rng.normal(0.0, spread, size=(ncomp, D))
    X = (centres[rng.integers(0, ncomp, size=N)] + rng.standard_normal((N, D))).astype(np.float32)
    Q = (centres[rng.integers(0, ncomp, size=nq)] + rng.standard_normal((nq, D))).astype(np.float32)
    P = make_P(D, seed + 7 if P_seed is None else P_seed).astype(np.float32)
    C, a = kmeans(X, nlist, kmeans_iters, seed + 11)
    return Workload("random_small_N%d_D%d" % (N, D), X, Q, P, C, a,
                    dict(N=N, D=D, nq=nq, nlist=nlist))
