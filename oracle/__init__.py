"""FP64 CPU oracle for IVF + ADSampling (Gao & Long, SIGMOD 2023).

TEST INFRASTRUCTURE ONLY.  The product library never imports, links or runs
anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` do.  It shares no
code with the CUDA path: the arithmetic lives in ``adsx_oracle.c`` (plain C,
double precision, no intrinsics), this module only marshals numpy arrays.

Functions (each follows the passage named in its docstring):
  rotate(P, X)                      Sec. 3.1, y := P' x
  knn_exact(Y, Qr, K)               Sec. 2.1, exact KNN
  probe(Cr, Qr, nprobe)             Sec. 2.2.2, nearest N_probe centroids
  ivf_exact(...)                    Sec. 2.2.2, IVF with FDScanning
  dco(o, q, r2, eps0, delta_d)      Algorithm 1 with the Sec. 3.2 test
  ivf_ads(...)                      Sec. 4, IVF+ (Algorithm 1 inside IVF)
  dco_fixed_r(Y, Qr, r2, ...)       Sec. 6.2.5 fixed-threshold linear scan
  dco_pd(o, q, r2, delta_d)         Sec. 6.1 PDScanning (exact partial-distance DCO)
  ivf_pd(...)                       Sec. 6.1 IVF* (IVF with PDScanning DCOs)
  recall_at(...), avg_dist_ratio()  Sec. 6.1 accuracy metrics
  normalize_rows(A)                 Sec. 8 ext. (1): cosine similarity is the
                                    Euclidean case on normalised vectors
  dco_ip(o, q, r, eps0, delta_d)    Sec. 8 ext. (1): inner-product DCO reduced
                                    to Algorithm 1 on normalised vectors
  ivf_exact_ip(...), ivf_ads_ip(...) IVF / IVF+ for inner products
  kac_apply(pairs, cs, X)           Sec. 6.2.3: the layered Kac walk as a
  kac_matrix(pairs, cs, D)          rotation, and its dense matrix
  graph_search(...)                 Sec. 2.2.1 / Sec. 4 (HNSW+): beam search on a
                                    proximity graph with Algorithm 1 DCOs
  cluster_entries(Y, Cr, assign, E) start vertices of the graph search (stand-in
                                    for HNSW's upper layers, Sec. 2.2.1):
                                    farthest-point samples per cluster
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adsx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

REJECTED, POSITIVE, NEGATIVE_AT_D = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile adsx_oracle.c into liboracle.so beside it (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, f64, cint = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            lib.orc_max_threads.restype = cint
            lib.orc_rotate.argtypes = [P, i32, P, i64, P, cint]
            lib.orc_knn_exact.argtypes = [P, i64, i32, P, i64, i32, P, P, cint]
            lib.orc_probe.argtypes = [P, i32, i32, P, i64, i32, P, P, cint]
            lib.orc_ivf_exact.argtypes = [P, i64, i32, P, i32, P, P, i64, i32, i32, P, P, cint]
            lib.orc_dco.argtypes = [P, P, i32, f64, f64, i32, P, P, P]
            lib.orc_dco.restype = cint
            lib.orc_ivf_ads.argtypes = [P, i64, i32, P, i32, P, P, i64, i32, i32,
                                        f64, i32, P, P, P, P, cint]
            lib.orc_dco_fixed_r.argtypes = [P, i64, i32, P, i64, P, f64, i32, P, P, P, cint]
            lib.orc_dco_pd.argtypes = [P, P, i32, f64, i32, P, P]
            lib.orc_dco_pd.restype = cint
            lib.orc_ivf_pd.argtypes = [P, i64, i32, P, i32, P, P, i64, i32, i32, i32, P, P, P, cint]
            lib.orc_dco_ip.argtypes = [P, P, i32, f64, f64, i32, P, P, P]
            lib.orc_dco_ip.restype = cint
            lib.orc_ivf_exact_ip.argtypes = [P, i64, i32, P, i32, P, P, i64, i32, i32, P, P, cint]
            lib.orc_ivf_ads_ip.argtypes = [P, i64, i32, P, i32, P, P, i64, i32, i32,
                                           f64, i32, P, P, P, P, cint]
            lib.orc_graph_search.argtypes = [P, i64, i32, P, i32, P, i32, P, i64, i32, i32, i32,
                                             f64, i32, i32, P, P, P, P, P, cint]
            _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def rotate(P, X, nthreads: int = 0):
    """Sec. 3.1: rows of X (float32 values) mapped to y = P x in FP64."""
    P = _c(P, np.float32)
    X = _c(X, np.float32)
    D = P.shape[0]
    assert P.shape == (D, D) and X.shape[1] == D
    Y = np.empty((X.shape[0], D), np.float64)
    _load().orc_rotate(_p(P), D, _p(X), X.shape[0], _p(Y), nthreads)
    return Y


def knn_exact(Y, Qr, K: int, nthreads: int = 0):
    """Sec. 2.1: exact KNN by brute force, ordered by (squared dist, id)."""
    Y = _c(Y, np.float64)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    ids = np.empty((nq, K), np.int64)
    d2 = np.empty((nq, K), np.float64)
    _load().orc_knn_exact(_p(Y), Y.shape[0], D, _p(Qr), nq, K, _p(ids), _p(d2), nthreads)
    return ids, d2


def probe(Cr, Qr, nprobe: int, nthreads: int = 0):
    """Sec. 2.2.2: the nprobe nearest centroids by (squared dist, cluster id)."""
    Cr = _c(Cr, np.float64)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    probes = np.empty((nq, nprobe), np.int32)
    pd2 = np.empty((nq, nprobe), np.float64)
    _load().orc_probe(_p(Cr), Cr.shape[0], D, _p(Qr), nq, nprobe, _p(probes), _p(pd2), nthreads)
    return probes, pd2


def ivf_exact(Y, Cr, assign, Qr, K: int, nprobe: int, nthreads: int = 0):
    """Sec. 2.2.2: IVF with exact (FDScanning) distances over the candidates."""
    Y = _c(Y, np.float64)
    Cr = _c(Cr, np.float64)
    assign = _c(assign, np.int32)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    ids = np.empty((nq, K), np.int64)
    d2 = np.empty((nq, K), np.float64)
    _load().orc_ivf_exact(_p(Y), Y.shape[0], D, _p(Cr), Cr.shape[0], _p(assign), _p(Qr),
                          nq, K, nprobe, _p(ids), _p(d2), nthreads)
    return ids, d2


def dco(o, q, r2: float, eps0: float, delta_d: int):
    """Algorithm 1 on one pair.  Returns (decision, dims, S, margin)."""
    o = _c(o, np.float64)
    q = _c(q, np.float64)
    dims = ctypes.c_int32(0)
    S = ctypes.c_double(0.0)
    m = ctypes.c_double(0.0)
    res = _load().orc_dco(_p(o), _p(q), o.shape[0], float(r2), float(eps0), int(delta_d),
                          ctypes.byref(dims), ctypes.byref(S), ctypes.byref(m))
    return int(res), int(dims.value), float(S.value), float(m.value)


def ivf_ads(Y, Cr, assign, Qr, K: int, nprobe: int, eps0: float, delta_d: int,
            nthreads: int = 0):
    """Sec. 4 (IVF+): sequential IVF with Algorithm 1 DCOs.

    Returns ids (nq,K), squared distances (nq,K), dims sampled per query,
    candidates per query."""
    Y = _c(Y, np.float64)
    Cr = _c(Cr, np.float64)
    assign = _c(assign, np.int32)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    ids = np.empty((nq, K), np.int64)
    d2 = np.empty((nq, K), np.float64)
    dims = np.empty(nq, np.int64)
    ncand = np.empty(nq, np.int64)
    _load().orc_ivf_ads(_p(Y), Y.shape[0], D, _p(Cr), Cr.shape[0], _p(assign), _p(Qr), nq,
                        K, nprobe, float(eps0), int(delta_d), _p(ids), _p(d2), _p(dims),
                        _p(ncand), nthreads)
    return ids, d2, dims, ncand


def dco_fixed_r(Y, Qr, r2, eps0: float, delta_d: int, nthreads: int = 0):
    """Sec. 6.2.5: Algorithm 1 for every (query, object) of a linear scan with a
    fixed per-query threshold r2.  Returns decisions, dims, margins (nq x N)."""
    Y = _c(Y, np.float64)
    Qr = _c(Qr, np.float64)
    r2 = _c(r2, np.float64)
    nq, D = Qr.shape
    N = Y.shape[0]
    dec = np.empty((nq, N), np.uint8)
    dims = np.empty((nq, N), np.int32)
    mar = np.empty((nq, N), np.float64)
    _load().orc_dco_fixed_r(_p(Y), N, D, _p(Qr), nq, _p(r2), float(eps0), int(delta_d),
                            _p(dec), _p(dims), _p(mar), nthreads)
    return dec, dims, mar


def dco_pd(o, q, r2: float, delta_d: int):
    """Sec. 6.1 PDScanning on one pair.  Returns (decision, dims, S)."""
    o = _c(o, np.float64)
    q = _c(q, np.float64)
    dims = ctypes.c_int32(0)
    S = ctypes.c_double(0.0)
    res = _load().orc_dco_pd(_p(o), _p(q), o.shape[0], float(r2), int(delta_d),
                             ctypes.byref(dims), ctypes.byref(S))
    return int(res), int(dims.value), float(S.value)


def ivf_pd(Y, Cr, assign, Qr, K: int, nprobe: int, delta_d: int, nthreads: int = 0):
    """Sec. 6.1 IVF*: sequential IVF with PDScanning DCOs.  Returns ids,
    squared distances and dims sampled per query."""
    Y = _c(Y, np.float64)
    Cr = _c(Cr, np.float64)
    assign = _c(assign, np.int32)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    ids = np.empty((nq, K), np.int64)
    d2 = np.empty((nq, K), np.float64)
    dims = np.empty(nq, np.int64)
    _load().orc_ivf_pd(_p(Y), Y.shape[0], D, _p(Cr), Cr.shape[0], _p(assign), _p(Qr), nq, K,
                       nprobe, int(delta_d), _p(ids), _p(d2), _p(dims), nthreads)
    return ids, d2, dims


# ------------------------------------------------------ graph search
def graph_search(Y, graph, entries, Qr, K: int, ef: int, eps0: float, delta_d: int,
                 max_iter: int = 0, nthreads: int = 0, pp: bool = False,
                 return_margin: bool = False):
    """Sec. 2.2.1 / Sec. 4 (HNSW+): greedy beam search on a proximity graph
    (graph: N x Rg int32 neighbour ids, -1 = none; entries: start vertex per
    query, or nq x E start vertices, -1 = none) whose DCOs run Algorithm 1
    against the largest distance of the result set of size ef, in the
    paper's order: one vertex at a time, the result set (and the threshold)
    updated after every vertex; the start vertices first, then the
    neighbours of each expansion of the nearest unexpanded result.
    max_iter = 0 means 16 * ef expansions at most.  pp: HNSW++ (Sec. 5.1),
    the result set's roles decoupled -- the DCO threshold and the output come
    from the K smallest exact distances, the beam (size ef) is kept with each
    DCO's observed distance (exact at d = D, else (D/d) S_d).  Returns ids,
    squared distances (K smallest), dims sampled and expansions per query,
    and with return_margin each query's closest call (the smallest relative
    gap of any DCO comparison or of two keys that decided the result set)."""
    Y = _c(Y, np.float64)
    graph = _c(graph, np.int32)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    entries = _c(np.asarray(entries).reshape(nq, -1), np.int64)
    ids = np.empty((nq, K), np.int64)
    d2 = np.empty((nq, K), np.float64)
    dims = np.empty(nq, np.int64)
    iters = np.empty(nq, np.int64)
    margin = np.empty(nq, np.float64)
    _load().orc_graph_search(_p(Y), Y.shape[0], D, _p(graph), graph.shape[1], _p(entries),
                             entries.shape[1], _p(Qr), nq, K, ef, int(max_iter or 16 * ef), float(eps0),
                             int(delta_d), int(bool(pp)), _p(ids), _p(d2), _p(dims), _p(iters),
                             _p(margin), nthreads)
    if return_margin:
        return ids, d2, dims, iters, margin
    return ids, d2, dims, iters


def cluster_entries(Y, Cr, assign, E: int):
    """Start vertices of the graph search, E per cluster (HNSW's upper layers
    only deliver a start vertex to the base layer, Sec. 2.2.1; clusters stand
    in for them).  Entry 0 of cluster c is its member nearest to the centroid
    Cr[c]; entry e is the member whose squared distance to the nearest of
    entries 0..e-1 is largest (farthest-point sampling); ties go to the lower
    id.  -1 once that largest distance is 0 (every member coincides with a
    chosen entry) and for an empty cluster.  FP64; returns nlist x E int64."""
    Y = np.asarray(Y, np.float64)
    Cr = np.asarray(Cr, np.float64)
    assign = np.asarray(assign)
    out = np.full((Cr.shape[0], E), -1, np.int64)
    for c in range(Cr.shape[0]):
        mem = np.nonzero(assign == c)[0]                 # ascending ids
        if len(mem) == 0:
            continue
        to_c = np.sum((Y[mem] - Cr[c]) ** 2, axis=1)
        pick = int(np.argmin(to_c))                      # first minimum = lowest id
        out[c, 0] = mem[pick]
        nearest = np.full(len(mem), np.inf)
        for e in range(1, E):
            nearest = np.minimum(nearest, np.sum((Y[mem] - Y[mem[pick]]) ** 2, axis=1))
            pick = int(np.argmax(nearest))               # first maximum = lowest id
            if not nearest[pick] > 0.0:
                break
            out[c, e] = mem[pick]
    return out


# ------------------------------------------------------ Kac's walk
def kac_apply(pairs, cs, X):
    """Sec. 6.2.3 (fast rotation by Kac's walk): applies the layered walk to
    every row of X in FP64, layer after layer; in layer l the pair
    (i, j) = (pairs[l, 2t], pairs[l, 2t+1]) with (c, s) = (cs[l, 2t],
    cs[l, 2t+1]) becomes (c x_i - s x_j, s x_i + c x_j).  Returns y = W x for
    each row (W the product of the layers)."""
    pairs = np.asarray(pairs)
    cs = np.asarray(cs, np.float64)
    Y = np.array(X, dtype=np.float64, copy=True)
    for l in range(pairs.shape[0]):
        i, j = pairs[l, 0::2], pairs[l, 1::2]
        c, s = cs[l, 0::2], cs[l, 1::2]
        xi, xj = Y[:, i].copy(), Y[:, j].copy()
        Y[:, i] = c * xi - s * xj
        Y[:, j] = s * xi + c * xj
    return Y


def kac_matrix(pairs, cs, D: int):
    """The dense D x D matrix W of a Kac walk (y = W x), built by walking the
    unit vectors; the IVF / ADSampling oracles then use it as P."""
    return kac_apply(pairs, cs, np.eye(D)).T


# ------------------------------------------- cosine and inner product
def normalize_rows(A):
    """Sec. 8, extension (1): cosine-similarity search is Euclidean search on
    the normalised vectors.  Rows of A scaled to unit norm in FP64 (a zero row
    stays zero)."""
    A = np.asarray(A, np.float64)
    n = np.sqrt(np.sum(A * A, axis=1, keepdims=True))
    return np.where(n > 0, A / np.where(n > 0, n, 1.0), 0.0)


def dco_ip(o, q, r: float, eps0: float, delta_d: int):
    """Sec. 8, extension (1): is <o, q> >= r?  Algorithm 1 on o/||o|| and
    q/||q|| against the squared threshold 2 - 2 r / (||o|| ||q||).  Returns
    (decision, dims, <o, q>, margin)."""
    o = _c(o, np.float64)
    q = _c(q, np.float64)
    dims = ctypes.c_int32(0)
    ip = ctypes.c_double(0.0)
    m = ctypes.c_double(0.0)
    res = _load().orc_dco_ip(_p(o), _p(q), o.shape[0], float(r), float(eps0), int(delta_d),
                             ctypes.byref(dims), ctypes.byref(ip), ctypes.byref(m))
    return int(res), int(dims.value), float(ip.value), float(m.value)


def ivf_exact_ip(Y, Cr, assign, Qr, K: int, nprobe: int, nthreads: int = 0):
    """IVF for inner products with exact scoring: the nprobe clusters of
    largest <c, q> (ties by id), the K largest <o, q> (ties by id) among their
    members.  Returns ids (nq,K) and inner products (nq,K), -1 / -inf padded."""
    Y = _c(Y, np.float64)
    Cr = _c(Cr, np.float64)
    assign = _c(assign, np.int32)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    ids = np.empty((nq, K), np.int64)
    ips = np.empty((nq, K), np.float64)
    _load().orc_ivf_exact_ip(_p(Y), Y.shape[0], D, _p(Cr), Cr.shape[0], _p(assign), _p(Qr),
                             nq, K, nprobe, _p(ids), _p(ips), nthreads)
    return ids, ips


def ivf_ads_ip(Y, Cr, assign, Qr, K: int, nprobe: int, eps0: float, delta_d: int,
               nthreads: int = 0):
    """IVF+ for inner products: sequential IVF whose DCOs are dco_ip against
    the K-th largest inner product held.  Returns ids, inner products, dims
    sampled per query, candidates per query."""
    Y = _c(Y, np.float64)
    Cr = _c(Cr, np.float64)
    assign = _c(assign, np.int32)
    Qr = _c(Qr, np.float64)
    nq, D = Qr.shape
    ids = np.empty((nq, K), np.int64)
    ips = np.empty((nq, K), np.float64)
    dims = np.empty(nq, np.int64)
    ncand = np.empty(nq, np.int64)
    _load().orc_ivf_ads_ip(_p(Y), Y.shape[0], D, _p(Cr), Cr.shape[0], _p(assign), _p(Qr), nq,
                           K, nprobe, float(eps0), int(delta_d), _p(ids), _p(ips), _p(dims),
                           _p(ncand), nthreads)
    return ids, ips, dims, ncand


# ---------------------------------------------------------------- metrics
def recall_at(ids, gt_ids, k: int) -> float:
    """Sec. 6.1: |first k returned  intersect  true top-k| / k, averaged."""
    ids = np.asarray(ids)[:, :k]
    gt = np.asarray(gt_ids)[:, :k]
    hit = 0
    for a, b in zip(ids, gt):
        hit += len(set(int(x) for x in a if x >= 0) & set(int(x) for x in b))
    return hit / float(k * ids.shape[0])


def avg_dist_ratio(d2, gt_d2) -> float:
    """Sec. 6.1: mean over rank-aligned pairs of dist(returned)/dist(true),
    Euclidean (square roots of the squared distances); pairs whose true
    distance is 0 or whose returned slot is empty are skipped."""
    a = np.sqrt(np.asarray(d2, np.float64))
    b = np.sqrt(np.asarray(gt_d2, np.float64))
    ok = (b > 0) & np.isfinite(a)
    return float(np.mean(a[ok] / b[ok])) if ok.any() else 1.0
