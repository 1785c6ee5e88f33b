"""Thin ctypes binding of libadsx.so (include/adsx.h).  Argument marshalling
only: every step of the path runs in the library's CUDA kernels.

Each function has the name of the C entry point without the ``adsx_`` prefix.
Inputs may be numpy arrays (host memory: outputs come back as numpy arrays
and the call synchronises) or torch CUDA tensors (outputs are allocated as
torch CUDA tensors and the work is enqueued on torch's current stream).

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2303_09855_gb300.build``); loading fails loudly otherwise.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadsx.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT = 0, -1, -2, -3, -4
F32, BF16, F16 = 0, 1, 2
L2, IP, COSINE = 0, 1, 2
REJECTED, POSITIVE, NEGATIVE_AT_D = 0, 1, 2

_lib = None


class AdsxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("adsx error %d: %s" % (code, msg))
        self.code = code


def load():
    """Loads libadsx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libadsx.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    try:
        import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    except Exception:
        pass
    lib = ctypes.CDLL(LIB_PATH)
    V, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    lib.adsx_build_index.argtypes = [V, i64, i32, V, V, i32, V, i32, V, ctypes.POINTER(V)]
    lib.adsx_build_index_metric.argtypes = [V, i64, i32, V, V, i32, V, i32, i32, V,
                                            ctypes.POINTER(V)]
    lib.adsx_index_metric.argtypes = [V, V]
    lib.adsx_build_graph.argtypes = [V, V, i32, i32, i32, V, ctypes.POINTER(V)]
    lib.adsx_free_graph.argtypes = [V]
    lib.adsx_graph_info.argtypes = [V, V, V, V, V]
    lib.adsx_graph_export.argtypes = [V, V, V]
    lib.adsx_search_graph.argtypes = [V, V, V, i64, i32, i32, i32, i32, f32, i32, V, V, V, V]
    lib.adsx_build_index_kac.argtypes = [V, i64, i32, V, V, i32, V, i32, V, i32, i32, V,
                                         ctypes.POINTER(V)]
    lib.adsx_free_index.argtypes = [V]
    lib.adsx_index_info.argtypes = [V, V, V, V, V, V]
    lib.adsx_search.argtypes = [V, V, i64, i32, i32, f32, i32, V, V, V, V]
    lib.adsx_probe.argtypes = [V, V, i64, i32, V, V, V]
    lib.adsx_rotate.argtypes = [V, V, i64, V, V]
    lib.adsx_dco_fixed_r.argtypes = [V, V, i64, V, f32, i32, V, V, V]
    lib.adsx_stream_status.argtypes = [V, V]
    lib.adsx_search_noalloc.argtypes = [V, V, i64, i32, i32, f32, i32, V, V, V, V]
    lib.adsx_search_batched.argtypes = [V, V, i64, V, V, i32, i32, f32, i32, V, i64, V, V, V, V]
    lib.adsx_search_pdscan.argtypes = [V, V, i64, i32, i32, i32, V, V, V, V]
    lib.adsx_autotune.argtypes = [V, V, i64, i32, i32, f32, V, V, V, V]
    lib.adsx_server_create.argtypes = [V, i32, i32, i32, i64, i32, i32, ctypes.POINTER(V)]
    lib.adsx_server_submit.argtypes = [V, V, i32, i32, f32, i32, V]
    lib.adsx_server_wait.argtypes = [V, i64, i32, V, V, V]
    lib.adsx_server_submit_many.argtypes = [V, V, i64, V, V, f32, i32, V]
    lib.adsx_server_cancel.argtypes = [V, i64]
    lib.adsx_server_stats.argtypes = [V, V, V, V, V, V, V, V]
    lib.adsx_server_reset_stats.argtypes = [V]
    lib.adsx_server_destroy.argtypes = [V]
    lib.adsx_set_stage_timing.argtypes = [V, i32]
    lib.adsx_set_scan_schedule.argtypes = [V, i32, i32, i32]
    lib.adsx_set_query_rotation.argtypes = [V, i32]
    lib.adsx_save_index.argtypes = [V, ctypes.c_char_p, V]
    lib.adsx_load_index.argtypes = [ctypes.c_char_p, V, V]
    lib.adsx_scan_config.argtypes = [V, V, V, V, V, V]
    lib.adsx_stage_ms.argtypes = [V, V]
    lib.adsx_scan_kernel_ms.argtypes = [V, V, V]
    lib.adsx_last_error.restype = ctypes.c_char_p
    for fn in ("adsx_build_index", "adsx_build_index_metric", "adsx_index_metric",
               "adsx_build_index_kac", "adsx_build_graph", "adsx_free_graph",
               "adsx_graph_info", "adsx_graph_export", "adsx_search_graph",
               "adsx_free_index", "adsx_index_info", "adsx_search",
               "adsx_probe", "adsx_rotate", "adsx_dco_fixed_r", "adsx_stream_status",
               "adsx_set_stage_timing", "adsx_stage_ms", "adsx_search_noalloc",
               "adsx_set_scan_schedule", "adsx_scan_config", "adsx_scan_kernel_ms",
               "adsx_set_query_rotation", "adsx_save_index", "adsx_load_index",
               "adsx_search_batched", "adsx_search_pdscan", "adsx_autotune",
               "adsx_server_create",
               "adsx_server_submit", "adsx_server_submit_many", "adsx_server_wait",
               "adsx_server_cancel",
               "adsx_server_stats", "adsx_server_reset_stats", "adsx_server_destroy"):
        getattr(lib, fn).restype = ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().adsx_last_error().decode()


def _check(rc):
    if rc != OK:
        raise AdsxError(rc, last_error())


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _stream_of(a, stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    if _is_torch_cuda(a):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return ctypes.c_void_p(0)


def _host(a, dtype):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _prep_queries(Q):
    if hasattr(Q, "data_ptr"):          # torch tensor: device, or (pinned) host memory
        import torch
        return Q.to(torch.float32).contiguous()
    return _host(Q, np.float32)


def _out(like, shape, np_dtype, torch_name):
    if hasattr(like, "data_ptr"):
        import torch
        if like.is_cuda:
            return torch.empty(shape, dtype=getattr(torch, torch_name), device=like.device)
        return torch.empty(shape, dtype=getattr(torch, torch_name),
                           pin_memory=like.is_pinned())
    return np.empty(shape, np_dtype)


class Index:
    """Owns an adsx_index handle (freed by close() or garbage collection)."""

    def __init__(self, handle):
        self.handle = handle
        N, D, nl, st, by = (ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(),
                            ctypes.c_int32(), ctypes.c_int64())
        _check(load().adsx_index_info(handle, ctypes.byref(N), ctypes.byref(D),
                                      ctypes.byref(nl), ctypes.byref(st), ctypes.byref(by)))
        self.N, self.D, self.nlist, self.storage, self.device_bytes = (
            N.value, D.value, nl.value, st.value, by.value)
        m = ctypes.c_int32()
        _check(load().adsx_index_metric(handle, ctypes.byref(m)))
        self.metric = m.value

    def close(self):
        if self.handle:
            load().adsx_free_index(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # method forms of the module functions
    def search(self, Q, K, nprobe, eps0=2.1, delta_d=32, return_dims=False, stream=None):
        return search(self, Q, K, nprobe, eps0, delta_d, return_dims, stream)

    def probe(self, Q, nprobe, stream=None):
        return probe(self, Q, nprobe, stream)

    def rotate(self, Q, stream=None):
        return rotate(self, Q, stream)

    def dco_fixed_r(self, Q, r2, eps0, delta_d, stream=None):
        return dco_fixed_r(self, Q, r2, eps0, delta_d, stream)

    def set_scan_schedule(self, schedule, queries_per_item=0, tiles_per_item=0):
        return set_scan_schedule(self, schedule, queries_per_item, tiles_per_item)

    def set_query_rotation(self, mode):
        return set_query_rotation(self, mode)

    def save(self, path, stream=None):
        return save_index(self, path, stream)


def build_index(X, P, centroids, assign, storage=F32, stream=None, metric=L2) -> Index:
    """adsx_build_index (metric L2) or adsx_build_index_metric (IP, COSINE):
    host arrays X (N x D), P (D x D), centroids, assign.  With IP / COSINE,
    searches return inner products / cosine similarities, largest first."""
    X = _host(X, np.float32)
    P = _host(P, np.float32)
    C = _host(centroids, np.float32)
    a = _host(assign, np.int32)
    h = ctypes.c_void_p()
    if metric == L2:
        _check(load().adsx_build_index(_ptr(X), X.shape[0], X.shape[1], _ptr(P), _ptr(C),
                                       C.shape[0], _ptr(a), int(storage),
                                       _stream_of(None, stream), ctypes.byref(h)))
    else:
        _check(load().adsx_build_index_metric(_ptr(X), X.shape[0], X.shape[1], _ptr(P), _ptr(C),
                                              C.shape[0], _ptr(a), int(storage), int(metric),
                                              _stream_of(None, stream), ctypes.byref(h)))
    return Index(h)


def save_index(index: Index, path: str, stream=None):
    """adsx_save_index: the built index to a file."""
    _check(load().adsx_save_index(index.handle, str(path).encode(), _stream_of(None, stream)))


def load_index(path: str, stream=None) -> Index:
    """adsx_load_index: an index saved by save_index, on the current device."""
    h = ctypes.c_void_p()
    _check(load().adsx_load_index(str(path).encode(), _stream_of(None, stream), ctypes.byref(h)))
    return Index(h)


def build_index_metric(X, P, centroids, assign, storage=F32, metric=L2, stream=None) -> Index:
    """adsx_build_index_metric (Sec. 8, extension (1))."""
    return build_index(X, P, centroids, assign, storage, stream, metric)


def build_index_kac(X, pairs, cs, centroids, assign, storage=F32, metric=L2, stream=None) -> Index:
    """adsx_build_index_kac: the rotation given as a layered Kac walk (Sec. 6.2.3),
    pairs and cs host arrays of shape (L, 2 * (D // 2)) (int32 / float32)."""
    X = _host(X, np.float32)
    pairs = _host(pairs, np.int32)
    cs = _host(cs, np.float32)
    C = _host(centroids, np.float32)
    a = _host(assign, np.int32)
    L = pairs.shape[0] if pairs.ndim == 2 else 0
    assert pairs.shape == cs.shape and (L == 0 or pairs.shape[1] == 2 * (X.shape[1] // 2))
    h = ctypes.c_void_p()
    _check(load().adsx_build_index_kac(_ptr(X), X.shape[0], X.shape[1], _ptr(pairs), _ptr(cs), L,
                                       _ptr(C), C.shape[0], _ptr(a), int(storage), int(metric),
                                       _stream_of(None, stream), ctypes.byref(h)))
    return Index(h)


class Graph:
    """Owns an adsx_graph handle (freed by close() or garbage collection)."""

    def __init__(self, handle, index):
        self.handle = handle
        self.index = index                 # the graph reads the index's vectors
        N, deg, nl, ne = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().adsx_graph_info(handle, ctypes.byref(N), ctypes.byref(deg), ctypes.byref(nl),
                                      ctypes.byref(ne)))
        self.N, self.degree, self.nlist = N.value, deg.value, nl.value
        self.entries_per_cluster = ne.value

    def close(self):
        if self.handle:
            load().adsx_free_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def search(self, Q, K, ef, eps0=2.1, delta_d=32, return_dims=False, stream=None,
               n_entry=4, decoupled=False):
        return search_graph(self.index, self, Q, K, ef, eps0, delta_d, return_dims, stream,
                            n_entry, decoupled)


def build_graph(index: Index, X, degree: int = 32, nprobe: int = 16,
                entries_per_cluster: int = 64, stream=None) -> Graph:
    """adsx_build_graph: a kNN proximity graph over the index's vectors (X: the
    raw vectors the index was built from) with entries_per_cluster
    farthest-point entry vertices per cluster."""
    X = _host(X, np.float32) if not _is_torch_cuda(X) else X.contiguous()
    h = ctypes.c_void_p()
    _check(load().adsx_build_graph(index.handle, _ptr(X), int(degree), int(nprobe),
                                   int(entries_per_cluster), _stream_of(None, stream),
                                   ctypes.byref(h)))
    return Graph(h, index)


def free_graph(graph: Graph):
    graph.close()


def graph_info(graph: Graph):
    """adsx_graph_info: (N, degree, nlist, entries_per_cluster)."""
    return graph.N, graph.degree, graph.nlist, graph.entries_per_cluster


def graph_export(graph: Graph):
    """adsx_graph_export: (neighbours N x degree int32, entries nlist x
    entries_per_cluster int64) as numpy."""
    nbr = np.empty((graph.N, graph.degree), np.int32)
    ent = np.empty((graph.nlist, graph.entries_per_cluster), np.int64)
    _check(load().adsx_graph_export(graph.handle, _ptr(nbr), _ptr(ent)))
    return nbr, ent


def search_graph(index: Index, graph: Graph, Q, K: int, ef: int, eps0: float = 2.1,
                 delta_d: int = 32, return_dims: bool = False, stream=None, n_entry: int = 4,
                 decoupled: bool = False):
    """adsx_search_graph (HNSW+, or HNSW++ with decoupled=True): returns (ids,
    squared dists[, dims]); the search starts from the entry vertices of each
    query's n_entry nearest clusters."""
    Q = _prep_queries(Q)
    nq = Q.shape[0]
    ids = _out(Q, (nq, K), np.int64, "int64")
    d2 = _out(Q, (nq, K), np.float32, "float32")
    dims = _out(Q, (nq,), np.int64, "int64") if return_dims else None
    _check(load().adsx_search_graph(index.handle, graph.handle, _ptr(Q), nq, int(K), int(ef),
                                    int(n_entry), int(bool(decoupled)), float(eps0) if math.isfinite(eps0) else float("inf"),
                                    int(delta_d), _ptr(ids), _ptr(d2), _ptr(dims),
                                    _stream_of(Q, stream)))
    return (ids, d2, dims) if return_dims else (ids, d2)


def index_metric(index: Index) -> int:
    """adsx_index_metric."""
    return index.metric


def free_index(index: Index):
    index.close()


def index_info(index: Index):
    """adsx_index_info: (N, D, nlist, storage, device_bytes)."""
    return index.N, index.D, index.nlist, index.storage, index.device_bytes


def search(index: Index, Q, K: int, nprobe: int, eps0: float = 2.1, delta_d: int = 32,
           return_dims: bool = False, stream=None):
    """adsx_search: returns (ids int64 nq x K, squared dists float32 nq x K[, dims nq])."""
    Q = _prep_queries(Q)
    nq = Q.shape[0]
    ids = _out(Q, (nq, K), np.int64, "int64")
    d2 = _out(Q, (nq, K), np.float32, "float32")
    dims = _out(Q, (nq,), np.int64, "int64") if return_dims else None
    _check(load().adsx_search(index.handle, _ptr(Q), nq, int(K), int(nprobe),
                              float(eps0) if math.isfinite(eps0) else float("inf"),
                              int(delta_d), _ptr(ids), _ptr(d2), _ptr(dims),
                              _stream_of(Q, stream)))
    return (ids, d2, dims) if return_dims else (ids, d2)


def _i32(a, like):
    if _is_torch_cuda(like):
        import torch
        return torch.as_tensor(a, dtype=torch.int32, device=like.device).contiguous()
    return _host(a, np.int32)


def search_batched(index: Index, Q, K, nprobe, eps0: float = 2.1, delta_d: int = 32,
                   max_K: int = 0, max_nprobe: int = 0, out_offsets=None, out_total: int = -1,
                   return_dims: bool = False, stream=None):
    """adsx_search_batched: per-query K and nprobe (arrays of length nq).

    Returns (ids, dists[, dims]) as flat arrays: query q's K[q] results start
    at out_offsets[q], or at the prefix sum of K when out_offsets is None.
    With CUDA tensors for Q, K and nprobe and max_K, max_nprobe and out_total
    given, nothing is read back to the host, so the call can be captured in a
    CUDA graph."""
    Q = _prep_queries(Q)
    nq = Q.shape[0]
    on_dev = _is_torch_cuda(Q)
    if not (max_K and max_nprobe and out_total >= 0):
        Kh = np.asarray(K.cpu() if hasattr(K, "cpu") else K, np.int64)
        Ph = np.asarray(nprobe.cpu() if hasattr(nprobe, "cpu") else nprobe, np.int64)
        max_K = int(max_K or (Kh.max() if nq else 1))
        max_nprobe = int(max_nprobe or (Ph.max() if nq else 1))
        if out_total < 0:
            if out_offsets is None:
                out_total = int(Kh.sum())
            else:
                oh = np.asarray(out_offsets.cpu() if hasattr(out_offsets, "cpu") else out_offsets)
                out_total = int(np.max(oh + Kh)) if nq else 0
    Kd = _i32(K, Q)
    Pd = _i32(nprobe, Q)
    offs = None
    if out_offsets is not None:
        if on_dev:
            import torch
            offs = torch.as_tensor(out_offsets, dtype=torch.int64, device=Q.device).contiguous()
        else:
            offs = _host(out_offsets, np.int64)
    ids = _out(Q, (out_total,), np.int64, "int64")
    d2 = _out(Q, (out_total,), np.float32, "float32")
    dims = _out(Q, (nq,), np.int64, "int64") if return_dims else None
    _check(load().adsx_search_batched(index.handle, _ptr(Q), nq, _ptr(Kd), _ptr(Pd), int(max_K),
                                      int(max_nprobe),
                                      float(eps0) if math.isfinite(eps0) else float("inf"),
                                      int(delta_d), _ptr(offs), int(out_total), _ptr(ids),
                                      _ptr(d2), _ptr(dims), _stream_of(Q, stream)))
    return (ids, d2, dims) if return_dims else (ids, d2)


def search_noalloc(index: Index, Q, K: int, nprobe: int, eps0: float = 2.1, delta_d: int = 32,
                   return_dims: bool = False, stream=None):
    """adsx_search_noalloc: adsx_search without any device allocation, for
    callers that must not allocate on the query path.  Q must be a CUDA
    tensor; outputs are CUDA tensors; the work is only enqueued on the
    stream.  Calls share one fixed scratch array: do not overlap them."""
    if not _is_torch_cuda(Q):
        raise ValueError("search_noalloc takes a CUDA tensor")
    Q = _prep_queries(Q)
    nq = Q.shape[0]
    ids = _out(Q, (nq, K), np.int64, "int64")
    d2 = _out(Q, (nq, K), np.float32, "float32")
    dims = _out(Q, (nq,), np.int64, "int64") if return_dims else None
    _check(load().adsx_search_noalloc(index.handle, _ptr(Q), nq, int(K), int(nprobe),
                                      float(eps0) if math.isfinite(eps0) else float("inf"),
                                      int(delta_d), _ptr(ids), _ptr(d2), _ptr(dims),
                                      _stream_of(Q, stream)))
    return (ids, d2, dims) if return_dims else (ids, d2)


def search_pdscan(index: Index, Q, K: int, nprobe: int, delta_d: int = 32,
                  return_dims: bool = False, stream=None):
    """adsx_search_pdscan: IVF* (PDScanning DCOs, exact results)."""
    Q = _prep_queries(Q)
    nq = Q.shape[0]
    ids = _out(Q, (nq, K), np.int64, "int64")
    d2 = _out(Q, (nq, K), np.float32, "float32")
    dims = _out(Q, (nq,), np.int64, "int64") if return_dims else None
    _check(load().adsx_search_pdscan(index.handle, _ptr(Q), nq, int(K), int(nprobe), int(delta_d),
                                     _ptr(ids), _ptr(d2), _ptr(dims), _stream_of(Q, stream)))
    return (ids, d2, dims) if return_dims else (ids, d2)


def probe(index: Index, Q, nprobe: int, stream=None):
    """adsx_probe: (cluster ids int32 nq x nprobe, squared centroid distances)."""
    Q = _prep_queries(Q)
    nq = Q.shape[0]
    pr = _out(Q, (nq, nprobe), np.int32, "int32")
    pd = _out(Q, (nq, nprobe), np.float32, "float32")
    _check(load().adsx_probe(index.handle, _ptr(Q), nq, int(nprobe), _ptr(pr), _ptr(pd),
                             _stream_of(Q, stream)))
    return pr, pd


def rotate(index: Index, Q, stream=None):
    """adsx_rotate: q' = P q for each row."""
    Q = _prep_queries(Q)
    out = _out(Q, tuple(Q.shape), np.float32, "float32")
    _check(load().adsx_rotate(index.handle, _ptr(Q), Q.shape[0], _ptr(out), _stream_of(Q, stream)))
    return out


def dco_fixed_r(index: Index, Q, r2, eps0: float, delta_d: int, stream=None):
    """adsx_dco_fixed_r: (decisions uint8 nq x N, dims int32 nq x N)."""
    Q = _prep_queries(Q)
    nq = Q.shape[0]
    if _is_torch_cuda(Q):
        import torch
        r2 = torch.as_tensor(r2, dtype=torch.float32, device=Q.device).contiguous()
    else:
        r2 = _host(r2, np.float32)
    dec = _out(Q, (nq, index.N), np.uint8, "uint8")
    dims = _out(Q, (nq, index.N), np.int32, "int32")
    _check(load().adsx_dco_fixed_r(index.handle, _ptr(Q), nq, _ptr(r2), float(eps0),
                                   int(delta_d), _ptr(dec), _ptr(dims), _stream_of(Q, stream)))
    return dec, dims


def autotune(index: Index, Q, K: int, nprobe: int, eps0: float = 2.1, stream=None,
             delta_d: int = 0):
    """adsx_autotune: returns (delta_d, items_per_sm, ms) of the fastest
    configuration on the sample Q (the schedule and its shape are stored in
    the index too: scan_config); searches with delta_d=0 then use the step.
    delta_d != 0 keeps the step fixed and tunes the rest."""
    Q = _prep_queries(Q)
    dd, ip, ms = ctypes.c_int32(int(delta_d)), ctypes.c_int32(), ctypes.c_float()
    _check(load().adsx_autotune(index.handle, _ptr(Q), Q.shape[0], int(K), int(nprobe),
                                float(eps0) if math.isfinite(eps0) else float("inf"),
                                ctypes.byref(dd), ctypes.byref(ip), ctypes.byref(ms),
                                _stream_of(Q, stream)))
    return dd.value, ip.value, ms.value


SCHED_AUTO, SCHED_QUERY, SCHED_CLUSTER = 0, 1, 2


def set_scan_schedule(index: Index, schedule: int, queries_per_item: int = 0,
                      tiles_per_item: int = 0):
    """adsx_set_scan_schedule: SCHED_AUTO, SCHED_QUERY (one warp per query)
    or SCHED_CLUSTER (one warp per cluster chunk and query group, in rounds);
    queries_per_item 1..64 (0 keeps the current value, -1 chooses it per
    batch) and tiles_per_item 1..64 (0 keeps the current value)."""
    _check(load().adsx_set_scan_schedule(index.handle, int(schedule), int(queries_per_item),
                                         int(tiles_per_item)))


ROT_FP32, ROT_TENSOR = 0, 1


def set_query_rotation(index: Index, mode: int):
    """adsx_set_query_rotation: ROT_TENSOR (tensor cores, exact digit
    products) or ROT_FP32 (compensated FP32 dot products, the default)."""
    _check(load().adsx_set_query_rotation(index.handle, int(mode)))


def scan_config(index: Index):
    """adsx_scan_config: dict of the index's delta_d (for delta_d = 0),
    schedule, queries_per_item (0: chosen per batch), tiles_per_item and
    items_per_sm."""
    v = [ctypes.c_int32() for _ in range(5)]
    _check(load().adsx_scan_config(index.handle, *[ctypes.byref(x) for x in v]))
    return dict(zip(("delta_d", "schedule", "queries_per_item", "tiles_per_item",
                     "items_per_sm"), (x.value for x in v)))


def set_stage_timing(index: Index, enable: bool = True):
    """adsx_set_stage_timing: record CUDA events between search stages."""
    _check(load().adsx_set_stage_timing(index.handle, 1 if enable else 0))


def stage_ms(index: Index):
    """adsx_stage_ms: device ms of (rotate, centroid distances, select, scan)
    of the last timed search."""
    out = (ctypes.c_float * 4)()
    _check(load().adsx_stage_ms(index.handle, out))
    return [float(x) for x in out]


def scan_kernel_ms(index: Index):
    """adsx_scan_kernel_ms: (device ms of the last timed search's scan-kernel
    launches summed, number of those launches)."""
    ms, n = ctypes.c_float(), ctypes.c_int32()
    _check(load().adsx_scan_kernel_ms(index.handle, ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def stream_status(index: Index, stream=None):
    """adsx_stream_status: synchronise and raise if a device wait gave up."""
    _check(load().adsx_stream_status(index.handle, _stream_of(None, stream)))


# ---------------------------------------------------------------- serving
class Server:
    """adsx_server_*: continuous-batching request loop (see include/adsx.h)."""

    def __init__(self, index: Index, max_slots=1024, max_batch=256, n_streams=4,
                 mem_budget_bytes=1 << 30, max_K=100, max_nprobe=64):
        self.index = index
        self.max_K = max_K
        h = ctypes.c_void_p()
        _check(load().adsx_server_create(index.handle, int(max_slots), int(max_batch),
                                         int(n_streams), int(mem_budget_bytes), int(max_K),
                                         int(max_nprobe), ctypes.byref(h)))
        self.handle = h

    def submit(self, q, K, nprobe, eps0=2.1, delta_d=32):
        q = _host(q, np.float32).reshape(-1)
        t = ctypes.c_int64()
        _check(load().adsx_server_submit(self.handle, _ptr(q), int(K), int(nprobe),
                                         float(eps0) if math.isfinite(eps0) else float("inf"),
                                         int(delta_d), ctypes.byref(t)))
        return t.value, int(K)

    def submit_many(self, Q, K, nprobe, eps0=2.1, delta_d=32):
        Q = _host(Q, np.float32)
        n = Q.shape[0]
        Kh = np.ascontiguousarray(np.broadcast_to(np.asarray(K, np.int32), (n,)))
        Ph = np.ascontiguousarray(np.broadcast_to(np.asarray(nprobe, np.int32), (n,)))
        t = np.empty(n, np.int64)
        _check(load().adsx_server_submit_many(self.handle, _ptr(Q), n, _ptr(Kh), _ptr(Ph),
                                              float(eps0) if math.isfinite(eps0) else float("inf"),
                                              int(delta_d), _ptr(t)))
        return [(int(x), int(k)) for x, k in zip(t, Kh)]

    def wait(self, ticket, timeout_ms=10000):
        t, K = ticket
        ids = np.empty(K, np.int64)
        d2 = np.empty(K, np.float32)
        dims = ctypes.c_int64()
        _check(load().adsx_server_wait(self.handle, t, int(timeout_ms), _ptr(ids), _ptr(d2),
                                       ctypes.byref(dims)))
        return ids, d2, dims.value

    def cancel(self, ticket):
        _check(load().adsx_server_cancel(self.handle, ticket[0]))

    def stats(self):
        p50, p99, qps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        c, b, mib, miq = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().adsx_server_stats(self.handle, ctypes.byref(p50), ctypes.byref(p99),
                                        ctypes.byref(qps), ctypes.byref(c), ctypes.byref(b),
                                        ctypes.byref(mib), ctypes.byref(miq)))
        return dict(p50_ms=p50.value, p99_ms=p99.value, qps=qps.value, completed=c.value,
                    batches=b.value, max_inflight_batches=mib.value,
                    max_inflight_queries=miq.value)

    def reset_stats(self):
        _check(load().adsx_server_reset_stats(self.handle))

    def close(self):
        if self.handle:
            load().adsx_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_create(index, **kw):
    return Server(index, **kw)


def server_submit(server, q, K, nprobe, eps0=2.1, delta_d=32):
    return server.submit(q, K, nprobe, eps0, delta_d)


def server_submit_many(server, Q, K, nprobe, eps0=2.1, delta_d=32):
    return server.submit_many(Q, K, nprobe, eps0, delta_d)


def server_wait(server, ticket, timeout_ms=10000):
    return server.wait(ticket, timeout_ms)


def server_cancel(server, ticket):
    server.cancel(ticket)


def server_stats(server):
    return server.stats()


def server_reset_stats(server):
    server.reset_stats()


def server_destroy(server):
    server.close()
