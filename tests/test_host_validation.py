"""CPU checks of the C ABI's host-side argument validation: every case here
is rejected with ADSX_EINVAL (and a message naming the problem) before the
library touches a device, so it runs without a GPU.  Covers the index build
(metric, sizes, storage type, assignments, malformed Kac walks), NULL
handles and output pointers, the graph and server entry points (create,
submit, wait, cancel, stats reset), index files that are missing, of
another kind or with header fields out of range (adsx_load_index), and the
thread-local error message of adsx_last_error.  Without a device, valid arguments fail with ADSX_ECUDA:
there is no host fallback."""
import ctypes
import threading

import numpy as np
import pytest


@pytest.fixture(scope="module")
def A():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    return adsx


def _small(N=12, D=8, nlist=3, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, D)).astype(np.float32)
    P = np.eye(D, dtype=np.float32)
    C = X[:nlist].copy()
    assign = (np.arange(N) % nlist).astype(np.int32)
    return X, P, C, assign


def _rejects(A, fn, needle):
    with pytest.raises(A.AdsxError) as ei:
        fn()
    assert ei.value.code == A.EINVAL, str(ei.value)
    assert needle in str(ei.value), str(ei.value)


def test_build_index_rejects_bad_arguments(A):
    X, P, C, a = _small()
    _rejects(A, lambda: A.build_index_metric(X, P, C, a, metric=7), "metric 7 not supported")
    _rejects(A, lambda: A.build_index(X, P, C, a, storage=9), "storage type 9 not supported")
    _rejects(A, lambda: A.build_index(X[:0], P, C, a[:0]), "N out of range")
    _rejects(A, lambda: A.build_index(np.zeros((12, 0), np.float32), P, C, a), "D out of range")
    big = np.zeros((2, 4081), np.float32)                 # above ADSX_MAX_D
    _rejects(A, lambda: A.build_index(big, np.eye(1, dtype=np.float32), big, np.zeros(2, np.int32)),
             "D out of range")
    _rejects(A, lambda: A.build_index(X[:2], P, C, a[:2]), "nlist out of range")   # nlist > N
    bad = a.copy()
    bad[5] = 3                                            # cluster ids are 0..nlist-1
    _rejects(A, lambda: A.build_index(X, P, C, bad), "assign[5] = 3 out of range")
    bad[5] = -1
    _rejects(A, lambda: A.build_index(X, P, C, bad), "assign[5] = -1 out of range")


def test_build_index_kac_rejects_malformed_walks(A):
    from paper_2303_09855_gb300 import workloads as W
    X, _, C, a = _small(D=8)
    pairs, cs = W.make_kac_walk(8, 3, 5)
    rep = pairs.copy()
    rep[1, 2] = rep[1, 3]                                 # an index twice in one layer
    _rejects(A, lambda: A.build_index_kac(X, rep, cs, C, a), "layer 1")
    oob = pairs.copy()
    oob[0, 0] = 8                                         # dims are 0..D-1
    _rejects(A, lambda: A.build_index_kac(X, oob, cs, C, a), "out of range or repeated")
    rot = cs.copy()
    rot[2, 0], rot[2, 1] = 0.6, 0.6                       # c^2 + s^2 = 0.72
    _rejects(A, lambda: A.build_index_kac(X, pairs, rot, C, a), "c^2 + s^2 != 1")
    many = np.tile(pairs[:1], (1025, 1))                  # above ADSX_MAX_KAC_LAYERS
    _rejects(A, lambda: A.build_index_kac(X, many, np.tile(cs[:1], (1025, 1)), C, a),
             "Kac walk layers out of range")


def test_null_handles_and_outputs(A):
    lib = A.load()
    V = ctypes.c_void_p
    ids = np.empty((1, 1), np.int64)
    d2 = np.empty((1, 1), np.float32)
    q = np.zeros((1, 8), np.float32)
    rc = lib.adsx_search(None, V(q.ctypes.data), 1, 1, 1, ctypes.c_float(2.1), 32,
                         V(ids.ctypes.data), V(d2.ctypes.data), None, None)
    assert rc == A.EINVAL and "index is NULL" in A.last_error()
    assert lib.adsx_free_index(None) == A.OK
    assert lib.adsx_free_graph(None) == A.OK
    assert lib.adsx_graph_info(None, None, None, None, None) == A.EINVAL
    assert lib.adsx_graph_export(None, None, None) == A.EINVAL
    assert "graph is NULL" in A.last_error()
    X = np.zeros((4, 8), np.float32)
    assert lib.adsx_build_graph(None, V(X.ctypes.data), 32, 1, 4, None, None) == A.EINVAL
    assert "out is NULL" in A.last_error()
    h = V()
    assert lib.adsx_build_graph(None, V(X.ctypes.data), 32, 1, 4, None, ctypes.byref(h)) == A.EINVAL
    assert "index is NULL" in A.last_error() and not h.value
    out = V()
    assert lib.adsx_server_create(None, 4, 4, 1, 1 << 20, 10, 4, ctypes.byref(out)) == A.EINVAL
    assert not out.value and "index is NULL" in A.last_error()
    assert lib.adsx_server_create(None, 4, 4, 1, 1 << 20, 10, 4, None) == A.EINVAL
    t = ctypes.c_int64()
    assert lib.adsx_server_submit(None, V(q.ctypes.data), 10, 4, ctypes.c_float(2.1), 32,
                                  ctypes.byref(t)) == A.EINVAL
    assert lib.adsx_server_wait(None, 0, 10, None, None, None) == A.EINVAL
    assert lib.adsx_server_cancel(None, 0) == A.EINVAL
    assert lib.adsx_server_reset_stats(None) == A.EINVAL
    assert "server is NULL" in A.last_error()


def test_last_error_is_per_thread(A):
    X, P, C, a = _small()
    with pytest.raises(A.AdsxError):
        A.build_index(X, P, C, a, storage=9)
    mine = A.last_error()
    assert "storage type 9" in mine
    seen = {}

    def other():
        seen["before"] = A.last_error()                   # a fresh thread has no message
        try:
            A.build_index_metric(X, P, C, a, metric=5)
        except A.AdsxError:
            pass
        seen["after"] = A.last_error()

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["before"] == "" and "metric 5" in seen["after"]
    assert A.last_error() == mine                         # untouched by the other thread


def test_no_cpu_fallback_without_a_device(A):
    """With valid arguments and no GPU the library fails with ADSX_ECUDA: it
    never computes a result on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    X, P, C, a = _small()
    with pytest.raises(A.AdsxError) as ei:
        A.build_index(X, P, C, a)
    assert ei.value.code == A.ECUDA, str(ei.value)


def test_load_index_rejects_bad_files(A, tmp_path):
    """adsx_load_index checks the file's magic and header before it
    allocates anything on a device."""
    _rejects(A, lambda: A.load_index(tmp_path / "missing.adsx"), "cannot open")
    p = tmp_path / "other.bin"
    p.write_bytes(b"NOTANIDX" + bytes(400))
    _rejects(A, lambda: A.load_index(p), "not an adsx index file")
    p.write_bytes(b"ADSXIDX1" + bytes(40))                      # header cut short
    _rejects(A, lambda: A.load_index(p), "not an adsx index file")
    hdr = np.zeros(36, dtype=np.int64)                          # N = 0, ... out of range
    p.write_bytes(b"ADSXIDX1" + hdr.tobytes())
    _rejects(A, lambda: A.load_index(p), "header fields out of range")
    lib = A.load()
    out = ctypes.c_void_p(123)
    assert lib.adsx_load_index(None, None, ctypes.byref(out)) == A.EINVAL and not out.value
    assert lib.adsx_load_index(str(p).encode(), None, None) == A.EINVAL
    assert lib.adsx_save_index(None, str(p).encode(), None) == A.EINVAL
    assert "index is NULL" in A.last_error()


def _header(**kw):
    """An adsx_load_index header (the file's int64 fields after the magic)
    for a 12 x 8 index with 3 clusters and the digit layout of P at Dp = 16
    (8-bit digits, T = 4, levels 2..6), with fields overridden by kw."""
    boff = [0, 0, 0, 256, 768, 1536, 2560] + [0] * 9
    f = dict(N=12, D=8, Dp=16, nlist=3, storage=0, metric=0, kac_L=0, total_tiles=3,
             max_tiles=1, tuned_delta_d=32, items_per_sm=48, sched=0, cm_G=0, cm_tpi=2,
             has_P=1, rot_ok=1, rot_b=8, rot_T=4, rot_Lmax=6, rot_floats=13 * 256)
    f.update(kw)
    vals = [f[k] for k in ("N", "D", "Dp", "nlist", "storage", "metric", "kac_L", "total_tiles",
                           "max_tiles", "tuned_delta_d", "items_per_sm", "sched", "cm_G",
                           "cm_tpi", "has_P", "rot_ok", "rot_b", "rot_T", "rot_Lmax",
                           "rot_floats")]
    return b"ADSXIDX1" + np.array(vals + kw.get("boff", boff), dtype=np.int64).tobytes()


@pytest.mark.parametrize("bad", [
    dict(rot_b=7),                      # digits not those the library derives from Dp
    dict(rot_floats=12 * 256),          # digit array size off
    dict(boff=[0, 0, 0, 256, 768, 1536, 2561] + [0] * 9),
    dict(Dp=32),                        # padding of D
    dict(has_P=0),                      # neither P nor a Kac walk
    dict(storage=3), dict(metric=7), dict(nlist=13), dict(tuned_delta_d=24),
    dict(sched=5), dict(kac_L=2),       # a Kac walk and P together
])
def test_load_index_checks_header_fields(A, tmp_path, bad):
    """Header fields outside the library's limits or inconsistent with one
    another are rejected before anything is allocated."""
    p = tmp_path / "h.adsx"
    p.write_bytes(_header(**bad))
    _rejects(A, lambda: A.load_index(p), "header fields out of range")


def test_load_index_valid_header_passes_the_checks(A, tmp_path):
    """The unmodified header of the cases above is accepted: the load gets
    past the header checks (and then fails on the missing arrays, or on the
    missing device)."""
    p = tmp_path / "h.adsx"
    p.write_bytes(_header())
    with pytest.raises(A.AdsxError) as ei:
        A.load_index(p)
    assert "header fields out of range" not in str(ei.value), str(ei.value)
