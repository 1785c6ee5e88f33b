"""An index written by adsx_save_index and read back by adsx_load_index
searches exactly like the one that was built (the paper keeps P from index
time, Sec. 6.1; here the whole index is kept).  Checked through the C ABI:
  - FP32 and BF16 storage, L2 and inner product, dense P and a Kac walk:
    identical query rotations, probes and exact-IVF results (eps0 = inf),
    and identical ADSampling results on the deterministic cluster-major
    schedule;
  - the tuned scan settings travel with the index;
  - the tensor-core rotation works on a loaded index;
  - a flipped byte, a truncated file and a file cut after the header are
    rejected (ADSX_EINVAL) and leave no index behind.
"""
import math

import numpy as np
import pytest

from paper_2303_09855_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    return adsx


def _build(adsx, kind, wl):
    if kind == "f32":
        return adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    if kind == "bf16":
        return adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign, storage=adsx.BF16)
    if kind == "ip":
        return adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign, metric=adsx.IP)
    pairs, cs = W.make_kac_walk(wl.X.shape[1], 12, 1)
    return adsx.build_index_kac(wl.X, pairs, cs, wl.centroids, wl.assign)


def _same_search(adsx, a, b, Q):
    assert np.array_equal(a.rotate(Q), b.rotate(Q))
    assert np.array_equal(a.probe(Q, 6), b.probe(Q, 6))
    for eps0 in (math.inf, 2.1):
        a.set_scan_schedule(adsx.SCHED_CLUSTER)
        b.set_scan_schedule(adsx.SCHED_CLUSTER)
        ia, da = a.search(Q, 10, 6, eps0=eps0)
        ib, db = b.search(Q, 10, 6, eps0=eps0)
        assert np.array_equal(ia, ib) and np.array_equal(da, db), eps0
    a.set_scan_schedule(adsx.SCHED_QUERY)
    b.set_scan_schedule(adsx.SCHED_QUERY)
    ia, da = a.search(Q, 10, 6, eps0=math.inf)
    ib, db = b.search(Q, 10, 6, eps0=math.inf)
    assert np.array_equal(ia, ib) and np.array_equal(da, db)


@pytest.mark.parametrize("kind", ["f32", "bf16", "ip", "kac"])
def test_saved_index_searches_identically(kind, tmp_path):
    adsx = _lib()
    wl = W.random_small(4000, 96, 300, 24, seed=11)
    ix = _build(adsx, kind, wl)
    path = tmp_path / ("%s.adsx" % kind)
    try:
        ix.save(path)
        lx = adsx.load_index(path)
        try:
            assert adsx.index_info(lx) == adsx.index_info(ix)
            assert lx.metric == ix.metric
            _same_search(adsx, ix, lx, wl.Q)
        finally:
            lx.close()
    finally:
        ix.close()


def test_tuned_settings_and_tensor_rotation_travel(tmp_path):
    adsx = _lib()
    wl = W.random_small(3000, 128, 400, 16, seed=12)
    ix = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign)
    try:
        adsx.autotune(ix, wl.Q, 10, 4)
        ix.set_scan_schedule(adsx.SCHED_CLUSTER, 8, 3)
        cfg = adsx.scan_config(ix)
        ix.save(tmp_path / "t.adsx")
        lx = adsx.load_index(tmp_path / "t.adsx")
        try:
            assert adsx.scan_config(lx) == cfg
            ix.set_query_rotation(adsx.ROT_TENSOR)
            lx.set_query_rotation(adsx.ROT_TENSOR)
            assert np.array_equal(ix.rotate(wl.Q), lx.rotate(wl.Q))
        finally:
            lx.close()
    finally:
        ix.close()


def test_damaged_files_are_rejected(tmp_path):
    adsx = _lib()
    wl = W.random_small(2000, 64, 50, 8, seed=13)
    ix = adsx.build_index(wl.X, wl.P, wl.centroids, wl.assign, storage=adsx.BF16)
    good = tmp_path / "g.adsx"
    try:
        ix.save(good)
    finally:
        ix.close()
    raw = good.read_bytes()
    cases = {
        "checksum mismatch": raw[:len(raw) // 2] + bytes([raw[len(raw) // 2] ^ 1]) + raw[len(raw) // 2 + 1:],
        "is truncated": raw[:len(raw) - 100],
        "is truncated ": raw[:8 + 36 * 8 + 10],
    }
    for needle, blob in cases.items():
        p = tmp_path / "bad.adsx"
        p.write_bytes(blob)
        with pytest.raises(adsx.AdsxError) as ei:
            adsx.load_index(p)
        assert ei.value.code == adsx.EINVAL and needle.strip() in str(ei.value), str(ei.value)
    lx = adsx.load_index(good)                        # the good file still loads
    lx.close()
