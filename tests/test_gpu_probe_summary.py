"""Top-nprobe selection from the centroid GEMM's tile summary (Sec. 2.2.2:
the N_probe nearest centroids, ties by cluster id), checked exactly.

With P = I and every coordinate a multiple of 1/256 in [0, 1), the tensor-core
GEMM (TF32 operands exact, FP32 sums of multiples of 2^-16 below 2^5) and the
FP64 oracle compute the same distances bit for bit, so the probe lists must
equal the oracle's element by element.  The shapes exercise every branch of
the summary path:
  - nlist 4099 / 4100 / 2000: a last tile of 3, 4 and 80 columns;
  - far queries (distances in [2, 8), spaced 2^-16 = 32 ulps apart), so that
    distinct distances share a truncated summary key;
  - duplicated centroids (exact ties across tiles, resolved by id);
  - centroids whose ids follow their position on a line, so that a query's
    nearest clusters crowd into one or two 128-id tiles (tiles read whole);
  - nprobe from 1 to 64.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _grid(rng, shape, lo=0, hi=256):
    return (rng.integers(lo, hi, size=shape) / 256.0).astype(np.float32)


def _case(nlist, seed):
    rng = np.random.default_rng(seed)
    D = 16
    C = _grid(rng, (nlist, D))
    # a quarter duplicated at other ids
    dup = rng.choice(nlist, nlist // 4, replace=False)
    C[dup] = C[rng.integers(0, nlist, dup.size)]
    # a run of ids along one coordinate (neighbours share tiles)
    run = np.arange(nlist // 3, nlist // 3 + 600)
    C[run] = _grid(rng, (run.size, D), 120, 136)
    C[run, 0] = (np.arange(run.size) % 256) / 256.0
    Q = np.concatenate([
        _grid(rng, (60, D)),                        # anywhere
        _grid(rng, (40, D), 0, 8),                  # near a corner: far from most
        _grid(rng, (40, D), 248, 256),              # the opposite corner
        np.concatenate([_grid(rng, (40, 1)), _grid(rng, (40, D - 1), 124, 132)], 1),  # on the run
    ]).astype(np.float32)
    N = 2 * nlist
    X = C[np.arange(N) % nlist]
    assign = (np.arange(N) % nlist).astype(np.int32)
    return X, C, Q, assign


@pytest.mark.parametrize("nlist,seed", [(4099, 1), (4100, 2), (2000, 3)])
def test_probe_lists_are_exact(nlist, seed):
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    X, C, Q, assign = _case(nlist, seed)
    P = np.eye(16, dtype=np.float32)
    ix = adsx.build_index(X, P, C, assign)
    try:
        C64, Q64 = C.astype(np.float64), Q.astype(np.float64)
        for nprobe in (1, 2, 3, 4, 5, 17, 31, 32, 63, 64):
            pr, pd = ix.probe(Q, nprobe)
            epr, epd = oracle.probe(C64, Q64, nprobe)
            assert np.array_equal(pr, epr), (nlist, nprobe, np.nonzero((pr != epr).any(1))[0][:5])
            assert np.array_equal(pd, epd.astype(np.float32)), (nlist, nprobe)
    finally:
        ix.close()
