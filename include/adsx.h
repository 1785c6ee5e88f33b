/*
 * adsx.h -- C ABI of libadsx.so: IVF + ADSampling distance comparison
 * operations on one GB300 GPU (sm_103a).
 *
 * Method: Gao & Long, "High-Dimensional Approximate Nearest Neighbor Search:
 * with Reliable and Efficient Distance Comparison Operations", SIGMOD 2023.
 *   - Sec. 2.1    KNN query; DCO = "is dis <= r, and if so return dis".
 *   - Sec. 2.2.2  IVF: probe the N_probe nearest centroids, scan their members
 *                 against the K-th distance of a KNN set (+inf until full).
 *   - Sec. 3.1    random orthogonal transform y = P x; dis' = sqrt(D/d)||y|_d||.
 *   - Sec. 3.2    hypothesis test: reject dis <= r iff dis' > (1+eps0/sqrt d) r.
 *   - Algorithm 1 incremental sampling, delta_d dims per step, exact at d = D.
 *   - Sec. 4      IVF+ = IVF whose DCOs run Algorithm 1.
 *   - Sec. 5.2    IVF++ = a data layout that stores the first dims of all
 *                 candidates together (generalised here to 16-dim blocks).
 *   - Sec. 6.2.5  fixed-threshold linear-scan verification protocol.
 *
 * Conventions for every entry point:
 *   - Return value: ADSX_OK (0) or a negative ADSX_E* code; the message of
 *     the last failure on the calling thread is adsx_last_error().  No C++
 *     exception crosses this ABI.
 *   - Vectors are float32, row-major, D contiguous floats per vector, in the
 *     RAW (unrotated) space; the library applies P itself.
 *   - Distances are SQUARED Euclidean distances (in the rotated space, which
 *     equals the raw space up to the float32 rounding of P).
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the current CUDA device; the library
 *     inspects each pointer.  When any output is in host memory the call
 *     copies results back and synchronises `stream` before returning; when
 *     all of them are in device memory the call only enqueues work on
 *     `stream` and returns (query results are valid once `stream` reaches
 *     that point; use adsx_stream_status for the device-side error word).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - The caller owns every buffer it passes; the library never retains a
 *     caller pointer after a call returns.
 *   - Thread safety: searches on one index may run concurrently on different
 *     streams; build and free must not overlap any other call on the index.
 *   - Temporary device memory of a call comes from the library's own
 *     stream-ordered memory pool on the current device, which keeps what it
 *     has grown to between calls (like a caching allocator) so that repeated
 *     searches do not map fresh memory; adsx_search_noalloc allocates none.
 */
#ifndef ADSX_H
#define ADSX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adsx_index adsx_index;

enum {
    ADSX_OK = 0,
    ADSX_EINVAL = -1,   /* invalid argument (sizes, ranges, null pointers)   */
    ADSX_ENOMEM = -2,   /* device memory could not be allocated             */
    ADSX_ECUDA = -3,    /* a CUDA runtime call failed                       */
    ADSX_ETIMEOUT = -4  /* a bounded device-side wait gave up (results bad)  */
};

/* Storage type of the dimension-blocked vector layout. */
typedef enum { ADSX_F32 = 0, ADSX_BF16 = 1, ADSX_F16 = 2 } adsx_dtype;

/* Similarity of an index (adsx_build_index_metric; Sec. 8, extension (1)). */
typedef enum { ADSX_L2 = 0, ADSX_IP = 1, ADSX_COSINE = 2 } adsx_metric;

/* Scan schedules (adsx_set_scan_schedule). */
typedef enum {
    ADSX_SCHED_AUTO = 0,     /* cluster-major for batches probing each cluster    */
                             /* about once or more, else query-major              */
    ADSX_SCHED_QUERY = 1,    /* one warp per (query, split): every query apart    */
    ADSX_SCHED_CLUSTER = 2   /* one warp per (cluster, query group), in rounds    */
} adsx_schedule;

/* Limits of the current kernels (checked; ADSX_EINVAL beyond them). */
#define ADSX_MAX_D 4080       /* dimensions (padded to a multiple of 16)   */
#define ADSX_MAX_K 1024       /* neighbours per query                        */
#define ADSX_MAX_NPROBE 1024  /* probed clusters per query                   */
#define ADSX_MAX_NLIST 16384  /* clusters                                    */
#define ADSX_MAX_CLUSTER ((1 << 27) - 1)  /* members of one cluster (16 x this
                                           indexes a 32-bit block stride)    */
#define ADSX_MAX_KAC_LAYERS 1024  /* layers of a Kac-walk rotation           */
#define ADSX_MAX_DEGREE 32    /* neighbours per vertex of a proximity graph  */
#define ADSX_MAX_EF 512       /* result-set size of a graph search           */
#define ADSX_MAX_GRAPH_ENTRIES 16  /* start clusters of a graph search        */
#define ADSX_MAX_CLUSTER_ENTRIES 64 /* entry vertices per cluster of a graph  */

/*
 * adsx_build_index -- index phase (Sec. 6.1 "Implementation", Sec. 4, Sec. 5.2).
 *   X          host, N x D float32, raw data vectors; N in [1, 2^31).
 *   P          host, D x D float32 row-major, the random orthogonal matrix
 *              (y = P x).  Orthogonality is checked on the device:
 *              max |P P^T - I| <= 1e-4.
 *   centroids  host, nlist x D float32, IVF centroids in the raw space.
 *   assign     host, N int32, cluster of each vector, each in [0, nlist).
 *   storage    ADSX_F32, ADSX_BF16 or ADSX_F16: the type of the dim-blocked
 *              layout the scan reads.  16-bit types halve the bytes per
 *              dimension; partial sums stay FP32, and the index also keeps an
 *              FP32 copy of every rotated vector and its norm, from which each
 *              candidate that reaches d = D and may be positive gets its exact
 *              FP32 distance, so low precision moves only reject decisions.
 *   stream     work is enqueued on it and the call synchronises it.
 *   out        receives an opaque handle owning all of the index's device
 *              memory (rotated vectors in the dim-blocked per-cluster layout,
 *              ids, CSR offsets, rotated centroids, P).
 * Errors: ADSX_EINVAL (bad sizes, non-orthogonal P, assign out of range, a
 * cluster above ADSX_MAX_CLUSTER members), ADSX_ENOMEM, ADSX_ECUDA.  On
 * error *out is NULL and nothing leaks.
 */
int adsx_build_index(const float *X, int64_t N, int32_t D, const float *P,
                     const float *centroids, int32_t nlist,
                     const int32_t *assign, int32_t storage, void *stream,
                     adsx_index **out);

/*
 * adsx_build_index_metric -- adsx_build_index for cosine similarity or inner
 * product, through the reductions of Sec. 8, extension (1):
 *   ADSX_L2      exactly adsx_build_index.
 *   ADSX_COSINE  data rows, centroids and (at search) queries are scaled to
 *                unit norm, so cosine search is Euclidean search on them;
 *                searches return cosine similarities (1 - ||x^ - q^||^2 / 2),
 *                largest first.  A zero data row is ADSX_EINVAL; a zero query
 *                row stays zero (its results are unspecified).
 *   ADSX_IP      data rows are stored normalised with their norms ||o||;
 *                "is <o,q> at least r" is Algorithm 1 on o/||o||, q/||q||
 *                against the per-object squared threshold
 *                2 - 2 r / (||o|| ||q||) (a negative threshold rejects at
 *                once: <o,q> <= ||o|| ||q|| < r); r is the query's current
 *                K-th largest inner product.  Clusters are probed by the
 *                largest <c, q> with the given (raw) centroids.  Searches
 *                return inner products, largest first.
 * For both, padding slots hold -INF (ids -1); ties are ordered by id.  Other
 * arguments and errors as adsx_build_index.  adsx_dco_fixed_r and
 * adsx_search_noalloc accept ADSX_L2 indexes only, the graph search L2 and
 * COSINE indexes (ADSX_EINVAL otherwise).
 */
int adsx_build_index_metric(const float *X, int64_t N, int32_t D, const float *P,
                            const float *centroids, int32_t nlist,
                            const int32_t *assign, int32_t storage, int32_t metric,
                            void *stream, adsx_index **out);

/*
 * adsx_build_index_kac -- adsx_build_index_metric with the random rotation
 * given as a layered Kac walk instead of a dense P: the O(D log D) transform
 * the paper names for this step (Sec. 6.2.3).  With m = D / 2, layer l
 * (l < L) replaces each coordinate pair (i, j) = (pairs[2m l + 2t],
 * pairs[2m l + 2t + 1]), t < m, by (c y_i - s y_j, s y_i + c y_j) with
 * (c, s) = (cs[2m l + 2t], cs[2m l + 2t + 1]); the layers apply in order.
 * Data, centroids and queries are rotated by the same walk, an orthogonal
 * map, so distances and inner products are kept.  The walk must mix well
 * enough for the hypothesis test (Sec. 3); about 2-3 log2(D) layers of
 * random matchings and angles do.
 *   pairs   host, L x 2m int32 in [0, D), each index at most once per layer.
 *   cs      host, L x 2m float32 (c, s) per pair, |c^2 + s^2 - 1| <= 1e-5.
 *   L       1..ADSX_MAX_KAC_LAYERS.
 * Other arguments, results and errors as adsx_build_index_metric.
 */
int adsx_build_index_kac(const float *X, int64_t N, int32_t D, const int32_t *pairs,
                         const float *cs, int32_t L, const float *centroids,
                         int32_t nlist, const int32_t *assign, int32_t storage,
                         int32_t metric, void *stream, adsx_index **out);

/* Frees the index and all of its device memory (synchronises the device). */
int adsx_free_index(adsx_index *index);

/* The metric an index was built with (ADSX_L2, ADSX_IP or ADSX_COSINE). */
int adsx_index_metric(const adsx_index *index, int32_t *metric);

/* Shape of an index: any output pointer may be NULL. */
int adsx_index_info(const adsx_index *index, int64_t *N, int32_t *D,
                    int32_t *nlist, int32_t *storage, int64_t *device_bytes);

/*
 * adsx_search -- IVF+ query phase (Sec. 4 with Algorithm 1 DCOs, Sec. 2.2.2).
 * For each query: q' = P q; the nprobe clusters with the smallest
 * (||q' - c'||^2, cluster id); every member is scanned in delta_d-dim steps
 * and rejected as soon as D * S_d > r^2 * d * (1 + eps0/sqrt(d))^2 with
 * d < D, where r^2 is the query's current K-th squared distance (+inf until
 * K exact distances are known); members reaching d = D with S_D <= r^2
 * enter the query's top-K, ordered by (distance, id).
 *   Qv         host or device, nq x D float32 raw queries; nq >= 0.
 *   K          1..ADSX_MAX_K.   nprobe 1..min(nlist, ADSX_MAX_NPROBE).
 *   eps0       >= 0; +INFINITY disables the test (FDScanning, exact IVF).
 *   delta_d    multiple of 16, >= 16 (a value >= D also disables the test);
 *              0 uses the index's tuned step (adsx_autotune; 32 until tuned).
 *   ids        host or device, nq x K int64 output; -1 pads missing slots.
 *   dists      host or device, nq x K float32 squared distances; +INF pads
 *              (cosine / inner-product indexes: similarities, -INF pads).
 *   dims_read  host or device, nq int64 (may be NULL): dimensions sampled
 *              per query, summed over its candidates (Sec. 6.1 metric).
 * The threshold r is shared among the warps scanning a query, so which
 * candidates are rejected depends on scheduling; every returned distance is
 * exact and every true top-K member of the probed clusters that would pass
 * its DCO at the final K-th distance is returned.
 * Errors: ADSX_EINVAL, ADSX_ENOMEM, ADSX_ECUDA, ADSX_ETIMEOUT.
 */
int adsx_search(const adsx_index *index, const float *Qv, int64_t nq,
                int32_t K, int32_t nprobe, float eps0, int32_t delta_d,
                int64_t *ids, float *dists, int64_t *dims_read, void *stream);

/*
 * adsx_search_pdscan -- the IVF* baseline of Sec. 6.1: IVF whose DCOs are
 * PDScanning -- dimensions scanned in delta_d steps, a candidate stopped as
 * soon as its partial squared distance S_d exceeds r^2 (strictly).  An exact
 * DCO: results equal exact IVF; only the dimensions read differ.  On an
 * index built with P = I the partial sums are over raw coordinates, which
 * with the dim-blocked layout is the paper's IVF** (Sec. 6.1).  Arguments and
 * outputs as adsx_search (no eps0).
 */
int adsx_search_pdscan(const adsx_index *index, const float *Qv, int64_t nq,
                       int32_t K, int32_t nprobe, int32_t delta_d, int64_t *ids,
                       float *dists, int64_t *dims_read, void *stream);

/*
 * adsx_search_batched -- the IVF+ query phase for a batch whose queries each
 * have their own K and nprobe (same method as adsx_search, Sec. 4), in one
 * persistent scan launch: a device-side planner validates the per-query
 * values, splits long queries into several work items and orders the
 * queries longest-first; split queries share their r through the device.
 *   Qv           host or device, nq x D float32 raw queries.
 *   K, nprobe    host or device, nq int32 each; K[q] in [1, max_K],
 *                nprobe[q] in [1, max_nprobe].  Host arrays are checked
 *                before any work (ADSX_EINVAL); device arrays are checked by
 *                the planner, which clamps bad values and sets the index's
 *                error word (reported as ADSX_EINVAL by this call when it
 *                synchronises, else by adsx_stream_status).
 *   max_K        1..ADSX_MAX_K; max_nprobe 1..min(nlist, ADSX_MAX_NPROBE).
 *   eps0, delta_d  as adsx_search; delta_d = 0 uses the index's tuned step
 *                (adsx_autotune; 32 until tuned).
 *   out_offsets  host or device, nq int64 (may be NULL): query q's results
 *                go to ids/dists[out_offsets[q] .. + K[q]); NULL means the
 *                prefix sums of K (results packed in query order).
 *   out_total    length of ids and dists; a query whose slice does not fit
 *                is skipped and flagged in the error word.
 *   ids, dists   host or device, out_total entries; -1 / +INF padding
 *                (cosine / inner-product indexes: similarities, -INF).
 *   dims_read    host or device, nq int64 (may be NULL).
 * With all pointers in device memory the call only enqueues work, and the
 * sequence can be captured in a CUDA graph.
 */
int adsx_search_batched(const adsx_index *index, const float *Qv, int64_t nq,
                        const int32_t *K, const int32_t *nprobe, int32_t max_K,
                        int32_t max_nprobe, float eps0, int32_t delta_d,
                        const int64_t *out_offsets, int64_t out_total,
                        int64_t *ids, float *dists, int64_t *dims_read,
                        void *stream);

/*
 * adsx_probe -- the query rotation and centroid selection steps of
 * adsx_search alone (Sec. 3.1, Sec. 2.2.2), for inspection and tests.
 *   probes     host or device, nq x nprobe int32, ascending (dist, id).
 *   probe_d2   host or device, nq x nprobe float32 (may be NULL): the
 *              ranking key ||q' - c'||^2; for cosine indexes on normalised
 *              q and c; for inner-product indexes ||q'||^2 + max ||c'||^2 -
 *              2 <q', c'> (ascending = largest inner product first).
 */
int adsx_probe(const adsx_index *index, const float *Qv, int64_t nq,
               int32_t nprobe, int32_t *probes, float *probe_d2, void *stream);

/*
 * adsx_rotate -- q' = P q for each query (Sec. 3.1), or the Kac walk of an
 * index built with adsx_build_index_kac.
 *   out        host or device, nq x D float32.
 */
int adsx_rotate(const adsx_index *index, const float *Qv, int64_t nq,
                float *out, void *stream);

/*
 * adsx_dco_fixed_r -- Algorithm 1 for every (query, indexed vector) pair with
 * a FIXED squared threshold per query: the verification protocol of
 * Sec. 6.2.5 (linear scan, independent DCOs), run by adsx_search's own scan
 * kernel in a fixed-threshold mode (every cluster scanned, no KNN set), so
 * each decision comes from the same per-step FP32 accumulation order, test
 * and (16-bit storage) exact recheck as in a search.  The test is off for
 * eps0 = +INF or delta_d >= D (one full-width step, as in a search).
 *   r2         host or device, nq float32 squared thresholds (+INF allowed).
 *   decisions  host or device, nq x N uint8, indexed by original vector id:
 *              0 = rejected at some d < D (Case 1), 1 = reached d = D with
 *              S_D <= r2 (positive), 2 = reached d = D with S_D > r2.
 *   dims       host or device, nq x N int32 dims sampled (may be NULL).
 */
int adsx_dco_fixed_r(const adsx_index *index, const float *Qv, int64_t nq,
                     const float *r2, float eps0, int32_t delta_d,
                     uint8_t *decisions, int32_t *dims, void *stream);

/*
 * adsx_stream_status -- synchronises `stream`, then reads and clears the
 * index's device-side error word (set by device-side argument checks of the
 * batched form, or when a bounded wait inside a kernel gives up).  Returns
 * ADSX_OK, ADSX_EINVAL (argument check), ADSX_ETIMEOUT or ADSX_ECUDA.
 */
int adsx_stream_status(const adsx_index *index, void *stream);

/*
 * adsx_set_scan_schedule -- how adsx_search and adsx_search_pdscan (and, when
 * forced to ADSX_SCHED_CLUSTER, adsx_dco_fixed_r) organise the candidate
 * scan on the GPU.  Results follow the same method either way; only the
 * order of work, and with it which r each DCO sees, differs.
 *   ADSX_SCHED_QUERY    a work item is one query (or a split of one): its
 *                       warp visits the probed clusters in order and
 *                       tightens r after every KNN-set update (Sec. 2.2.2).
 *   ADSX_SCHED_CLUSTER  a work item is one cluster and up to
 *                       queries_per_item of the queries probing it: each
 *                       Delta_d step of a 32-member tile is read once and
 *                       tested against all of them.  The probe ranks are
 *                       covered in rounds -- each query's nearest cluster
 *                       in full (no r is known yet), then rank ranges
 *                       growing 4x -- each round testing against the K-th
 *                       distance of the rounds before it (a valid r: the
 *                       K-th of a subset of exact candidate distances), so
 *                       results do not depend on scheduling.  A tile's
 *                       first step is computed for every (query, member);
 *                       its later steps only for the pairs still live.  A
 *                       cluster is shared among items in chunks of
 *                       tiles_per_item tiles.  Needs delta_d <= 64 (or the
 *                       test off) and an L2 or cosine index; other searches
 *                       run query-major.
 *   ADSX_SCHED_AUTO     cluster-major when it applies and the batch probes
 *                       each cluster about once or more on average (nq >=
 *                       128, nq * nprobe >= nlist; with 16-bit storage and
 *                       D >= 512, nq * nprobe >= 8 nlist), else query-major.
 *                       The initial setting.
 *   queries_per_item    1..64; 0 keeps the current setting; -1 returns to
 *                       the initial one, chosen per batch from q = nq *
 *                       nprobe / nlist: 16 from q = 24, 8 from q = 6, else 4
 *                       (at D >= 512 at most 8, and 4 with 16-bit storage).
 *   tiles_per_item      1..64 32-member tiles, or 0 to keep the current value
 *                       (2 initially).
 * Not thread-safe with other calls on the same index.
 */
int adsx_set_scan_schedule(adsx_index *index, int32_t schedule, int32_t queries_per_item,
                           int32_t tiles_per_item);

/*
 * adsx_save_index -- writes a built index to the file `path` (the paper keeps
 * P from index time, Sec. 6.1 "Implementation"; this keeps the whole index:
 * the rotation (P or the Kac walk), rotated centroids, the dim-blocked
 * vectors and, for 16-bit storage, their FP32 copy, ids and offsets, the
 * tuned scan settings), so that another process can search it without
 * rebuilding.  The file is in the host's byte order with an FNV-1a
 * checksum; it is about as large as the index's device memory.
 *   index   a built index; its stream work is finished first (`stream` is
 *           synchronised).
 * Errors: ADSX_EINVAL (NULL arguments, the file cannot be written),
 * ADSX_ECUDA.
 * adsx_load_index -- reads such a file onto the current CUDA device; the
 * index searches exactly like the one saved (same results, bit for bit).
 * The query-rotation mode starts as ADSX_ROT_FP32.  Synchronous.
 * Errors: ADSX_EINVAL (no such file, not an index file, fields outside the
 * library's limits, truncated, checksum mismatch, inconsistent offsets),
 * ADSX_ENOMEM, ADSX_ECUDA; *out is NULL then and nothing leaks.
 */
int adsx_save_index(const adsx_index *index, const char *path, void *stream);
int adsx_load_index(const char *path, void *stream, adsx_index **out);

/* Query rotation modes (adsx_set_query_rotation). */
#define ADSX_ROT_FP32 0      /* compensated FP32 dot products (Dot2)                */
#define ADSX_ROT_TENSOR 1    /* tcgen05 tensor cores, exact digit products           */

/*
 * adsx_set_query_rotation -- how searches on this index rotate their queries,
 * q' = P q (Sec. 3.1).  ADSX_ROT_TENSOR, available on every index with a
 * dense P and a padded D of at most 1024: every query value and every
 * entry of P is split into T signed integer digits of b bits (with a power
 * of two per row; bT >= 28), the digit products are summed on the tensor
 * cores (tcgen05.mma kind::tf32), where every partial sum of a level is an
 * integer held exactly in FP32 (T Dp (2^b - 1)^2 < 2^24), and the levels
 * are added by compensated summation (as if in twice the precision) and
 * rounded once to FP32: q' is the FP64 product of the
 * FP32 inputs, rounded to FP32, up to the digits' truncated tails (below
 * 2^(-bT) of each row's largest value) -- the error-free splitting of
 * Ozaki, Ogita, Oishi and Rump (2012).  ADSX_ROT_FP32: compensated FP32 dot
 * products on the CUDA cores, as accurate as twice the working precision:
 * the initial mode, measured faster on GB300 for query batches (0.21 vs
 * 0.27 ms for 10k queries at D = 128, 0.47 vs 0.79 ms for 1000 at D = 960)
 * and the only one for D > 1024 (Kac-walk indexes use their walk).  The digits
 * of P take (about half of T^2) Dp^2 floats of device memory per index
 * (122 MB at D = 960), a search (units + T) Dp floats of scratch per query
 * (units, the work units of one output tile: 5 to 6 for D <= 128, 19 for
 * D = 960; T = 4 to 6).  Returns ADSX_EINVAL for an
 * unknown mode or ADSX_ROT_TENSOR where it is not available.  Not
 * thread-safe with other calls on the same index.
 */
int adsx_set_query_rotation(adsx_index *index, int32_t mode);

/*
 * adsx_scan_config -- the index's current scan settings: the step delta_d
 * used when a search passes 0, the schedule, queries (0: chosen per batch)
 * and tiles per cluster-major item, and the query-major work items per SM
 * (any output pointer may be NULL).
 */
int adsx_scan_config(const adsx_index *index, int32_t *delta_d, int32_t *schedule,
                     int32_t *queries_per_item, int32_t *tiles_per_item,
                     int32_t *items_per_sm);

/*
 * adsx_autotune -- picks, by timing adsx_search on a caller-supplied query
 * sample (one warm-up and three timed runs each, CUDA events on `stream`),
 * the step delta_d (Sec. 6.2.4: 16..64 give the best trade-off; the
 * candidates are 16, 32, 48, 64, up to the padded D) under each scan
 * schedule (query-major, cluster-major), then the winner's shape: queries
 * per item (chosen per batch, 4, 8, 16, 32) and tiles per item (1, 2, 4) for
 * cluster-major, work items per SM (24, 48, 96) for query-major.  The winner is stored in the
 * index: the schedule and shape apply to every later search, the step to
 * searches that pass delta_d = 0 (adsx_scan_config reads them back).  Tune
 * on a sample the size of the batches to be searched: the schedule that
 * wins depends on it.
 *   Qv               host or device, nq x D sample queries (nq >= 1).
 *   K, nprobe, eps0  the search parameters to tune for.
 *   best_delta_d     in: 0 to tune the step, or a step (a multiple of 16) to
 *                    keep fixed while the schedule and shape are tuned; out:
 *                    the step chosen (may be NULL: the step is tuned).
 *   best_items_per_sm, best_ms  outputs (each may be NULL).
 * Not thread-safe with other calls on the same index.
 */
int adsx_autotune(adsx_index *index, const float *Qv, int64_t nq, int32_t K,
                  int32_t nprobe, float eps0, int32_t *best_delta_d,
                  int32_t *best_items_per_sm, float *best_ms, void *stream);

/*
 * adsx_set_stage_timing -- when `enable` is non-zero, every later
 * adsx_search on this index records CUDA events on its stream between its
 * stages (query rotation, centroid distances, top-nprobe select, candidate
 * scan).  Timing is per index: do not enable it while searches on the index
 * run concurrently on several streams.
 * adsx_stage_ms -- waits for the last timed search and writes the device
 * time of its four stages, in milliseconds, to ms[0..3] (in the order above).
 * Returns ADSX_EINVAL if no timed search has run.
 */
int adsx_set_stage_timing(adsx_index *index, int32_t enable);
int adsx_stage_ms(const adsx_index *index, float *ms);

/*
 * adsx_scan_kernel_ms -- with stage timing on, waits for the last timed
 * search and writes the device time of its scan-kernel launches alone, in
 * milliseconds, summed (*ms: the candidate scan without the planning and
 * merging kernels around it; the query-major scan or each cluster-major
 * round), and their number (*launches, may be NULL).
 */
int adsx_scan_kernel_ms(const adsx_index *index, float *ms, int32_t *launches);

/*
 * adsx_search_noalloc -- adsx_search for callers that must not allocate
 * device memory while serving queries: for example a process whose GPU memory
 * is reserved up front by another allocator or a fixed budget, where
 * cudaMalloc / cudaMallocAsync would fail, or would lock or synchronise and
 * stall other work.  The paper has no counterpart; this is an interface
 * variant of adsx_search, computing the same results.
 *   - Same arguments and results as adsx_search (delta_d = 0 too: the
 *     index's tuned step), but Qv, ids, dists and dims_read must all be
 *     DEVICE pointers on the index's GPU (ADSX_EINVAL otherwise); the call
 *     only enqueues work on `stream` and never synchronises.
 *   - No device memory is allocated or freed: every temporary buffer is cut
 *     from one fixed array of ADSX_NOALLOC_SCRATCH_BYTES that the library
 *     holds on every GPU that loads it, until the process exits.  A call
 *     whose temporaries would not fit (roughly nq * (12*D + 4*nlist +
 *     4*nprobe) bytes: q', its TF32 halves for the centroid GEMM, the
 *     centroid distances and the probes -- with the tensor-core query
 *     rotation the 4*nlist
 *     part is at least the rotation's digits and partial sums of
 *     min(nq, 1024) queries, 4 * (units + T) * Dp each (see
 *     adsx_set_query_rotation) --
 *     plus partial top-K lists when nq is small) returns ADSX_EINVAL with the
 *     size it needed; split the batch.
 *   - The first call on each device looks up the array's device address on
 *     that device and keeps it; make that first call before any stream
 *     capture.  The address belongs to the device's primary context: after
 *     cudaDeviceReset (which destroys it) this entry point must not be called
 *     again in the process.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (different streams, or host threads) race on it and give wrong
 *     results.  Serialise them, e.g. on one stream.
 */
#define ADSX_NOALLOC_SCRATCH_BYTES (32 << 20)
int adsx_search_noalloc(const adsx_index *index, const float *Qv, int64_t nq,
                        int32_t K, int32_t nprobe, float eps0, int32_t delta_d,
                        int64_t *ids, float *dists, int64_t *dims_read,
                        void *stream);

/*
 * Serving: a continuous-batching request loop over adsx_search_batched.
 * A worker thread keeps up to n_streams batches in flight (one per CUDA
 * stream, so their work overlaps on the device).  Whenever a stream is free
 * it forms the next batch from the queue head: requests sharing the head's
 * (eps0, delta_d), as many as the free query slots (max_slots in flight),
 * max_batch and the device-memory budget allow (admission by memory: each
 * request is charged the device bytes its search needs).  The index stays
 * resident; per-request results return through pinned host buffers.
 *
 * adsx_server_create   index must outlive the server.  max_K / max_nprobe
 *                      bound every request.  ADSX_ENOMEM if staging fails.
 * adsx_server_submit   q: host, D float32 (copied).  Returns a ticket.
 *                      ADSX_ENOMEM if the request alone exceeds the budget.
 * adsx_server_wait     blocks up to timeout_ms (host wait, bounded) for the
 *                      ticket; copies K ids / dists (host) and dims_read (may
 *                      be NULL) and forgets the ticket.  ADSX_ETIMEOUT if not
 *                      done in time (the ticket stays valid), ADSX_EINVAL if
 *                      it was cancelled.
 * adsx_server_cancel   cancels a request that is still queued.
 * adsx_server_stats    latency percentiles (submit -> results on the host)
 *                      and throughput of completed requests since the last
 *                      reset, batches launched, the largest number of batches
 *                      and of queries in flight at once.
 */
typedef struct adsx_server adsx_server;
int adsx_server_create(const adsx_index *index, int32_t max_slots, int32_t max_batch,
                       int32_t n_streams, int64_t mem_budget_bytes, int32_t max_K,
                       int32_t max_nprobe, adsx_server **out);
int adsx_server_submit(adsx_server *server, const float *q, int32_t K, int32_t nprobe,
                       float eps0, int32_t delta_d, int64_t *ticket);
/* adsx_server_submit_many: n requests at once (host Q n x D, K[n], nprobe[n]),
 * all with one arrival time; tickets[n] receives their tickets. */
int adsx_server_submit_many(adsx_server *server, const float *Q, int64_t n, const int32_t *K,
                            const int32_t *nprobe, float eps0, int32_t delta_d,
                            int64_t *tickets);
int adsx_server_wait(adsx_server *server, int64_t ticket, int32_t timeout_ms,
                     int64_t *ids, float *dists, int64_t *dims_read);
int adsx_server_cancel(adsx_server *server, int64_t ticket);
int adsx_server_stats(adsx_server *server, double *p50_ms, double *p99_ms, double *qps,
                      int64_t *completed, int64_t *batches,
                      int64_t *max_inflight_batches, int64_t *max_inflight_queries);
int adsx_server_reset_stats(adsx_server *server);
int adsx_server_destroy(adsx_server *server);

/* Message of the last failure on the calling thread ("" if none). */
const char *adsx_last_error(void);

/* ------------------------------------------------------------------------
 * Graph-based search with ADSampling DCOs: HNSW+ (Sec. 4) -- the greedy beam
 * search HNSW runs on its base layer (Sec. 2.2.1) with Algorithm 1 as every
 * DCO -- on a kNN proximity graph over the vectors of an FP32 L2 (or cosine)
 * index.
 * ---------------------------------------------------------------------- */
typedef struct adsx_graph adsx_graph;

/*
 * adsx_build_graph -- vertex x's neighbours are its `degree` nearest other
 * vectors among the members of its nprobe nearest clusters (ties by id),
 * found with the library's own exact IVF search (adsx_search, eps0 = +INF).
 * HNSW's upper layers only locate a start vertex: a search starts from the
 * entry vertices of the query's nearest clusters instead.  A cluster's E =
 * entries_per_cluster entries are chosen by farthest-point sampling: entry 0
 * is its member nearest to the centroid, entry e its member whose squared
 * distance to the nearest of entries 0..e-1 is largest (ties by id; -1 once
 * that distance is 0, and for an empty cluster).  A k-means cluster can hold
 * parts of the kNN graph that no edge joins; E > 1 gives each a start, and a
 * larger E makes the entries a small upper layer (the query starts from the
 * nearest of them).  The
 * vectors themselves are read in place from the index, which must outlive
 * the graph.
 *   index    an FP32 index built with the L2 or the COSINE metric (ADSX_EINVAL
 *            otherwise); with COSINE the graph is the Euclidean one over the
 *            normalised vectors.
 *   X        host or device, N x D float32: the vectors the index was built from.
 *   degree   1..ADSX_MAX_DEGREE.   nprobe 1..min(nlist, ADSX_MAX_NPROBE).
 *   entries_per_cluster   1..ADSX_MAX_CLUSTER_ENTRIES.
 *   out      receives the graph (owns its device memory).
 * Errors: ADSX_EINVAL, ADSX_ENOMEM, ADSX_ECUDA.
 */
int adsx_build_graph(const adsx_index *index, const float *X, int32_t degree,
                     int32_t nprobe, int32_t entries_per_cluster, void *stream,
                     adsx_graph **out);

/* Frees the graph and its device memory (synchronises the device). */
int adsx_free_graph(adsx_graph *graph);

/* Shape of a graph: any output pointer may be NULL. */
int adsx_graph_info(const adsx_graph *graph, int64_t *N, int32_t *degree, int32_t *nlist,
                    int32_t *entries_per_cluster);

/* Copies the neighbour lists (N x degree int32, -1 = none) and the entry
 * vertices (nlist x entries_per_cluster int64, row-major, -1 = none) to host
 * or device memory (either pointer may be NULL). */
int adsx_graph_export(const adsx_graph *graph, int32_t *neighbors, int64_t *entries);

/*
 * adsx_search_graph -- HNSW+: greedy beam search with a result set R of ef
 * entries (Sec. 2.2.1).  The start vertices are all entry vertices of the
 * query's n_entry nearest clusters (vertex 0 if there are none), nearest
 * cluster first.  Every vertex not visited before, start vertex or
 * neighbour, runs Algorithm 1 against r = the largest distance in R (+INF
 * while R holds fewer than ef) and, if it reaches d = D with (distance, id)
 * below R's largest, joins R, which keeps its ef smallest -- in the paper's
 * order: one vertex at a time, each vertex facing R as it stands after the
 * vertices before it in the start list or neighbour list.  (The GPU tests
 * up to 32 vertices side by side against the threshold at their start and
 * then replays the decisions in list order from the recorded partial
 * distances, which gives the sequential outcome exactly; dims_read counts
 * the dims of the sequential order.)  The search repeatedly expands the
 * nearest not-yet-expanded entry of R.
 * The search stops when every entry of R is expanded, or after 4 ef
 * expansions.  The K smallest entries of R are returned, by (distance, id).
 * decoupled = 1 runs HNSW++ (Sec. 5.1) instead: R's two roles are split --
 * a set R1 of the K smallest exact distances gives every DCO its threshold
 * (R1's largest) and is returned, while R (size ef) and the expansions use
 * each DCO's observed distance (exact at d = D, else (D/d) S_d where
 * Algorithm 1 stopped).
 *   Qv, nq, ids, dists, dims_read, eps0, delta_d   as adsx_search
 *                (eps0 = +INF: exact DCOs, i.e. HNSW's own search); on a
 *                COSINE index queries are normalised and dists are cosine
 *                similarities 1 - d^2/2, largest first (-INF padding).
 *   K          1..ef.     ef 1..ADSX_MAX_EF.
 *   n_entry    1..min(nlist, ADSX_MAX_GRAPH_ENTRIES).
 * The graph keeps per-warp scratch for the visited test: searches on one
 * graph must not overlap on the GPU.
 * Errors: ADSX_EINVAL, ADSX_ENOMEM, ADSX_ECUDA.
 */
int adsx_search_graph(const adsx_index *index, const adsx_graph *graph, const float *Qv,
                      int64_t nq, int32_t K, int32_t ef, int32_t n_entry, int32_t decoupled,
                      float eps0, int32_t delta_d, int64_t *ids, float *dists,
                      int64_t *dims_read, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ADSX_H */
