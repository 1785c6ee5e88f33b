/*
 * adsx_oracle.c -- plain FP64 CPU reference for IVF + ADSampling
 * (Gao & Long, "High-Dimensional Approximate Nearest Neighbor Search: with
 * Reliable and Efficient Distance Comparison Operations", SIGMOD 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Everything is computed in double precision from the float32 inputs the GPU
 * library receives (the same X, P, centroids, assignments and queries), in the
 * order the paper states, with no blocking or reordering:
 *   - orc_rotate          Sec. 3.1: the transformed vector y := P' x.
 *   - orc_knn_exact       Sec. 2.1: exact KNN by brute force.
 *   - orc_probe           Sec. 2.2.2 (IVF): the N_probe nearest centroids.
 *   - orc_ivf_exact       Sec. 2.2.2 (IVF) with FDScanning DCOs.
 *   - orc_dco             Algorithm 1 (ADSampling) with the test of Sec. 3.2.
 *   - orc_ivf_ads         Sec. 4 (IVF+): IVF whose DCOs run Algorithm 1
 *                         against the current K-th distance of the KNN set.
 *   - orc_dco_fixed_r     Sec. 6.2.5: Algorithm 1 over a linear scan with a
 *                         fixed threshold per query (verification protocol).
 *   - orc_dco_pd,         Sec. 6.1: PDScanning, the exact partial-distance
 *     orc_ivf_pd          DCO of the IVF* / IVF** baselines.
 *   - orc_dco_ip,         Sec. 8, extension (1): inner-product DCOs reduced
 *     orc_ivf_exact_ip,   to Algorithm 1 on normalised vectors with a
 *     orc_ivf_ads_ip      per-object threshold; IVF for inner products.
 *     (Cosine similarity is the Euclidean case on normalised vectors, done
 *     in the Python wrapper.)
 *   - orc_graph_search    Sec. 2.2.1 / Sec. 4 (HNSW+): greedy beam search on
 *                         a proximity graph with Algorithm 1 DCOs against the
 *                         largest distance of the result set; Sec. 5.1
 *                         (HNSW++) with the result set's roles decoupled.
 *
 * Conventions (readings of points the paper leaves open):
 *   - distances are SQUARED Euclidean distances in the rotated space;
 *   - the hypothesis test is used in its squared form,
 *       reject  iff  D * S_d  >  r^2 * d * (1 + eps0/sqrt(d))^2,
 *     which equals dis' > (1 + eps0/sqrt(d)) r for dis', r >= 0 (Sec. 3.2);
 *   - d grows by delta_d per step, the last step may be shorter
 *     (d_j = min(j*delta_d, D)); no test at d = D (Algorithm 1, Case 3);
 *   - eps0 = +inf or r = +inf means "never reject" (no 0*inf);
 *   - the KNN set is totally ordered by (distance, id); a candidate enters
 *     iff it is positive and (dist, id) < the set's maximum (or the set has
 *     fewer than K members, whose maximum is +inf; Sec. 2.2.2);
 *   - clusters are visited in ascending (centroid distance, cluster id),
 *     members of a cluster in ascending id.
 *
 * Parity pins (see tests/test_oracle_*.py): brute force on tiny inputs,
 * permutation and orthogonal rotations, IVF with nprobe = nlist equals
 * exact KNN, eps0 = inf and delta_d >= D reduce IVF+ to IVF exactly, the
 * Beta law of a single rejection step (Lemma 3.1 made exact), hand-worked
 * boundary cases of the strict test, the Lemma 3.2 / 3.3 trends.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_REJECTED 0      /* Case 1: H0 rejected at some d < D            */
#define ORC_POSITIVE 1      /* Case 3: d = D and dis <= r                    */
#define ORC_NEGATIVE_AT_D 2 /* Case 3: d = D and dis > r                     */

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Sec. 3.1: y := P' x, with P' a D x D orthogonal matrix, row-major.      */
void orc_rotate(const float *P, int32_t D, const float *X, int64_t N,
                double *Y, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        const float *x = X + n * (int64_t)D;
        for (int32_t i = 0; i < D; ++i) {
            double s = 0.0;
            for (int32_t j = 0; j < D; ++j)
                s += (double)P[(int64_t)i * D + j] * (double)x[j];
            Y[n * (int64_t)D + i] = s;
        }
    }
}

static double sqdist(const double *a, const double *b, int32_t D)
{
    double s = 0.0;
    for (int32_t i = 0; i < D; ++i) {
        double t = a[i] - b[i];
        s += t * t;
    }
    return s;
}

typedef struct {
    double d;
    int64_t id;
} orc_pair;

static int pair_cmp(const void *pa, const void *pb)
{
    const orc_pair *a = (const orc_pair *)pa, *b = (const orc_pair *)pb;
    if (a->d < b->d) return -1;
    if (a->d > b->d) return 1;
    if (a->id < b->id) return -1;
    if (a->id > b->id) return 1;
    return 0;
}

/* (d1,i1) < (d2,i2) in the total order used for the KNN set. */
static int pair_less(double d1, int64_t i1, double d2, int64_t i2)
{
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

static void write_sorted(orc_pair *pairs, int64_t n, int32_t K,
                         int64_t *ids, double *d2)
{
    qsort(pairs, (size_t)n, sizeof(orc_pair), pair_cmp);
    for (int32_t k = 0; k < K; ++k) {
        if (k < n) {
            ids[k] = pairs[k].id;
            d2[k] = pairs[k].d;
        } else {
            ids[k] = -1;
            d2[k] = INFINITY;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Sec. 2.1: exact KNN -- all N distances, K smallest by (distance, id).   */
void orc_knn_exact(const double *Y, int64_t N, int32_t D, const double *Qr,
                   int64_t nq, int32_t K, int64_t *ids, double *d2,
                   int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(N > 0 ? N : 1));
        for (int64_t n = 0; n < N; ++n) {
            pairs[n].d = sqdist(Y + n * D, Qr + q * D, D);
            pairs[n].id = n;
        }
        write_sorted(pairs, N, K, ids + q * K, d2 + q * K);
        free(pairs);
    }
}

/* ---------------------------------------------------------------------- */
/* Sec. 2.2.2: the N_probe clusters whose centroids are nearest to q,     */
/* ordered by (centroid distance, cluster id).                            */
static void probe_one(const double *Cr, int32_t nlist, int32_t D,
                      const double *qr, int32_t nprobe, int32_t *probes,
                      double *pd2)
{
    orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)nlist);
    for (int32_t c = 0; c < nlist; ++c) {
        pairs[c].d = sqdist(Cr + (int64_t)c * D, qr, D);
        pairs[c].id = c;
    }
    qsort(pairs, (size_t)nlist, sizeof(orc_pair), pair_cmp);
    for (int32_t p = 0; p < nprobe; ++p) {
        probes[p] = (int32_t)pairs[p].id;
        if (pd2) pd2[p] = pairs[p].d;
    }
    free(pairs);
}

void orc_probe(const double *Cr, int32_t nlist, int32_t D, const double *Qr,
               int64_t nq, int32_t nprobe, int32_t *probes, double *pd2,
               int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q)
        probe_one(Cr, nlist, D, Qr + q * D, nprobe, probes + q * nprobe,
                  pd2 ? pd2 + q * nprobe : NULL);
}

/* Buckets of the inverted file: members of each cluster in ascending id. */
typedef struct {
    int64_t *start; /* nlist + 1 */
    int64_t *member;
} orc_buckets;

static orc_buckets make_buckets(const int32_t *assign, int64_t N, int32_t nlist)
{
    orc_buckets b;
    b.start = (int64_t *)calloc((size_t)nlist + 1, sizeof(int64_t));
    b.member = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t n = 0; n < N; ++n) b.start[assign[n] + 1] += 1;
    for (int32_t c = 0; c < nlist; ++c) b.start[c + 1] += b.start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nlist);
    for (int32_t c = 0; c < nlist; ++c) fill[c] = b.start[c];
    for (int64_t n = 0; n < N; ++n) b.member[fill[assign[n]]++] = n;
    free(fill);
    return b;
}

static void free_buckets(orc_buckets *b)
{
    free(b->start);
    free(b->member);
}

/* ---------------------------------------------------------------------- */
/* Sec. 2.2.2 with FDScanning (Sec. 2.1): exact distance of every         */
/* candidate of the probed clusters, K smallest by (distance, id).        */
void orc_ivf_exact(const double *Y, int64_t N, int32_t D, const double *Cr,
                   int32_t nlist, const int32_t *assign, const double *Qr,
                   int64_t nq, int32_t K, int32_t nprobe, int64_t *ids,
                   double *d2, int nthreads)
{
    orc_buckets b = make_buckets(assign, N, nlist);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        const double *qr = Qr + q * D;
        int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)nprobe);
        probe_one(Cr, nlist, D, qr, nprobe, probes, NULL);
        int64_t ncand = 0;
        for (int32_t p = 0; p < nprobe; ++p)
            ncand += b.start[probes[p] + 1] - b.start[probes[p]];
        orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(ncand > 0 ? ncand : 1));
        int64_t k = 0;
        for (int32_t p = 0; p < nprobe; ++p)
            for (int64_t m = b.start[probes[p]]; m < b.start[probes[p] + 1]; ++m) {
                int64_t id = b.member[m];
                pairs[k].d = sqdist(Y + id * D, qr, D);
                pairs[k].id = id;
                ++k;
            }
        write_sorted(pairs, ncand, K, ids + q * K, d2 + q * K);
        free(pairs);
        free(probes);
    }
    free_buckets(&b);
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 (ADSampling) for one DCO: object o', query q', threshold   */
/* r^2.  Samples delta_d more dimensions per step, updates the partial    */
/* squared distance S_d (so dis' = sqrt(D/d * S_d), Eq. 3), and tests     */
/* H0: dis <= r at every d < D (Sec. 3.2).  At d = D the comparison is    */
/* exact (Case 3).                                                         */
/*   returns ORC_REJECTED / ORC_POSITIVE / ORC_NEGATIVE_AT_D              */
/*   *dims   = number of dimensions sampled                                */
/*   *S_out  = S_d at termination (the exact squared distance if d = D)    */
/*   *margin = smallest |lhs/rhs - 1| over every comparison made, where    */
/*             lhs/rhs are the two sides of the test (or S_D vs r^2)      */
int orc_dco(const double *o, const double *q, int32_t D, double r2,
            double eps0, int32_t delta_d, int32_t *dims, double *S_out,
            double *margin)
{
    int32_t d = 0;
    double S = 0.0;
    double closest = INFINITY;
    int test_on = isfinite(eps0) && isfinite(r2);
    while (d < D) {
        int32_t dn = d + delta_d;
        if (dn > D) dn = D;
        for (int32_t i = d; i < dn; ++i) {
            double t = o[i] - q[i];
            S += t * t;
        }
        d = dn;
        if (d < D) {
            if (test_on) {
                double g = 1.0 + eps0 / sqrt((double)d);
                double lhs = (double)D * S;
                double rhs = r2 * (double)d * g * g;
                if (rhs > 0.0) {
                    double m = fabs(lhs / rhs - 1.0);
                    if (m < closest) closest = m;
                } else if (lhs == 0.0) {
                    closest = 0.0;
                }
                if (lhs > rhs) { /* Case 1 */
                    if (dims) *dims = d;
                    if (S_out) *S_out = S;
                    if (margin) *margin = closest;
                    return ORC_REJECTED;
                }
            }
            /* Case 2: continue sampling */
        }
    }
    /* Case 3: d = D, S is the exact squared distance. */
    if (isfinite(r2)) {
        if (r2 > 0.0) {
            double m = fabs(S / r2 - 1.0);
            if (m < closest) closest = m;
        } else if (S == 0.0) {
            closest = 0.0;
        }
    }
    if (dims) *dims = D;
    if (S_out) *S_out = S;
    if (margin) *margin = closest;
    return (S <= r2) ? ORC_POSITIVE : ORC_NEGATIVE_AT_D;
}

/* ---------------------------------------------------------------------- */
/* Sec. 4 (IVF+): IVF whose DCOs are Algorithm 1 against r = the current   */
/* K-th distance of the KNN set (r = +inf until it holds K objects).      */
/* Outputs ids/d2 sorted by (distance, id), -1/+inf padded, the total     */
/* number of dimensions sampled per query, and the number of candidates.  */
void orc_ivf_ads(const double *Y, int64_t N, int32_t D, const double *Cr,
                 int32_t nlist, const int32_t *assign, const double *Qr,
                 int64_t nq, int32_t K, int32_t nprobe, double eps0,
                 int32_t delta_d, int64_t *ids, double *d2,
                 int64_t *dims_total, int64_t *ncand_out, int nthreads)
{
    orc_buckets b = make_buckets(assign, N, nlist);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        const double *qr = Qr + q * D;
        int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)nprobe);
        probe_one(Cr, nlist, D, qr, nprobe, probes, NULL);
        /* KNN set: unordered array, its maximum found by a linear scan. */
        double *hd = (double *)malloc(sizeof(double) * (size_t)K);
        int64_t *hi = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
        int32_t count = 0;
        int64_t dims_sum = 0, ncand = 0;
        for (int32_t p = 0; p < nprobe; ++p) {
            for (int64_t m = b.start[probes[p]]; m < b.start[probes[p] + 1]; ++m) {
                int64_t id = b.member[m];
                int32_t imax = 0;
                double r2 = INFINITY;
                if (count == K) {
                    for (int32_t k = 1; k < K; ++k)
                        if (pair_less(hd[imax], hi[imax], hd[k], hi[k])) imax = k;
                    r2 = hd[imax];
                }
                int32_t dims = 0;
                double S = 0.0;
                int res = orc_dco(Y + id * D, qr, D, r2, eps0, delta_d, &dims, &S, NULL);
                dims_sum += dims;
                ncand += 1;
                if (res != ORC_POSITIVE) continue;
                if (count < K) {
                    hd[count] = S;
                    hi[count] = id;
                    ++count;
                } else if (pair_less(S, id, hd[imax], hi[imax])) {
                    hd[imax] = S;
                    hi[imax] = id;
                }
            }
        }
        orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(count > 0 ? count : 1));
        for (int32_t k = 0; k < count; ++k) {
            pairs[k].d = hd[k];
            pairs[k].id = hi[k];
        }
        write_sorted(pairs, count, K, ids + q * K, d2 + q * K);
        if (dims_total) dims_total[q] = dims_sum;
        if (ncand_out) ncand_out[q] = ncand;
        free(pairs);
        free(hd);
        free(hi);
        free(probes);
    }
    free_buckets(&b);
}

/* ---------------------------------------------------------------------- */
/* Sec. 6.2.5 verification protocol: Algorithm 1 on every (query, object)  */
/* pair of a linear scan with a FIXED threshold r2[q] per query, so the    */
/* DCOs are independent.  decisions/dims/margins are nq x N, object order. */
void orc_dco_fixed_r(const double *Y, int64_t N, int32_t D, const double *Qr,
                     int64_t nq, const double *r2, double eps0,
                     int32_t delta_d, uint8_t *decisions, int32_t *dims,
                     double *margins, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        for (int64_t n = 0; n < N; ++n) {
            int32_t dd = 0;
            double m = 0.0;
            int res = orc_dco(Y + n * D, Qr + q * D, D, r2[q], eps0, delta_d,
                              &dd, NULL, &m);
            decisions[q * N + n] = (uint8_t)res;
            if (dims) dims[q * N + n] = dd;
            if (margins) margins[q * N + n] = m;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* PDScanning (Sec. 6.1, the IVF* / IVF** baseline): scan dimensions in     */
/* steps of delta_d and stop as soon as the partial squared distance S_d    */
/* exceeds r^2 -- an exact DCO (S_d <= S_D, so a positive is never          */
/* stopped).  Same outputs as orc_dco (decision, dims, S, margin).          */
int orc_dco_pd(const double *o, const double *q, int32_t D, double r2, int32_t delta_d,
               int32_t *dims, double *S_out)
{
    int32_t d = 0;
    double S = 0.0;
    while (d < D) {
        int32_t dn = d + delta_d;
        if (dn > D) dn = D;
        for (int32_t i = d; i < dn; ++i) {
            double t = o[i] - q[i];
            S += t * t;
        }
        d = dn;
        if (d < D && S > r2) {
            if (dims) *dims = d;
            if (S_out) *S_out = S;
            return ORC_REJECTED;
        }
    }
    if (dims) *dims = D;
    if (S_out) *S_out = S;
    return (S <= r2) ? ORC_POSITIVE : ORC_NEGATIVE_AT_D;
}

/* IVF* (Sec. 6.1): IVF whose DCOs are PDScanning against the current K-th  */
/* distance; returns exactly the IVF result, with fewer dimensions read.    */
void orc_ivf_pd(const double *Y, int64_t N, int32_t D, const double *Cr, int32_t nlist,
                const int32_t *assign, const double *Qr, int64_t nq, int32_t K,
                int32_t nprobe, int32_t delta_d, int64_t *ids, double *d2,
                int64_t *dims_total, int nthreads)
{
    orc_buckets b = make_buckets(assign, N, nlist);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        const double *qr = Qr + q * D;
        int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)nprobe);
        probe_one(Cr, nlist, D, qr, nprobe, probes, NULL);
        double *hd = (double *)malloc(sizeof(double) * (size_t)K);
        int64_t *hi = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
        int32_t count = 0;
        int64_t dims_sum = 0;
        for (int32_t p = 0; p < nprobe; ++p) {
            for (int64_t m = b.start[probes[p]]; m < b.start[probes[p] + 1]; ++m) {
                int64_t id = b.member[m];
                int32_t imax = 0;
                double r2 = INFINITY;
                if (count == K) {
                    for (int32_t k = 1; k < K; ++k)
                        if (pair_less(hd[imax], hi[imax], hd[k], hi[k])) imax = k;
                    r2 = hd[imax];
                }
                int32_t dims = 0;
                double S = 0.0;
                int res = orc_dco_pd(Y + id * D, qr, D, r2, delta_d, &dims, &S);
                dims_sum += dims;
                if (res != ORC_POSITIVE) continue;
                if (count < K) {
                    hd[count] = S;
                    hi[count] = id;
                    ++count;
                } else if (pair_less(S, id, hd[imax], hi[imax])) {
                    hd[imax] = S;
                    hi[imax] = id;
                }
            }
        }
        orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(count > 0 ? count : 1));
        for (int32_t k = 0; k < count; ++k) {
            pairs[k].d = hd[k];
            pairs[k].id = hi[k];
        }
        write_sorted(pairs, count, K, ids + q * K, d2 + q * K);
        if (dims_total) dims_total[q] = dims_sum;
        free(pairs);
        free(hd);
        free(hi);
        free(probes);
    }
    free_buckets(&b);
}

/* ---------------------------------------------------------------------- */
/* Inner product (Sec. 8, extension (1)).  <o,q> >= r holds iff            */
/*     || o/||o|| - q/||q|| ||^2  <=  2 - 2 r / (||o|| ||q||),              */
/* so the DCO "is <o,q> at least r?" is Algorithm 1 on the normalised      */
/* vectors against the per-object squared threshold                        */
/*     tau = 2 - 2 r / (||o|| ||q||).                                       */
/* Readings: r = -inf (fewer than K objects held) gives tau = +inf (never  */
/* reject); tau < 0 means <o,q> <= ||o|| ||q|| < r, a negative decided     */
/* without sampling (dims 0); a zero-norm o or q has <o,q> = 0, decided    */
/* exactly (positive iff 0 >= r, dims D).  *ip_out is <o,q> computed       */
/* directly; o, q are rotated vectors (rotation preserves both norms and   */
/* inner products).                                                        */
static double dot(const double *a, const double *b, int32_t D)
{
    double s = 0.0;
    for (int32_t i = 0; i < D; ++i) s += a[i] * b[i];
    return s;
}

int orc_dco_ip(const double *o, const double *q, int32_t D, double r,
               double eps0, int32_t delta_d, int32_t *dims, double *ip_out,
               double *margin)
{
    const double no = sqrt(dot(o, o, D)), nq = sqrt(dot(q, q, D));
    const double ip = dot(o, q, D);
    if (ip_out) *ip_out = ip;
    if (no == 0.0 || nq == 0.0) {
        if (dims) *dims = D;
        if (margin) *margin = INFINITY;
        return (0.0 >= r) ? ORC_POSITIVE : ORC_NEGATIVE_AT_D;
    }
    const double tau = isinf(r) && r < 0 ? INFINITY : 2.0 - 2.0 * r / (no * nq);
    if (tau < 0.0) {
        if (dims) *dims = 0;
        if (margin) *margin = INFINITY;
        return ORC_REJECTED;
    }
    double *oh = (double *)malloc(sizeof(double) * (size_t)D);
    double *qh = (double *)malloc(sizeof(double) * (size_t)D);
    for (int32_t i = 0; i < D; ++i) {
        oh[i] = o[i] / no;
        qh[i] = q[i] / nq;
    }
    int res = orc_dco(oh, qh, D, tau, eps0, delta_d, dims, NULL, margin);
    free(oh);
    free(qh);
    return res;
}

/* IVF for inner products: the N_probe clusters with the largest <c, q>    */
/* (ties by cluster id), then the K largest <o, q> (ties by id) among     */
/* their members.  Pairs hold -<.,q> so the ascending order of orc_pair   */
/* is the descending order of inner products.                             */
static void probe_one_ip(const double *Cr, int32_t nlist, int32_t D,
                         const double *qr, int32_t nprobe, int32_t *probes)
{
    orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)nlist);
    for (int32_t c = 0; c < nlist; ++c) {
        pairs[c].d = -dot(Cr + (int64_t)c * D, qr, D);
        pairs[c].id = c;
    }
    qsort(pairs, (size_t)nlist, sizeof(orc_pair), pair_cmp);
    for (int32_t p = 0; p < nprobe; ++p) probes[p] = (int32_t)pairs[p].id;
    free(pairs);
}

static void write_sorted_ip(orc_pair *pairs, int64_t n, int32_t K, int64_t *ids, double *ips)
{
    write_sorted(pairs, n, K, ids, ips);
    for (int32_t k = 0; k < K; ++k) ips[k] = (k < n) ? -ips[k] : -INFINITY;
}

void orc_ivf_exact_ip(const double *Y, int64_t N, int32_t D, const double *Cr,
                      int32_t nlist, const int32_t *assign, const double *Qr,
                      int64_t nq, int32_t K, int32_t nprobe, int64_t *ids,
                      double *ips, int nthreads)
{
    orc_buckets b = make_buckets(assign, N, nlist);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        const double *qr = Qr + q * D;
        int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)nprobe);
        probe_one_ip(Cr, nlist, D, qr, nprobe, probes);
        int64_t ncand = 0;
        for (int32_t p = 0; p < nprobe; ++p)
            ncand += b.start[probes[p] + 1] - b.start[probes[p]];
        orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(ncand > 0 ? ncand : 1));
        int64_t k = 0;
        for (int32_t p = 0; p < nprobe; ++p)
            for (int64_t m = b.start[probes[p]]; m < b.start[probes[p] + 1]; ++m) {
                int64_t id = b.member[m];
                pairs[k].d = -dot(Y + id * D, qr, D);
                pairs[k].id = id;
                ++k;
            }
        write_sorted_ip(pairs, ncand, K, ids + q * K, ips + q * K);
        free(pairs);
        free(probes);
    }
    free_buckets(&b);
}

/* IVF+ for inner products: sequential IVF whose DCOs are orc_dco_ip       */
/* against r = the K-th largest inner product held (-inf until K are).    */
void orc_ivf_ads_ip(const double *Y, int64_t N, int32_t D, const double *Cr,
                    int32_t nlist, const int32_t *assign, const double *Qr,
                    int64_t nq, int32_t K, int32_t nprobe, double eps0,
                    int32_t delta_d, int64_t *ids, double *ips,
                    int64_t *dims_total, int64_t *ncand_out, int nthreads)
{
    orc_buckets b = make_buckets(assign, N, nlist);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        const double *qr = Qr + q * D;
        int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)nprobe);
        probe_one_ip(Cr, nlist, D, qr, nprobe, probes);
        /* KNN set of (-<o,q>, id): unordered array, maximum by linear scan. */
        double *hd = (double *)malloc(sizeof(double) * (size_t)K);
        int64_t *hi = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
        int32_t count = 0;
        int64_t dims_sum = 0, ncand = 0;
        for (int32_t p = 0; p < nprobe; ++p) {
            for (int64_t m = b.start[probes[p]]; m < b.start[probes[p] + 1]; ++m) {
                int64_t id = b.member[m];
                int32_t imax = 0;
                double r = -INFINITY;
                if (count == K) {
                    for (int32_t k = 1; k < K; ++k)
                        if (pair_less(hd[imax], hi[imax], hd[k], hi[k])) imax = k;
                    r = -hd[imax];
                }
                int32_t dims = 0;
                double ip = 0.0;
                int res = orc_dco_ip(Y + id * D, qr, D, r, eps0, delta_d, &dims, &ip, NULL);
                dims_sum += dims;
                ncand += 1;
                if (res != ORC_POSITIVE) continue;
                if (count < K) {
                    hd[count] = -ip;
                    hi[count] = id;
                    ++count;
                } else if (pair_less(-ip, id, hd[imax], hi[imax])) {
                    hd[imax] = -ip;
                    hi[imax] = id;
                }
            }
        }
        orc_pair *pairs = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(count > 0 ? count : 1));
        for (int32_t k = 0; k < count; ++k) {
            pairs[k].d = hd[k];
            pairs[k].id = hi[k];
        }
        write_sorted_ip(pairs, count, K, ids + q * K, ips + q * K);
        if (dims_total) dims_total[q] = dims_sum;
        if (ncand_out) ncand_out[q] = ncand;
        free(pairs);
        free(hd);
        free(hi);
        free(probes);
    }
    free_buckets(&b);
}

/* ---------------------------------------------------------------------- */
/* Sec. 2.2.1 / Sec. 4 (HNSW+): greedy beam search on a proximity graph    */
/* whose DCOs run Algorithm 1 against the largest distance of the result  */
/* set R (size N_ef), in the paper's order: one vertex at a time, R (and   */
/* with it the threshold) updated after every vertex.  The search set S is */
/* the set of R's entries not yet expanded (an entry leaving R has a       */
/* distance above R's maximum, which would stop the search, so it can      */
/* never be expanded usefully).  The start vertices are visited first, in  */
/* list order, like neighbours of a virtual root; then each iteration      */
/* expands R's nearest unexpanded entry and visits its neighbours in list  */
/* order, skipping -1 and vertices visited before.  A vertex whose DCO is  */
/* positive (d = D, S_D <= r^2) joins R when (S_D, id) precedes R's        */
/* maximum (or R is not full), R keeping its N_ef smallest by (d, id).      */
/* The search stops when every entry of R is expanded (or after max_iter   */
/* expansions).                                                             */
/*   graph     N x Rg int32 neighbour ids (-1 = none), by original id      */
/*   entries   nq x E int64 start vertices (-1 = none)                    */
/* Outputs ids/d2 (K smallest of R by (distance, id); -1/+inf padded),    */
/* the dims sampled and the expansions per query, and (margin_out, may be */
/* NULL) the query's closest call: the smallest relative gap over every   */
/* DCO comparison (orc_dco's margin), every comparison of a new key with   */
/* the largest of R (or R1) that decided an insertion, and every choice of */
/* the entry to expand (R's nearest unexpanded entry against the next      */
/* one) -- a query whose closest call is below a tolerance may take        */
/* another path under another rounding (the order of the returned keys    */
/* among themselves is not included: it does not steer the search).       */
/* pp = 1: HNSW++ (Sec. 5.1) -- R's two roles decoupled: R1 (size K, exact  */
/* distances) holds the results and gives every DCO its threshold (R1's   */
/* largest distance); R (size N_ef) and S are kept with the observed      */
/* distance of each DCO: exact if it reached d = D, else the estimate     */
/* (D/d) S_d at the d where Algorithm 1 stopped.  The output is R1.       */
typedef struct {
    const double *Y, *qr;
    int32_t D, K, ef, delta_d, pp;
    double eps0;
    unsigned char *visited, *expd;
    orc_pair *R, *R1;
    int32_t nR, n1;
    int64_t dims_sum;
    double closest;
} orc_beam;

static void orc_note_gap(orc_beam *b, double x, double y)
{
    if (!isfinite(x) || !isfinite(y)) return;
    const double m = fabs(x) > fabs(y) ? fabs(x) : fabs(y);
    const double g = m > 0.0 ? fabs(x - y) / m : 0.0;
    if (g < b->closest) b->closest = g;
}

/* Inserts (d, id) into the sorted set A[0..*n) of capacity cap (flags: the
   expanded flags carried along, may be NULL), dropping the largest when
   full.  The caller has checked that it belongs there. */
static void orc_set_insert(orc_beam *b, orc_pair *A, unsigned char *flags, int32_t *n,
                           int32_t cap, double d, int64_t id)
{
    int32_t p = *n < cap ? *n : cap - 1;        /* slot freed at the end */
    while (p > 0 && pair_less(d, id, A[p - 1].d, A[p - 1].id)) {
        A[p] = A[p - 1];
        if (flags) flags[p] = flags[p - 1];
        --p;
    }
    A[p].d = d;
    A[p].id = id;
    if (flags) flags[p] = 0;
    if (*n < cap) ++*n;
}

/* One vertex: its DCO against the current threshold, then R (and R1). */
static void orc_beam_visit(orc_beam *b, int64_t v)
{
    if (v < 0 || b->visited[v]) return;
    b->visited[v] = 1;
    const int full = b->nR == b->ef, full1 = b->n1 == b->K;
    const double rmax = full ? b->R[b->nR - 1].d : INFINITY;
    const int64_t rid = full ? b->R[b->nR - 1].id : INT64_MAX;
    const double r1max = full1 ? b->R1[b->n1 - 1].d : INFINITY;
    const int64_t r1id = full1 ? b->R1[b->n1 - 1].id : INT64_MAX;
    const double r2 = b->pp ? r1max : rmax;        /* the DCO threshold */
    const int32_t D = b->D;
    int32_t dims = 0;
    double S = 0.0, mar = INFINITY;
    const int res = orc_dco(b->Y + v * D, b->qr, D, r2, b->eps0, b->delta_d, &dims, &S, &mar);
    b->dims_sum += dims;
    if (mar < b->closest) b->closest = mar;
    if (!b->pp) {
        if (res != ORC_POSITIVE) return;
        if (full) orc_note_gap(b, S, rmax);
        if (!full || pair_less(S, v, rmax, rid))
            orc_set_insert(b, b->R, b->expd, &b->nR, b->ef, S, v);
        return;
    }
    const double obs = dims == D ? S : S * (double)D / (double)dims;
    if (res == ORC_POSITIVE) {
        if (full1) orc_note_gap(b, S, r1max);
        if (!full1 || pair_less(S, v, r1max, r1id))
            orc_set_insert(b, b->R1, NULL, &b->n1, b->K, S, v);
    }
    if (full) orc_note_gap(b, obs, rmax);
    if (!full || pair_less(obs, v, rmax, rid))
        orc_set_insert(b, b->R, b->expd, &b->nR, b->ef, obs, v);
}

void orc_graph_search(const double *Y, int64_t N, int32_t D, const int32_t *graph,
                      int32_t Rg, const int64_t *entries, int32_t E, const double *Qr,
                      int64_t nq, int32_t K, int32_t ef, int32_t max_iter, double eps0,
                      int32_t delta_d, int32_t pp, int64_t *ids, double *d2,
                      int64_t *dims_total, int64_t *iters_out, double *margin_out,
                      int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int64_t q = 0; q < nq; ++q) {
        orc_beam b;
        b.Y = Y;
        b.qr = Qr + q * D;
        b.D = D;
        b.K = K;
        b.ef = ef;
        b.delta_d = delta_d;
        b.pp = pp;
        b.eps0 = eps0;
        b.visited = (unsigned char *)calloc((size_t)(N > 0 ? N : 1), 1);
        b.R = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)ef);
        b.expd = (unsigned char *)malloc((size_t)ef);
        b.R1 = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)K);
        b.nR = 0;
        b.n1 = 0;
        b.dims_sum = 0;
        b.closest = INFINITY;
        int32_t it = 0;
        for (int32_t k = 0; k < E; ++k) orc_beam_visit(&b, entries[q * E + k]);
        while (it < max_iter) {
            int32_t u = -1;
            for (int32_t k = 0; k < b.nR; ++k)
                if (!b.expd[k]) { u = k; break; }
            if (u < 0) break;
            /* which entry is expanded: R's nearest unexpanded one, against
               the next unexpanded one */
            for (int32_t k = u + 1; k < b.nR; ++k)
                if (!b.expd[k]) { orc_note_gap(&b, b.R[u].d, b.R[k].d); break; }
            b.expd[u] = 1;
            const int64_t node = b.R[u].id;
            for (int32_t j = 0; j < Rg; ++j) orc_beam_visit(&b, graph[node * Rg + j]);
            ++it;
        }
        const orc_pair *res = pp ? b.R1 : b.R;
        const int32_t nres = pp ? b.n1 : b.nR;
        for (int32_t k = 0; k < K; ++k) {
            ids[q * K + k] = k < nres ? res[k].id : -1;
            d2[q * K + k] = k < nres ? res[k].d : INFINITY;
        }
        if (dims_total) dims_total[q] = b.dims_sum;
        if (iters_out) iters_out[q] = it;
        if (margin_out) margin_out[q] = b.closest;
        free(b.R1);
        free(b.expd);
        free(b.R);
        free(b.visited);
    }
}
