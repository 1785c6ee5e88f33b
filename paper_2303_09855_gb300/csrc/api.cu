// api.cu -- the C ABI declared in include/adsx.h: argument checks, index
// construction (host CSR build + device rotation and layout scatter) and the
// search pipeline (rotate -> centroid distances -> top-nprobe -> scan), all
// enqueued on the caller's stream.  Temporary device buffers come from the
// library's own stream-ordered memory pool (cudaMallocFromPoolAsync /
// cudaFreeAsync), which keeps its memory between calls.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "adsx_internal.cuh"

using adsx::Index;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation)
        return fail(ADSX_ENOMEM, "%s: out of device memory", what);
    return fail(ADSX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The library's stream-ordered memory pool on the current device, created
// on first use with no release threshold: memory freed by a search stays in
// the pool for the next one.  (The device's default pool hands freed memory
// back to the system at every synchronisation, so each search would map its
// temporaries -- 164 MB of centroid distances for 10k queries x 4096
// clusters -- afresh, on the host's critical path.)  NULL if no pool can be
// made: the default pool is used then.
cudaMemPool_t scratch_pool()
{
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[MAXDEV] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t mp = nullptr;
        if (cudaMemPoolCreate(&mp, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        if (cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaGetLastError();
            cudaMemPoolDestroy(mp);
            return nullptr;
        }
        pools[dev] = mp;
    }
    return pools[dev];
}

// Stream-ordered scratch buffers, released on the stream when the scope ends.
// While the stream is being captured into a CUDA graph the allocations are
// left to the graph (cudaMallocAsync becomes a graph allocation node).
struct Scratch {
    cudaStream_t s;
    cudaMemPool_t pool = nullptr;
    std::vector<void *> bufs;
    explicit Scratch(cudaStream_t st) : s(st)
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cudaGetLastError();
        if (cs == cudaStreamCaptureStatusNone) pool = scratch_pool();
    }
    ~Scratch()
    {
        for (void *p : bufs) cudaFreeAsync(p, s);
    }
    template <typename T>
    cudaError_t get(T **out, size_t count)
    {
        void *p = nullptr;
        const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s)
                             : cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) return e;
        bufs.push_back(p);
        *out = static_cast<T *>(p);
        return cudaSuccess;
    }
};

// A caller buffer of `count` T: used in place when it is device memory, else
// staged through a scratch buffer (inputs copied in now, outputs copied out by
// finish()).
template <typename T>
struct Buf {
    T *dev = nullptr;
    T *host = nullptr;
    size_t count = 0;
};

template <typename T>
cudaError_t stage_in(Scratch &sc, const T *user, size_t count, Buf<T> &b)
{
    b.count = count;
    if (is_device_ptr(user)) {
        b.dev = const_cast<T *>(user);
        return cudaSuccess;
    }
    cudaError_t e = sc.get(&b.dev, count);
    if (e != cudaSuccess) return e;
    if (count) e = cudaMemcpyAsync(b.dev, user, count * sizeof(T), cudaMemcpyHostToDevice, sc.s);
    return e;
}

template <typename T>
cudaError_t stage_out(Scratch &sc, T *user, size_t count, Buf<T> &b)
{
    b.count = count;
    if (!user) return cudaSuccess;
    if (is_device_ptr(user)) {
        b.dev = user;
        return cudaSuccess;
    }
    b.host = user;
    return sc.get(&b.dev, count);
}

template <typename T>
cudaError_t copy_back(const Buf<T> &b, cudaStream_t s)
{
    if (!b.host || !b.count) return cudaSuccess;
    return cudaMemcpyAsync(b.host, b.dev, b.count * sizeof(T), cudaMemcpyDeviceToHost, s);
}

int check_index(const Index *ix)
{
    if (!ix) return fail(ADSX_EINVAL, "index is NULL");
    cudaError_t e = cudaSetDevice(ix->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return ADSX_OK;
}

// q' = P q for nq raw queries into a Dp-strided buffer (zero padded dims).
// Query rotation q' = P q (Sec. 3.1): on the tensor cores, exactly up to the
// final rounding, when the index has P's digits and that mode is on
// (adsx_set_query_rotation); else the compensated FP32 (or Kac) rotation.
cudaError_t rotate_queries(const Index *ix, const float *q_dev, int64_t nq, float *qrot,
                           Scratch &sc)
{
    if (ix->rot_tc && nq > 0) {
        float *part = nullptr;
        int32_t *xexp = nullptr;
        const int64_t pf = adsx::tc_rot_scratch_floats(ix, nq);
        cudaError_t e = sc.get(&part, (size_t)pf);
        if (e == cudaSuccess) e = sc.get(&xexp, (size_t)nq);
        if (e != cudaSuccess) return e;
        return adsx::rotate_queries_tc(ix, q_dev, nq, qrot, part, pf, xexp, sc.s);
    }
    return adsx::rotate_rows(ix, q_dev, nq, qrot, sc.s);
}

// ||q'-c'||^2 for every (query, centroid) as ||q'||^2 + ||c'||^2 - 2 q'.c',
// with the tile summary of the result for the top-nprobe select when
// `summary` is not NULL.
cudaError_t centroid_distances(const Index *ix, const float *qrot, int64_t nq, float *dist,
                               Scratch &sc, unsigned *summary = nullptr)
{
    float *qn = nullptr;
    uint32_t *qs = nullptr;
    cudaError_t e = sc.get(&qn, (size_t)nq);
    if (e == cudaSuccess) e = sc.get(&qs, (size_t)adsx::tf32_split_words(nq, ix->Dp));
    if (e != cudaSuccess) return e;
    e = adsx::launch_row_sqnorm(qrot, nq, ix->Dp, ix->Dp, qn, sc.s);
    if (e == cudaSuccess) e = adsx::launch_tf32_split(qrot, nq, ix->Dp, ix->Dp, qs, sc.s);
    if (e != cudaSuccess) return e;
    return adsx::launch_tc_gemm(qs, nq, ix->cents_split, ix->Dp, dist, ix->nlist, ix->nlist, qn,
                                ix->cnorm, ix->err, sc.s, summary);
}

// The tile summary (four entries per 128 centroids) is written for the
// select when it can bound the nprobe-th distance of a row from at least
// twice nprobe entries; the select uses it for rows with nprobe <= 64.
cudaError_t probe_summary(const Index *ix, int64_t nq, int nprobe, Scratch &sc, unsigned **summary)
{
    *summary = nullptr;
    const int64_t ntiles = (ix->nlist + adsx::SUMMARY_TILE - 1) / adsx::SUMMARY_TILE;
    if (4 * ntiles < 2 * (int64_t)std::min(nprobe, 64)) return cudaSuccess;
    return sc.get(summary, (size_t)(nq * ntiles * 4));
}

// Stage timing: an event before (begin) or after (end) a scan-kernel launch.
cudaError_t mark_kernel(const Index *ix, bool begin, cudaStream_t s)
{
    if (!ix->timing) return cudaSuccess;
    Index *w = const_cast<Index *>(ix);
    if (w->nkev >= Index::MAX_KEV) return cudaSuccess;
    cudaError_t e = cudaEventRecord(w->kev[2 * w->nkev + (begin ? 0 : 1)], s);
    if (!begin) ++w->nkev;
    return e;
}

cudaError_t mark(const Index *ix, int i, cudaStream_t s)
{
    if (!ix->timing) return cudaSuccess;
    return cudaEventRecord(ix->ev[i], s);
}

cudaError_t probe_queries(const Index *ix, const float *qrot, int64_t nq, int nprobe,
                          int32_t *probes, float *pd2, Scratch &sc)
{
    float *dist = nullptr;
    unsigned *summ = nullptr;
    cudaError_t e = sc.get(&dist, (size_t)nq * ix->nlist);
    if (e == cudaSuccess) e = probe_summary(ix, nq, nprobe, sc, &summ);
    if (e != cudaSuccess) return e;
    e = centroid_distances(ix, qrot, nq, dist, sc, summ);
    if (e != cudaSuccess) return e;
    if ((e = mark(ix, 2, sc.s)) != cudaSuccess) return e;
    return adsx::launch_select_nprobe(dist, nq, ix->nlist, nprobe, probes, pd2, sc.s, nullptr, summ);
}

// Sec. 8, extension (1): cosine queries are scaled to unit norm before the
// centroid ranking (the centroids are); inner-product queries are ranked raw
// (largest <c, q>) and scaled afterwards, keeping ||q|| for the per-object
// thresholds and the returned inner products.
cudaError_t queries_before_probe(const Index *ix, float *qrot, int64_t nq, cudaStream_t s)
{
    if (ix->metric != ADSX_COSINE) return cudaSuccess;
    return adsx::launch_normalize_rows(qrot, nq, ix->Dp, ix->Dp, nullptr, nullptr, s);
}

cudaError_t queries_after_probe(const Index *ix, float *qrot, int64_t nq, Scratch &sc,
                                float **qnorm)
{
    *qnorm = nullptr;
    if (ix->metric != ADSX_IP) return cudaSuccess;
    cudaError_t e = sc.get(qnorm, (size_t)nq);
    if (e != cudaSuccess) return e;
    return adsx::launch_normalize_rows(qrot, nq, ix->Dp, ix->Dp, *qnorm, nullptr, sc.s);
}

int finish(cudaStream_t s, bool any_host, const char *what)
{
    if (!any_host) return ADSX_OK;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return ADSX_OK;
}

int check_blocks(int32_t delta_d, float eps0)
{
    if (delta_d < 16 || (delta_d % 16) != 0)
        return fail(ADSX_EINVAL, "delta_d must be a positive multiple of 16 (got %d)", delta_d);
    if (!(eps0 >= 0.f)) return fail(ADSX_EINVAL, "eps0 must be >= 0 (got %g)", (double)eps0);
    return ADSX_OK;
}

}  // namespace

namespace adsx {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace adsx

extern "C" {

const char *adsx_last_error(void) { return g_last_error.c_str(); }

// The rotation is either a dense P (kac_L = 0) or a layered Kac walk.
// The P side of the tensor-core query rotation (gemm_tc.cu): every row c of
// P split into T signed b-bit digits of V = trunc(P[c][k] 2^(bT - F_c)) (F_c
// the exponent of the row's largest |P[c][k]|), laid out per level
// L = 2..Lmax as a Dp x n_L Dp matrix whose row c holds, in block j, digit
// L - t of the row for t = max(1, L - T) + j (n_L = the level's digit pairs).
// Host code, once per index.
static void rot_slices_host(const float *P, int D, int Dp, int b, int T, int Lmax,
                            std::vector<float> &B, std::vector<int32_t> &F, int64_t *boff)
{
    const long long mask = (1ll << b) - 1;
    std::vector<int32_t> dig((size_t)T * Dp * Dp, 0);
    F.assign((size_t)Dp, 0);
    for (int c = 0; c < D; ++c) {
        double m = 0.0;
        for (int k = 0; k < D; ++k) m = std::max(m, fabs((double)P[(size_t)c * D + k]));
        int E = 0;
        if (m > 0.0) frexp(m, &E);
        F[c] = E;
        for (int k = 0; k < D; ++k) {
            const long long V = (long long)trunc(ldexp((double)P[(size_t)c * D + k], b * T - E));
            const long long av = V < 0 ? -V : V;
            for (int u = 1; u <= T; ++u) {
                const long long d = (av >> (b * (T - u))) & mask;
                dig[((size_t)(u - 1) * Dp + c) * Dp + k] = (int32_t)(V < 0 ? -d : d);
            }
        }
    }
    int64_t total = 0;
    for (int L = 0; L < 16; ++L) boff[L] = 0;
    for (int L = 2; L <= Lmax; ++L) {
        const int lo = std::max(1, L - T), hi = std::min(T, L - 1);
        boff[L] = total;
        total += (int64_t)(hi - lo + 1) * Dp * Dp;
    }
    B.assign((size_t)total, 0.f);
    for (int L = 2; L <= Lmax; ++L) {
        const int lo = std::max(1, L - T), hi = std::min(T, L - 1);
        const int64_t ld = (int64_t)(hi - lo + 1) * Dp;
        for (int c = 0; c < Dp; ++c)
            for (int t = lo; t <= hi; ++t) {
                const int u = L - t;
                for (int k = 0; k < Dp; ++k)
                    B[(size_t)(boff[L] + c * ld + (int64_t)(t - lo) * Dp + k)] =
                        (float)dig[((size_t)(u - 1) * Dp + c) * Dp + k];
            }
    }
}

static int build_impl(const float *X, int64_t N, int32_t D, const float *P,
                      const int32_t *kac_pairs, const float *kac_cs, int32_t kac_L,
                      const float *centroids, int32_t nlist, const int32_t *assign,
                      int32_t storage, int32_t metric, void *stream, adsx_index **out)
{
    if (!out) return fail(ADSX_EINVAL, "out is NULL");
    *out = nullptr;
    if (metric != ADSX_L2 && metric != ADSX_IP && metric != ADSX_COSINE)
        return fail(ADSX_EINVAL, "metric %d not supported", metric);
    const bool kac = kac_L != 0;
    if (!X || (!kac && !P) || !centroids || !assign) return fail(ADSX_EINVAL, "NULL input pointer");
    if (kac) {
        if (kac_L < 1 || kac_L > ADSX_MAX_KAC_LAYERS)
            return fail(ADSX_EINVAL, "Kac walk layers out of range (1..%d)", ADSX_MAX_KAC_LAYERS);
        if (!kac_pairs || !kac_cs) return fail(ADSX_EINVAL, "NULL Kac walk");
        if (is_device_ptr(kac_pairs) || is_device_ptr(kac_cs))
            return fail(ADSX_EINVAL, "the Kac walk takes host pointers");
        if (D >= 1 && D <= ADSX_MAX_D) {
            const int m = D / 2;
            std::vector<int32_t> stamp((size_t)D, -1);
            for (int32_t l = 0; l < kac_L; ++l)
                for (int t = 0; t < 2 * m; ++t) {
                    const int32_t i = kac_pairs[(size_t)l * 2 * m + t];
                    if (i < 0 || i >= D || stamp[(size_t)i] == l)
                        return fail(ADSX_EINVAL, "Kac walk layer %d: index %d out of range or repeated", l, i);
                    stamp[(size_t)i] = l;
                }
            for (size_t k = 0; k < (size_t)kac_L * m; ++k) {
                const double c = kac_cs[2 * k], sn = kac_cs[2 * k + 1];
                if (!(fabs(c * c + sn * sn - 1.0) <= 1e-5))
                    return fail(ADSX_EINVAL, "Kac walk pair %zu: c^2 + s^2 != 1", k);
            }
        }
    }
    if (N < 1 || N >= (int64_t)1 << 31) return fail(ADSX_EINVAL, "N out of range");
    if (D < 1 || D > ADSX_MAX_D) return fail(ADSX_EINVAL, "D out of range (1..%d)", ADSX_MAX_D);
    if (nlist < 1 || nlist > ADSX_MAX_NLIST || nlist > N)
        return fail(ADSX_EINVAL, "nlist out of range (1..min(N, %d))", ADSX_MAX_NLIST);
    if (storage != ADSX_F32 && storage != ADSX_BF16 && storage != ADSX_F16)
        return fail(ADSX_EINVAL, "storage type %d not supported", storage);
    if (is_device_ptr(X) || (P && is_device_ptr(P)) || is_device_ptr(centroids) || is_device_ptr(assign))
        return fail(ADSX_EINVAL, "adsx_build_index takes host pointers");

    // Inverted file (Sec. 2.2.2): stable counting sort by cluster.
    std::vector<int64_t> off((size_t)nlist + 1, 0), pos((size_t)N);
    for (int64_t n = 0; n < N; ++n) {
        int32_t c = assign[n];
        if (c < 0 || c >= nlist) return fail(ADSX_EINVAL, "assign[%lld] = %d out of range", (long long)n, c);
        off[(size_t)c + 1]++;
    }
    for (int32_t c = 0; c < nlist; ++c) off[(size_t)c + 1] += off[(size_t)c];
    std::vector<int32_t> ids((size_t)N);
    {
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int64_t n = 0; n < N; ++n) {
            int64_t p = fill[(size_t)assign[n]]++;
            pos[(size_t)n] = p;
            ids[(size_t)p] = (int32_t)n;
        }
    }
    std::vector<int32_t> tile_off((size_t)nlist + 1, 0);
    for (int32_t c = 0; c < nlist; ++c) {
        if (off[(size_t)c + 1] - off[(size_t)c] > ADSX_MAX_CLUSTER)
            return fail(ADSX_EINVAL, "cluster %d has more than %d members", c, ADSX_MAX_CLUSTER);
        int64_t t = tile_off[(size_t)c] + (off[(size_t)c + 1] - off[(size_t)c] + 31) / 32;
        if (t >= (int64_t)1 << 31) return fail(ADSX_EINVAL, "too many tiles");
        tile_off[(size_t)c + 1] = (int32_t)t;
    }

    Index *ix = new Index();
    ix->N = N;
    ix->metric = metric;
    ix->D = D;
    ix->Dp = (D + 15) / 16 * 16;
    ix->nlist = nlist;
    ix->storage = storage;
    ix->h_off = off;
    ix->total_tiles = tile_off[(size_t)nlist];
    for (int c = 0; c < nlist; ++c)
        ix->max_tiles = std::max<int32_t>(ix->max_tiles, tile_off[(size_t)c + 1] - tile_off[(size_t)c]);
    cudaGetDevice(&ix->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int Dp = ix->Dp;

    auto cleanup = [&](int rc) {
        adsx_free_index(reinterpret_cast<adsx_index *>(ix));
        return rc;
    };
    auto dalloc = [&](void **p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) ix->bytes += (int64_t)bytes;
        return e;
    };
    cudaError_t e;
#define BCK(call, what)                                        \
    do {                                                       \
        e = (call);                                            \
        if (e != cudaSuccess) return cleanup(cuda_fail(e, what)); \
    } while (0)

    if (!kac) BCK(dalloc((void **)&ix->P, sizeof(float) * Dp * Dp), "alloc P");
    BCK(dalloc((void **)&ix->cents, sizeof(float) * (size_t)nlist * Dp), "alloc centroids");
    BCK(dalloc((void **)&ix->cnorm, sizeof(float) * (size_t)nlist), "alloc centroid norms");
    const size_t esz = storage == ADSX_F32 ? 4 : 2;
    BCK(dalloc((void **)&ix->data, esz * (size_t)N * Dp), "alloc data");
    if (storage != ADSX_F32) {
        BCK(dalloc((void **)&ix->rows32, sizeof(float) * (size_t)N * Dp), "alloc FP32 rows");
        BCK(dalloc((void **)&ix->norms, sizeof(float) * (size_t)N), "alloc norms");
    }
    if (metric == ADSX_IP) BCK(dalloc((void **)&ix->onorm, sizeof(float) * (size_t)N), "alloc norms");
    BCK(dalloc((void **)&ix->ids, sizeof(int32_t) * (size_t)N), "alloc ids");
    BCK(dalloc((void **)&ix->off, sizeof(int64_t) * ((size_t)nlist + 1)), "alloc offsets");
    BCK(dalloc((void **)&ix->tile_off, sizeof(int32_t) * ((size_t)nlist + 1)), "alloc tiles");
    BCK(dalloc((void **)&ix->err, sizeof(unsigned)), "alloc error word");

    if (kac) {
        // Kac-walk rotation (Sec. 6.2.3) instead of a dense P: orthogonal by
        // construction (products of Givens rotations with c^2 + s^2 = 1).
        const size_t cnt = (size_t)kac_L * 2 * (D / 2);
        BCK(dalloc((void **)&ix->kac_pairs, sizeof(int32_t) * cnt), "alloc Kac walk");
        BCK(dalloc((void **)&ix->kac_cs, sizeof(float) * cnt), "alloc Kac walk");
        ix->kac_L = kac_L;
        if (cnt) {
            BCK(cudaMemcpyAsync(ix->kac_pairs, kac_pairs, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s), "copy Kac walk");
            BCK(cudaMemcpyAsync(ix->kac_cs, kac_cs, sizeof(float) * cnt, cudaMemcpyHostToDevice, s), "copy Kac walk");
        }
    } else {
        // P padded to Dp x Dp with zeros: padded rotated dims are exactly 0.
        {
            std::vector<float> Pp((size_t)Dp * Dp, 0.f);
            for (int32_t i = 0; i < D; ++i) memcpy(&Pp[(size_t)i * Dp], P + (size_t)i * D, sizeof(float) * D);
            BCK(cudaMemcpyAsync(ix->P, Pp.data(), sizeof(float) * Dp * Dp, cudaMemcpyHostToDevice, s), "copy P");
            BCK(cudaStreamSynchronize(s), "sync");
        }
        // P must be orthogonal (Sec. 3.1): max |P P^T - I| <= 1e-4, checked with
        // the compensated rotation kernel on the device (P P^T = rotating P's rows).
        {
            float *pd = nullptr, *gd = nullptr;
            BCK(cudaMalloc(&pd, sizeof(float) * (size_t)D * D), "alloc P check");
            e = cudaMalloc(&gd, sizeof(float) * (size_t)D * Dp);
            if (e != cudaSuccess) {
                cudaFree(pd);
                return cleanup(cuda_fail(e, "alloc P check"));
            }
            std::vector<float> G((size_t)D * Dp);
            e = cudaMemcpyAsync(pd, P, sizeof(float) * (size_t)D * D, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = adsx::launch_rotate(pd, D, D, ix->P, Dp, gd, Dp, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(G.data(), gd, sizeof(float) * (size_t)D * Dp, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cudaFree(pd);
            cudaFree(gd);
            if (e != cudaSuccess) return cleanup(cuda_fail(e, "P check"));
            double worst = 0.0;
            for (int32_t i = 0; i < D; ++i)
                for (int32_t j = 0; j < D; ++j)
                    worst = std::max(worst, fabs((double)G[(size_t)i * Dp + j] - (i == j ? 1.0 : 0.0)));
            if (!(worst <= 1e-4))
                return cleanup(fail(ADSX_EINVAL, "P is not orthogonal (max|P P^T - I| = %g)", worst));
        }
        // the digits of P for the tensor-core query rotation (Dp <= 1024)
        int rb = 0, rT = 0, rL = 0;
        adsx::tc_rot_params(Dp, &rb, &rT, &rL);
        if (rT > 0) {
            std::vector<float> RB;
            std::vector<int32_t> RF;
            rot_slices_host(P, D, Dp, rb, rT, rL, RB, RF, ix->rot_boff);
            BCK(dalloc((void **)&ix->rot_B, sizeof(float) * RB.size()), "alloc rotation digits");
            BCK(dalloc((void **)&ix->rot_F, sizeof(int32_t) * RF.size()), "alloc rotation digits");
            BCK(cudaMemcpyAsync(ix->rot_B, RB.data(), sizeof(float) * RB.size(), cudaMemcpyHostToDevice, s),
                "copy rotation digits");
            BCK(cudaMemcpyAsync(ix->rot_F, RF.data(), sizeof(int32_t) * RF.size(), cudaMemcpyHostToDevice, s),
                "copy rotation digits");
            BCK(cudaStreamSynchronize(s), "sync");
            ix->rot_b = rb;
            ix->rot_T = rT;
            ix->rot_Lmax = rL;
            // available; the compensated FP32 rotation stays the initial
            // mode (measured faster at these shapes)
            ix->rot_ok = true;
        }
    }
    BCK(cudaMemcpyAsync(ix->ids, ids.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s), "copy ids");
    BCK(cudaMemcpyAsync(ix->off, off.data(), sizeof(int64_t) * (nlist + 1), cudaMemcpyHostToDevice, s), "copy off");
    BCK(cudaMemcpyAsync(ix->tile_off, tile_off.data(), sizeof(int32_t) * (nlist + 1), cudaMemcpyHostToDevice, s), "copy tiles");
    BCK(cudaMemsetAsync(ix->err, 0, sizeof(unsigned), s), "clear error word");

    {
        Scratch sc(s);
        float *xd = nullptr, *yd = nullptr, *cd = nullptr;
        int32_t *ad = nullptr;
        int64_t *pd = nullptr;
        BCK(sc.get(&xd, (size_t)N * D), "alloc X");
        BCK(sc.get(&yd, (size_t)N * Dp), "alloc Y");
        BCK(sc.get(&ad, (size_t)N), "alloc assign");
        BCK(sc.get(&pd, (size_t)N), "alloc positions");
        BCK(sc.get(&cd, (size_t)nlist * D), "alloc C");
        BCK(cudaMemcpyAsync(xd, X, sizeof(float) * N * D, cudaMemcpyHostToDevice, s), "copy X");
        BCK(cudaMemcpyAsync(ad, assign, sizeof(int32_t) * N, cudaMemcpyHostToDevice, s), "copy assign");
        BCK(cudaMemcpyAsync(pd, pos.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice, s), "copy positions");
        BCK(cudaMemcpyAsync(cd, centroids, sizeof(float) * (size_t)nlist * D, cudaMemcpyHostToDevice, s), "copy C");
        // Sec. 8, extension (1): cosine and inner-product indexes store the
        // data rows normalised (inner product keeps their norms); cosine
        // centroids are normalised too, inner-product ones stay raw.
        float *xnorm = nullptr;
        if (metric != ADSX_L2) {
            if (metric == ADSX_IP) BCK(sc.get(&xnorm, (size_t)N), "alloc norms");
            BCK(adsx::launch_normalize_rows(xd, N, D, D, xnorm,
                                            metric == ADSX_COSINE ? ix->err : nullptr, s),
                "normalise data");
            if (metric == ADSX_COSINE)
                BCK(adsx::launch_normalize_rows(cd, nlist, D, D, nullptr, nullptr, s),
                    "normalise centroids");
        }
        // Sec. 3.1 / Sec. 6.1: rotate every data vector and centroid once.
        // Index phase: rotation of the data and the centroids, once per index.
        BCK(adsx::rotate_rows(ix, xd, N, yd, s), "rotate data");
        BCK(adsx::rotate_rows(ix, cd, nlist, ix->cents, s), "rotate centroids");
        BCK(adsx::launch_row_sqnorm(ix->cents, nlist, Dp, Dp, ix->cnorm, s), "centroid norms");
        // the centroids' TF32 halves for the centroid-distance GEMM
        BCK(dalloc((void **)&ix->cents_split,
                   sizeof(uint32_t) * (size_t)adsx::tf32_split_words(nlist, Dp)),
            "alloc split centroids");
        BCK(adsx::launch_tf32_split(ix->cents, nlist, Dp, Dp, ix->cents_split, s), "split centroids");
        // inner product: ||q'||^2 + max ||c'||^2 - 2 q'.c' >= 0 ranks clusters
        // by the largest <c, q> with the distance GEMM unchanged
        if (metric == ADSX_IP) BCK(adsx::launch_fill_max(ix->cnorm, nlist, s), "centroid term");
        BCK(adsx::launch_scatter_layout(yd, N, Dp, ad, pd, ix->off, ix->data, storage, ix->rows32,
                                        ix->norms, s), "scatter layout");
        if (metric == ADSX_IP) BCK(adsx::launch_scatter_f32(xnorm, pd, N, ix->onorm, s), "scatter norms");
        BCK(cudaStreamSynchronize(s), "build sync");
    }
    if (metric == ADSX_COSINE) {
        unsigned err = 0;
        BCK(cudaMemcpy(&err, ix->err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error word");
        if (err & adsx::ERR_ZERO_ROW)
            return cleanup(fail(ADSX_EINVAL, "a data row has zero norm (cosine similarity undefined)"));
    }
    BCK(cudaStreamSynchronize(s), "build sync");
#undef BCK
    *out = reinterpret_cast<adsx_index *>(ix);
    return ADSX_OK;
}

int adsx_build_index(const float *X, int64_t N, int32_t D, const float *P,
                     const float *centroids, int32_t nlist, const int32_t *assign,
                     int32_t storage, void *stream, adsx_index **out)
{
    return build_impl(X, N, D, P, nullptr, nullptr, 0, centroids, nlist, assign, storage, ADSX_L2,
                      stream, out);
}

int adsx_build_index_metric(const float *X, int64_t N, int32_t D, const float *P,
                            const float *centroids, int32_t nlist, const int32_t *assign,
                            int32_t storage, int32_t metric, void *stream, adsx_index **out)
{
    return build_impl(X, N, D, P, nullptr, nullptr, 0, centroids, nlist, assign, storage, metric,
                      stream, out);
}

int adsx_build_index_kac(const float *X, int64_t N, int32_t D, const int32_t *pairs,
                         const float *cs, int32_t L, const float *centroids, int32_t nlist,
                         const int32_t *assign, int32_t storage, int32_t metric, void *stream,
                         adsx_index **out)
{
    if (L == 0) return fail(ADSX_EINVAL, "Kac walk layers out of range (1..%d)", ADSX_MAX_KAC_LAYERS);
    return build_impl(X, N, D, nullptr, pairs, cs, L, centroids, nlist, assign, storage, metric,
                      stream, out);
}

int adsx_index_metric(const adsx_index *index, int32_t *metric)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    if (!ix || !metric) return fail(ADSX_EINVAL, "NULL argument");
    *metric = ix->metric;
    return ADSX_OK;
}

int adsx_free_index(adsx_index *index)
{
    Index *ix = reinterpret_cast<Index *>(index);
    if (!ix) return ADSX_OK;
    cudaSetDevice(ix->device);
    cudaDeviceSynchronize();
    cudaFree(ix->P);
    cudaFree(ix->cents);
    cudaFree(ix->cents_split);
    cudaFree(ix->cnorm);
    cudaFree(ix->data);
    cudaFree(ix->rows32);
    cudaFree(ix->norms);
    cudaFree(ix->onorm);
    cudaFree(ix->kac_pairs);
    cudaFree(ix->kac_cs);
    cudaFree(ix->rot_B);
    cudaFree(ix->rot_F);
    cudaFree(ix->ids);
    cudaFree(ix->off);
    cudaFree(ix->tile_off);
    cudaFree(ix->err);
    for (cudaEvent_t e : ix->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ix->kev)
        if (e) cudaEventDestroy(e);
    delete ix;
    return ADSX_OK;
}

int adsx_index_info(const adsx_index *index, int64_t *N, int32_t *D, int32_t *nlist,
                    int32_t *storage, int64_t *device_bytes)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    if (!ix) return fail(ADSX_EINVAL, "index is NULL");
    if (N) *N = ix->N;
    if (D) *D = ix->D;
    if (nlist) *nlist = ix->nlist;
    if (storage) *storage = ix->storage;
    if (device_bytes) *device_bytes = ix->bytes;
    return ADSX_OK;
}

int adsx_rotate(const adsx_index *index, const float *Qv, int64_t nq, float *out, void *stream)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (nq < 0 || (nq > 0 && (!Qv || !out))) return fail(ADSX_EINVAL, "bad query arguments");
    if (nq == 0) return ADSX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Buf<float> q, o;
    float *qrot = nullptr;
    CK(stage_in(sc, Qv, (size_t)nq * ix->D, q), "stage queries");
    CK(stage_out(sc, out, (size_t)nq * ix->D, o), "stage output");
    CK(sc.get(&qrot, (size_t)nq * ix->Dp), "alloc q'");
    CK(rotate_queries(ix, q.dev, nq, qrot, sc), "rotate");
    CK(cudaMemcpy2DAsync(o.dev, sizeof(float) * ix->D, qrot, sizeof(float) * ix->Dp,
                         sizeof(float) * ix->D, (size_t)nq, cudaMemcpyDeviceToDevice, s), "copy q'");
    CK(copy_back(o, s), "copy back");
    return finish(s, o.host != nullptr, "rotate");
}

int adsx_probe(const adsx_index *index, const float *Qv, int64_t nq, int32_t nprobe,
               int32_t *probes, float *probe_d2, void *stream)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (nq < 0 || (nq > 0 && (!Qv || !probes))) return fail(ADSX_EINVAL, "bad query arguments");
    if (nprobe < 1 || nprobe > ix->nlist || nprobe > ADSX_MAX_NPROBE)
        return fail(ADSX_EINVAL, "nprobe out of range (1..min(nlist, %d))", ADSX_MAX_NPROBE);
    if (nq == 0) return ADSX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Buf<float> q, pd;
    Buf<int32_t> pr;
    float *qrot = nullptr;
    CK(stage_in(sc, Qv, (size_t)nq * ix->D, q), "stage queries");
    CK(stage_out(sc, probes, (size_t)nq * nprobe, pr), "stage probes");
    CK(stage_out(sc, probe_d2, (size_t)nq * nprobe, pd), "stage probe distances");
    CK(sc.get(&qrot, (size_t)nq * ix->Dp), "alloc q'");
    CK(rotate_queries(ix, q.dev, nq, qrot, sc), "rotate");
    CK(queries_before_probe(ix, qrot, nq, s), "normalise queries");
    CK(probe_queries(ix, qrot, nq, nprobe, pr.dev, pd.dev, sc), "probe");
    CK(copy_back(pr, s), "copy back");
    CK(copy_back(pd, s), "copy back");
    return finish(s, pr.host || pd.host, "probe");
}

}  // extern "C"

// ---------------------------------------------------------------- scan schedules
// The query-major scan of `a` (scan.cu), with the shared bounds, partial
// lists and their merge when queries are split (S > 1).
static cudaError_t qm_scan(const Index *ix, adsx::ScanArgs a, Scratch &sc)
{
    cudaStream_t s = sc.s;
    unsigned *counter = nullptr;
    cudaError_t e = sc.get(&counter, 1);
    if (e != cudaSuccess) return e;
    a.work_counter = counter;
    if (a.S > 1) {
        if ((e = sc.get(&a.part_d, (size_t)a.n_items * a.K)) != cudaSuccess) return e;
        if ((e = sc.get(&a.part_i, (size_t)a.n_items * a.K)) != cudaSuccess) return e;
        if ((e = sc.get(&a.r2g, (size_t)a.nq)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.r2g, 0xff, sizeof(unsigned) * a.nq, s)) != cudaSuccess) return e;
        if (a.out_dims &&
            (e = cudaMemsetAsync(a.out_dims, 0, sizeof(int64_t) * a.nq, s)) != cudaSuccess)
            return e;
    }
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    if ((e = mark_kernel(ix, true, s)) != cudaSuccess) return e;
    if ((e = adsx::launch_ads_scan(a, adsx::ads_scan_grid(a, ix->device), s)) != cudaSuccess)
        return e;
    if ((e = mark_kernel(ix, false, s)) != cudaSuccess) return e;
    return adsx::launch_finalize_topk(a, s);
}

// Whether the uniform search set up in `a` runs cluster-major (cmscan.cu).
static bool use_cluster_major(const Index *ix, const adsx::ScanArgs &a)
{
    if (ix->sched == ADSX_SCHED_QUERY) return false;
    if (a.metric == ADSX_IP || a.db > adsx::CM_MAX_DB) return false;
    if (a.nprobe <= ix->cm_r0) return false;           // round 0 alone would cover every probe
    if (ix->sched == ADSX_SCHED_CLUSTER) return true;
    // Measured on GB300 (SIFT-shaped 1M x 128, GIST-shaped 250k and 1M x 960,
    // 125..10k queries): cluster-major is faster once a batch probes each
    // cluster about once on average (from 1.1x at 250 SIFT-shaped queries to
    // 1.6x for 1000 GIST-shaped ones in FP32), except with 16-bit storage at
    // high D, where query-major stays ahead below about 8 queries per cluster.
    const int64_t probes = a.nq * (int64_t)a.nprobe, nl = ix->nlist;
    if (a.nq < 128 || probes < nl) return false;
    if (a.storage != ADSX_F32 && ix->D >= 512 && probes < 8 * nl) return false;
    return true;
}

// Queries per cluster-major work item: the index's setting, or chosen by
// the batch from the mean number of queries probing a cluster, q = nq *
// nprobe / nlist: 16 from q = 24, 8 from q = 6, else 4 (at D >= 512 at most 8,
// and 4 with 16-bit storage: there most candidates stop at the first steps
// and a slot's per-step bookkeeping outweighs the shared tile loads).
static int cm_queries_per_item(const Index *ix, int64_t nq, int nprobe)
{
    if (ix->cm_G > 0) return ix->cm_G;
    const double q = (double)nq * nprobe / ix->nlist;
    int G = q >= 24.0 ? 16 : (q >= 6.0 ? 8 : 4);
    if (ix->D >= 512) G = std::min(G, ix->storage == ADSX_F32 ? 8 : 4);
    return G;
}

// The probe-rank ranges of the cluster-major rounds after round 0: each
// `growth` times as far as where it starts; a short tail joins the last.
static std::vector<std::pair<int, int>> cm_rounds(int r0, int nprobe, int growth)
{
    std::vector<std::pair<int, int>> r;
    int lo = r0;
    while (lo < nprobe) {
        int hi = std::max(lo + 1, lo * growth);
        if (hi >= nprobe || 2 * (nprobe - hi) < hi - lo) hi = nprobe;
        r.push_back({lo, hi});
        lo = hi;
    }
    return r;
}

// The fields of a cluster-major pass taken from a query-major setup.
static adsx::CmArgs cm_args_from(const adsx::ScanArgs &a, int G)
{
    adsx::CmArgs c;
    c.data = a.data;
    c.rows32 = a.rows32;
    c.norms = a.norms;
    c.storage = a.storage;
    c.ids = a.ids;
    c.off = a.off;
    c.qrot = a.qrot;
    c.D = a.D;
    c.Dp = a.Dp;
    c.nblk = a.nblk;
    c.db = a.db;
    c.test_on = a.test_on;
    c.ftab = a.ftab;
    c.r2 = nullptr;
    c.G = G;
    c.tpi = 1;
    c.app_d = nullptr;
    c.app_i = nullptr;
    c.app_n = nullptr;
    c.cap = 0;
    c.out_dims = a.out_dims;
    return c;
}

// Plan buffers of the rounds R (probe ranks already set in R.lo): per round
// its item capacity -- ceil(cnt_c / G) query groups times the chunks of
// cluster c, at most (cnt_c / G + 1) * chunks_c summed over the clusters --
// and the offset of its items (R.ibase).
static cudaError_t cm_plan_buffers(const Index *ix, int64_t nq, int G, adsx::CmRounds &R,
                                   Scratch &sc, adsx::CmPlan &pl, int64_t *icap)
{
    cudaError_t e;
    const size_t nl = (size_t)ix->nlist, nr = (size_t)R.n;
    const int64_t tpi = ix->cm_tpi;
    const int64_t maxch = (ix->max_tiles + tpi - 1) / tpi;
    int64_t total = 0;
    for (int r = 0; r < R.n; ++r) {
        const int64_t w = R.lo[r + 1] - R.lo[r];
        icap[r] = nq * w * maxch / G + ix->total_tiles / tpi + ix->nlist + 1;
        R.ibase[r] = total;
        total += icap[r];
    }
    if ((e = sc.get(&pl.cnt, nr * nl)) != cudaSuccess) return e;
    if ((e = sc.get(&pl.coff, nr * (nl + 1))) != cudaSuccess) return e;
    if ((e = sc.get(&pl.ioff, nr * nl)) != cudaSuccess) return e;
    if ((e = sc.get(&pl.cur, nr * nl)) != cudaSuccess) return e;
    if ((e = sc.get(&pl.n_items, nr)) != cudaSuccess) return e;
    if ((e = sc.get(&pl.qlist, (size_t)(nq * (int64_t)(R.lo[R.n] - R.lo[0])))) != cudaSuccess)
        return e;
    return sc.get(&pl.items, (size_t)total);
}

// The scan fields of round r of the plan.
static void cm_round_args(adsx::CmArgs &c, const adsx::CmPlan &pl, const adsx::CmRounds &R,
                          const int64_t *icap, int64_t nq, int nlist, int r)
{
    c.coff = pl.coff + (size_t)r * (nlist + 1);
    c.qlist = pl.qlist + nq * (int64_t)(R.lo[r] - R.lo[0]);
    c.items = pl.items + R.ibase[r];
    c.n_items = pl.n_items + r;
    c.items_cap = (int32_t)std::min<int64_t>(icap[r], INT32_MAX);
}

// The cluster-major schedule of a uniform search (ADSX_SCHED_CLUSTER): round
// 0 over each query's nearest cm_r0 clusters with the test off, then the later
// probe ranks in rounds, each scanned cluster-major against the K-th
// distance of the rounds before it and merged into the query's top-K; a
// query whose round list overflowed is searched again query-major.  `a` is
// the query-major setup of the whole search.
static cudaError_t cm_scan(const Index *ix, const adsx::ScanArgs &a, Scratch &sc)
{
    cudaStream_t s = sc.s;
    cudaError_t e;
    const int64_t nq = a.nq;
    const int K = a.K, nprobe = a.nprobe, G = cm_queries_per_item(ix, nq, a.nprobe);
    const int r0 = std::min(ix->cm_r0, nprobe);
    // capacity of a round's list per query: candidates reaching d = D within
    // the previous rounds' r -- in round 0 (no r yet) every member of the
    // query's r0 nearest clusters (a query beyond it is searched again
    // query-major)
    const int cap = std::max(std::max(4 * K, 1024), r0 * 32 * ix->max_tiles);
    float *r2 = nullptr, *app_d = nullptr;
    int32_t *app_i = nullptr, *ovf = nullptr;
    unsigned *app_n = nullptr, *counter = nullptr;
    if ((e = sc.get(&r2, (size_t)nq)) != cudaSuccess) return e;
    if ((e = sc.get(&app_n, (size_t)nq)) != cudaSuccess) return e;
    if ((e = sc.get(&ovf, (size_t)nq)) != cudaSuccess) return e;
    if ((e = sc.get(&app_d, (size_t)nq * cap)) != cudaSuccess) return e;
    if ((e = sc.get(&app_i, (size_t)nq * cap)) != cudaSuccess) return e;
    if ((e = sc.get(&counter, 1)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(app_n, 0, sizeof(unsigned) * nq, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ovf, 0, sizeof(int32_t) * nq, s)) != cudaSuccess) return e;
    // empty top-K lists (ids -1) and dims counters; the merge then sets r = +inf
    if ((e = cudaMemsetAsync(a.out_ids, 0xff, sizeof(int64_t) * nq * K, s)) != cudaSuccess) return e;
    if (a.out_dims &&
        (e = cudaMemsetAsync(a.out_dims, 0, sizeof(int64_t) * nq, s)) != cudaSuccess)
        return e;
    adsx::CmMergeArgs m;
    m.nq = nq;
    m.K = K;
    m.cap = cap;
    m.T = 0;
    m.ids = a.out_ids;
    m.d2 = a.out_d2;
    m.app_d = app_d;
    m.app_i = app_i;
    m.app_n = app_n;
    m.r2 = r2;
    m.ovf = ovf;
    m.metric = a.metric;
    m.final_pass = 0;
    if ((e = adsx::launch_cm_merge(m, s)) != cudaSuccess) return e;

    // round 0: each query's r0 nearest clusters, every member to d = D (no r
    // yet: the test cannot reject); then the later ranks against r.  All
    // rounds are planned at once (the probe lists are known).
    auto rounds = cm_rounds(r0, nprobe, ix->cm_growth);
    rounds.insert(rounds.begin(), {0, r0});
    if ((int)rounds.size() > adsx::CM_MAX_ROUNDS) return cudaErrorInvalidValue;
    adsx::CmRounds R;
    R.n = (int32_t)rounds.size();
    for (int r = 0; r < R.n; ++r) R.lo[r] = rounds[r].first;
    R.lo[R.n] = nprobe;
    adsx::CmPlan pl;
    int64_t icap[adsx::CM_MAX_ROUNDS];
    if ((e = cm_plan_buffers(ix, nq, G, R, sc, pl, icap)) != cudaSuccess) return e;
    if ((e = adsx::launch_cm_plan(a.probes, nq, nprobe, R, ix->nlist, G, ix->cm_tpi, ix->off, pl,
                                  s)) != cudaSuccess)
        return e;
    adsx::CmArgs c = cm_args_from(a, G);
    c.tpi = ix->cm_tpi;
    c.r2 = r2;
    c.work_counter = counter;
    c.app_d = app_d;
    c.app_i = app_i;
    c.app_n = app_n;
    c.cap = cap;
    // 16-bit storage: round 0 appends approximate distances, and only the
    // members that can be among the K nearest are rechecked in FP32
    const bool defer = ix->storage != ADSX_F32;
    adsx::CmRecheck0Args rc0;
    rc0.nq = nq;
    rc0.K = K;
    rc0.cap = cap;
    rc0.Dp = ix->Dp;
    rc0.u = ix->storage == ADSX_BF16 ? 1.0f / 256.0f : 1.0f / 2048.0f;
    rc0.rows32 = ix->rows32;
    rc0.norms = ix->norms;
    rc0.qrot = a.qrot;
    rc0.ids = ix->ids;
    rc0.app_d = app_d;
    rc0.app_i = app_i;
    rc0.app_n = app_n;
    for (int i = 0; i < R.n; ++i) {
        cm_round_args(c, pl, R, icap, nq, ix->nlist, i);
        c.test_on = i == 0 ? 0 : a.test_on;
        c.defer_recheck = defer && i == 0;
        if ((e = mark_kernel(ix, true, s)) != cudaSuccess) return e;
        if ((e = adsx::launch_cm_scan(c, ix->device, s)) != cudaSuccess) return e;
        if ((e = mark_kernel(ix, false, s)) != cudaSuccess) return e;
        if (c.defer_recheck && (e = adsx::launch_cm_recheck0(rc0, s)) != cudaSuccess) return e;
        m.final_pass = i + 1 == R.n;
        if ((e = adsx::launch_cm_merge(m, s)) != cudaSuccess) return e;
    }
    // queries whose list overflowed: the whole search again, query-major
    int2 *fitems = nullptr;
    int32_t *fn = nullptr;
    if ((e = sc.get(&fitems, (size_t)nq)) != cudaSuccess) return e;
    if ((e = sc.get(&fn, 1)) != cudaSuccess) return e;
    if ((e = adsx::launch_cm_overflow_items(ovf, nq, fitems, fn, s)) != cudaSuccess) return e;
    adsx::ScanArgs af = a;
    af.items = fitems;
    af.n_items_dev = fn;
    af.n_items = (int32_t)nq;
    af.S = 1;
    af.probe_stride = nprobe;
    af.work_counter = counter;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    return adsx::launch_ads_scan(af, adsx::ads_scan_grid(af, ix->device), s);
}

static int search_impl(const adsx_index *index, const float *Qv, int64_t nq, int32_t K,
                       int32_t nprobe, float eps0, int32_t delta_d, int64_t *ids, float *dists,
                       int64_t *dims_read, void *stream, int pd)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (nq < 0 || (nq > 0 && (!Qv || !ids || !dists))) return fail(ADSX_EINVAL, "bad query arguments");
    if (K < 1 || K > ADSX_MAX_K) return fail(ADSX_EINVAL, "K out of range (1..%d)", ADSX_MAX_K);
    if (nprobe < 1 || nprobe > ix->nlist || nprobe > ADSX_MAX_NPROBE)
        return fail(ADSX_EINVAL, "nprobe out of range (1..min(nlist, %d))", ADSX_MAX_NPROBE);
    if (delta_d == 0) delta_d = ix->tuned_delta_d;
    if ((rc = check_blocks(delta_d, eps0))) return rc;
    if (nq == 0) return ADSX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Buf<float> q, od;
    Buf<int64_t> oi, odims;
    float *qrot = nullptr;
    int32_t *probes = nullptr;
    const_cast<Index *>(ix)->nkev = 0;
    CK(stage_in(sc, Qv, (size_t)nq * ix->D, q), "stage queries");
    CK(stage_out(sc, ids, (size_t)nq * K, oi), "stage ids");
    CK(stage_out(sc, dists, (size_t)nq * K, od), "stage dists");
    CK(stage_out(sc, dims_read, (size_t)nq, odims), "stage dims");
    CK(sc.get(&qrot, (size_t)nq * ix->Dp), "alloc q'");
    CK(sc.get(&probes, (size_t)nq * nprobe), "alloc probes");
    CK(mark(ix, 0, s), "event");
    CK(rotate_queries(ix, q.dev, nq, qrot, sc), "rotate");
    CK(mark(ix, 1, s), "event");
    CK(queries_before_probe(ix, qrot, nq, s), "normalise queries");
    CK(probe_queries(ix, qrot, nq, nprobe, probes, nullptr, sc), "probe");
    CK(mark(ix, 3, s), "event");
    float *qnorm = nullptr;
    CK(queries_after_probe(ix, qrot, nq, sc, &qnorm), "normalise queries");

    adsx::ScanArgs a;
    if (!adsx::fill_uniform_scan(a, ix, nq, K, nprobe, eps0, delta_d, pd))
        return fail(ADSX_EINVAL, "too many queries in one call");
    a.qnorm = qnorm;
    a.qrot = qrot;
    a.probes = probes;
    a.out_ids = oi.dev;
    a.out_d2 = od.dev;
    a.out_dims = odims.dev;
    float *ftab = nullptr;
    CK(sc.get(&ftab, (size_t)a.nblk + 1), "alloc test factors");
    a.ftab = ftab;
    CK(adsx::launch_test_factors(ftab, a.nblk, a.D, (a.test_on && !pd) ? eps0 : 0.f, s, pd),
       "test factors");
    if (use_cluster_major(ix, a)) CK(cm_scan(ix, a, sc), "cluster-major scan");
    else CK(qm_scan(ix, a, sc), "scan");
    CK(mark(ix, 4, s), "event");
    if (ix->timing) const_cast<Index *>(ix)->timed_once = true;
    CK(copy_back(oi, s), "copy back");
    CK(copy_back(od, s), "copy back");
    CK(copy_back(odims, s), "copy back");
    bool any_host = oi.host || od.host || odims.host;
    rc = finish(s, any_host, "search");
    if (rc) return rc;
    if (any_host) {
        unsigned err = 0;
        CK(cudaMemcpy(&err, ix->err, sizeof err, cudaMemcpyDeviceToHost), "read error word");
        if (err) {
            cudaMemset(ix->err, 0, sizeof(unsigned));
            return fail(ADSX_ETIMEOUT, "a bounded device wait gave up (error word 0x%x)", err);
        }
    }
    return ADSX_OK;
}

extern "C" {

int adsx_search(const adsx_index *index, const float *Qv, int64_t nq, int32_t K, int32_t nprobe,
                float eps0, int32_t delta_d, int64_t *ids, float *dists, int64_t *dims_read,
                void *stream)
{
    return search_impl(index, Qv, nq, K, nprobe, eps0, delta_d, ids, dists, dims_read, stream, 0);
}

int adsx_search_pdscan(const adsx_index *index, const float *Qv, int64_t nq, int32_t K,
                       int32_t nprobe, int32_t delta_d, int64_t *ids, float *dists,
                       int64_t *dims_read, void *stream)
{
    return search_impl(index, Qv, nq, K, nprobe, 0.f, delta_d, ids, dists, dims_read, stream, 1);
}

int adsx_search_batched(const adsx_index *index, const float *Qv, int64_t nq, const int32_t *K,
                        const int32_t *nprobe, int32_t max_K, int32_t max_nprobe, float eps0,
                        int32_t delta_d, const int64_t *out_offsets, int64_t out_total,
                        int64_t *ids, float *dists, int64_t *dims_read, void *stream)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (nq < 0 || (nq > 0 && (!Qv || !K || !nprobe || !ids || !dists)))
        return fail(ADSX_EINVAL, "bad query arguments");
    if (max_K < 1 || max_K > ADSX_MAX_K) return fail(ADSX_EINVAL, "max_K out of range (1..%d)", ADSX_MAX_K);
    if (max_nprobe < 1 || max_nprobe > ix->nlist || max_nprobe > ADSX_MAX_NPROBE)
        return fail(ADSX_EINVAL, "max_nprobe out of range (1..min(nlist, %d))", ADSX_MAX_NPROBE);
    if (delta_d == 0) delta_d = ix->tuned_delta_d;
    if ((rc = check_blocks(delta_d, eps0))) return rc;
    if (out_total < 0) return fail(ADSX_EINVAL, "out_total < 0");
    if (nq == 0) return ADSX_OK;
    if (nq >= ((int64_t)1 << 31) / adsx::BATCH_MAX_SPLITS) return fail(ADSX_EINVAL, "too many queries in one call");
    // Host copies of K / nprobe are checked here when the caller passes host
    // arrays; device arrays are checked by the planner (error word).
    if (!is_device_ptr(K) && !is_device_ptr(nprobe)) {
        int64_t sumK = 0;
        for (int64_t q = 0; q < nq; ++q) {
            if (K[q] < 1 || K[q] > max_K) return fail(ADSX_EINVAL, "K[%lld] = %d outside [1, max_K]", (long long)q, K[q]);
            if (nprobe[q] < 1 || nprobe[q] > max_nprobe)
                return fail(ADSX_EINVAL, "nprobe[%lld] = %d outside [1, max_nprobe]", (long long)q, nprobe[q]);
            sumK += K[q];
        }
        if (!out_offsets && out_total < sumK) return fail(ADSX_EINVAL, "out_total below the sum of K");
    }
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Buf<float> q, od;
    Buf<int32_t> kq, pq;
    Buf<int64_t> oo, oi, odims;
    CK(stage_in(sc, Qv, (size_t)nq * ix->D, q), "stage queries");
    CK(stage_in(sc, K, (size_t)nq, kq), "stage K");
    CK(stage_in(sc, nprobe, (size_t)nq, pq), "stage nprobe");
    if (out_offsets) CK(stage_in(sc, out_offsets, (size_t)nq, oo), "stage offsets");
    CK(stage_out(sc, ids, (size_t)out_total, oi), "stage ids");
    CK(stage_out(sc, dists, (size_t)out_total, od), "stage dists");
    CK(stage_out(sc, dims_read, (size_t)nq, odims), "stage dims");
    float *qrot = nullptr;
    int32_t *probes = nullptr, *item_first = nullptr, *n_items = nullptr, *qperm = nullptr;
    int2 *items = nullptr;
    int64_t *out_off = nullptr;
    unsigned *counter = nullptr;
    const int64_t items_cap = nq * adsx::BATCH_MAX_SPLITS;
    CK(sc.get(&qrot, (size_t)nq * ix->Dp), "alloc q'");
    CK(sc.get(&probes, (size_t)nq * max_nprobe), "alloc probes");
    CK(sc.get(&items, (size_t)items_cap), "alloc items");
    CK(sc.get(&item_first, (size_t)nq), "alloc items");
    CK(sc.get(&n_items, 1), "alloc items");
    CK(sc.get(&qperm, (size_t)nq), "alloc order");
    CK(sc.get(&out_off, (size_t)nq), "alloc offsets");
    CK(sc.get(&counter, 1), "alloc counter");
    CK(mark(ix, 0, s), "event");
    CK(rotate_queries(ix, q.dev, nq, qrot, sc), "rotate");
    CK(mark(ix, 1, s), "event");
    CK(queries_before_probe(ix, qrot, nq, s), "normalise queries");
    {
        float *dist = nullptr;
        unsigned *summ = nullptr;
        CK(sc.get(&dist, (size_t)nq * ix->nlist), "alloc distances");
        CK(probe_summary(ix, nq, max_nprobe, sc, &summ), "alloc tile summary");
        CK(centroid_distances(ix, qrot, nq, dist, sc, summ), "centroid distances");
        CK(mark(ix, 2, s), "event");
        CK(adsx::launch_select_nprobe(dist, nq, ix->nlist, max_nprobe, probes, nullptr, s, pq.dev,
                                      summ),
           "select");
    }
    const int target = adsx::scan_items_target(ix->device, ix->items_per_sm);
    CK(adsx::launch_plan_batched(kq.dev, pq.dev, nq, max_K, max_nprobe, target,
                                 ix->N / ix->nlist, items, item_first, n_items,
                                 qperm, oo.dev, out_off, ix->err, s), "plan");
    CK(mark(ix, 3, s), "event");
    float *qnorm = nullptr;
    CK(queries_after_probe(ix, qrot, nq, sc, &qnorm), "normalise queries");

    adsx::ScanArgs a;
    a.metric = ix->metric;
    a.onorm = ix->onorm;
    a.qnorm = qnorm;
    a.data = ix->data;
    a.rows32 = ix->rows32;
    a.norms = ix->norms;
    a.storage = ix->storage;
    a.ids = ix->ids;
    a.off = ix->off;
    a.qrot = qrot;
    a.probes = probes;
    a.nq = nq;
    a.D = ix->D;
    a.Dp = ix->Dp;
    a.nblk = ix->Dp / adsx::BLK;
    a.nprobe = max_nprobe;
    a.K = max_K;
    {
        int Kp = 1;
        while (Kp < max_K) Kp <<= 1;
        a.C = 1;
        while (a.C < std::max(2 * Kp, max_K + 32)) a.C <<= 1;
    }
    a.S = 1;
    a.n_items = (int32_t)items_cap;       // upper bound; the kernel reads the planned count
    a.db = delta_d / adsx::BLK;
    a.test_on = isinf(eps0) ? 0 : 1;
    if (a.db >= a.nblk) a.test_on = 0;
    if (!a.test_on) a.db = adsx::FD_STEP_BLOCKS < a.nblk ? adsx::FD_STEP_BLOCKS : a.nblk;
    a.out_ids = oi.dev;
    a.out_d2 = od.dev;
    a.out_dims = odims.dev;
    a.work_counter = counter;
    a.err = ix->err;
    a.Kq = kq.dev;
    a.nprobe_q = pq.dev;
    a.out_off = out_off;
    a.out_total = out_total;
    a.items = items;
    a.item_first = item_first;
    a.n_items_dev = n_items;
    a.Kmax = max_K;
    a.probe_stride = max_nprobe;
    float *ftab = nullptr;
    CK(sc.get(&ftab, (size_t)a.nblk + 1), "alloc test factors");
    a.ftab = ftab;
    CK(adsx::launch_test_factors(ftab, a.nblk, a.D, a.test_on ? eps0 : 0.f, s), "test factors");
    CK(sc.get(&a.part_d, (size_t)items_cap * max_K), "alloc partial lists");
    CK(sc.get(&a.part_i, (size_t)items_cap * max_K), "alloc partial lists");
    CK(sc.get(&a.r2g, (size_t)nq), "alloc r2 bounds");
    CK(cudaMemsetAsync(a.r2g, 0xff, sizeof(unsigned) * nq, s), "clear r2 bounds");
    if (a.out_dims) CK(cudaMemsetAsync(a.out_dims, 0, sizeof(int64_t) * nq, s), "clear dims");
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), s), "clear counter");
    CK(adsx::launch_ads_scan(a, adsx::ads_scan_grid(a, ix->device), s), "scan");
    CK(adsx::launch_finalize_topk(a, s), "finalize");
    CK(mark(ix, 4, s), "event");
    if (ix->timing) const_cast<Index *>(ix)->timed_once = true;
    CK(copy_back(oi, s), "copy back");
    CK(copy_back(od, s), "copy back");
    CK(copy_back(odims, s), "copy back");
    bool any_host = oi.host || od.host || odims.host;
    rc = finish(s, any_host, "batched search");
    if (rc) return rc;
    if (any_host) {
        unsigned err = 0;
        CK(cudaMemcpy(&err, ix->err, sizeof err, cudaMemcpyDeviceToHost), "read error word");
        if (err) {
            cudaMemset(ix->err, 0, sizeof(unsigned));
            return fail((err & (adsx::ERR_BATCH_ARGS | adsx::ERR_OUT_RANGE)) ? ADSX_EINVAL : ADSX_ETIMEOUT,
                        "device-side check failed (error word 0x%x)", err);
        }
    }
    return ADSX_OK;
}

int adsx_dco_fixed_r(const adsx_index *index, const float *Qv, int64_t nq, const float *r2,
                     float eps0, int32_t delta_d, uint8_t *decisions, int32_t *dims, void *stream)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (ix->metric != ADSX_L2) return fail(ADSX_EINVAL, "adsx_dco_fixed_r supports L2 indexes only");
    if (nq < 0 || (nq > 0 && (!Qv || !r2 || !decisions))) return fail(ADSX_EINVAL, "bad arguments");
    if ((rc = check_blocks(delta_d, eps0))) return rc;
    if (nq == 0) return ADSX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Buf<float> q, rr;
    Buf<uint8_t> dec;
    Buf<int32_t> dm;
    float *qrot = nullptr, *ftab = nullptr;
    unsigned *counter = nullptr;
    CK(stage_in(sc, Qv, (size_t)nq * ix->D, q), "stage queries");
    CK(stage_in(sc, r2, (size_t)nq, rr), "stage r2");
    CK(stage_out(sc, decisions, (size_t)nq * ix->N, dec), "stage decisions");
    CK(stage_out(sc, dims, (size_t)nq * ix->N, dm), "stage dims");
    CK(sc.get(&qrot, (size_t)nq * ix->Dp), "alloc q'");
    CK(sc.get(&counter, 1), "alloc counter");
    CK(rotate_queries(ix, q.dev, nq, qrot, sc), "rotate");
    // The search's own scan kernel in its fixed-threshold mode: every
    // cluster is a probe slot, r^2 stays r2[q], no KNN set.
    adsx::ScanArgs a;
    if (!adsx::fill_uniform_scan(a, ix, nq, 1, ix->nlist, eps0, delta_d, 0))
        return fail(ADSX_EINVAL, "too many queries in one call");
    a.qrot = qrot;
    a.probes = nullptr;
    a.out_ids = nullptr;
    a.out_d2 = nullptr;
    a.work_counter = counter;
    a.r2fixed = rr.dev;
    a.decisions = dec.dev;
    a.dec_dims = dm.dev;
    a.N = ix->N;
    CK(sc.get(&ftab, (size_t)a.nblk + 1), "alloc test factors");
    a.ftab = ftab;
    CK(adsx::launch_test_factors(ftab, a.nblk, a.D, a.test_on ? eps0 : 0.f, s), "test factors");
    if (ix->sched == ADSX_SCHED_CLUSTER && a.db <= adsx::CM_MAX_DB) {
        // the cluster-major kernel's fixed-threshold mode: every query
        // probes every cluster, one round
        int32_t *probes = nullptr;
        CK(sc.get(&probes, (size_t)nq * ix->nlist), "alloc probe lists");
        CK(adsx::launch_cm_all_clusters(probes, nq, ix->nlist, s), "probe lists");
        adsx::CmPlan pl;
        adsx::CmRounds R;
        R.n = 1;
        R.lo[0] = 0;
        R.lo[1] = ix->nlist;
        int64_t icap[1];
        const int G = cm_queries_per_item(ix, nq, ix->nlist);
        CK(cm_plan_buffers(ix, nq, G, R, sc, pl, icap), "alloc plan");
        CK(adsx::launch_cm_plan(probes, nq, ix->nlist, R, ix->nlist, G, ix->cm_tpi, ix->off, pl, s),
           "plan");
        adsx::CmArgs c = cm_args_from(a, G);
        c.tpi = ix->cm_tpi;
        cm_round_args(c, pl, R, icap, nq, ix->nlist, 0);
        c.work_counter = counter;
        c.r2fixed = rr.dev;
        c.decisions = dec.dev;
        c.dec_dims = dm.dev;
        c.N = ix->N;
        c.out_dims = nullptr;
        CK(adsx::launch_cm_scan(c, ix->device, s), "fixed-r scan (cluster-major)");
    } else {
        CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), s), "clear counter");
        CK(adsx::launch_ads_scan(a, adsx::ads_scan_grid(a, ix->device), s), "fixed-r scan");
    }
    CK(copy_back(dec, s), "copy back");
    CK(copy_back(dm, s), "copy back");
    return finish(s, dec.host || dm.host, "fixed-r");
}

// One configuration of the search's tunables.
struct TuneCfg {
    int dd, sched, G, tpi, ip;
};

static void apply_cfg(Index *ix, const TuneCfg &c)
{
    ix->sched = c.sched;
    ix->cm_G = c.G;
    ix->cm_tpi = c.tpi;
    ix->items_per_sm = c.ip;
}

int adsx_autotune(adsx_index *index, const float *Qv, int64_t nq, int32_t K, int32_t nprobe,
                  float eps0, int32_t *best_delta_d, int32_t *best_items_per_sm, float *best_ms,
                  void *stream)
{
    Index *ix = reinterpret_cast<Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (nq < 1 || !Qv) return fail(ADSX_EINVAL, "autotune needs a non-empty query sample");
    if (K < 1 || K > ADSX_MAX_K || nprobe < 1 || nprobe > ix->nlist || nprobe > ADSX_MAX_NPROBE)
        return fail(ADSX_EINVAL, "K or nprobe out of range");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Buf<float> q;
    float *d2 = nullptr;
    int64_t *ids = nullptr;
    CK(stage_in(sc, Qv, (size_t)nq * ix->D, q), "stage queries");
    CK(sc.get(&d2, (size_t)nq * K), "alloc outputs");
    CK(sc.get(&ids, (size_t)nq * K), "alloc outputs");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const bool timing = ix->timing;
    ix->timing = false;
    const TuneCfg saved{ix->tuned_delta_d, ix->sched, ix->cm_G, ix->cm_tpi, ix->items_per_sm};
    // mean of three timed searches after a warm-up (CUDA events on `stream`)
    auto time_cfg = [&](const TuneCfg &c, float *ms_out) -> int {
        apply_cfg(ix, c);
        float tot = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            int r = adsx_search(index, q.dev, nq, K, nprobe, eps0, c.dd, ids, d2, nullptr, stream);
            cudaEventRecord(e1, s);
            if (r) return r;
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(ADSX_ECUDA, "autotune sync failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;
        }
        *ms_out = tot / 3.f;
        return ADSX_OK;
    };
    // Coordinate search: the step delta_d (Sec. 6.2.4's 16..64) under each
    // schedule, then the winning schedule's own shape -- queries per item and
    // tiles per item (cluster-major) or work items per SM (query-major).
    // *best_delta_d != 0 on entry keeps the step fixed at that value
    int dds[4] = {16, 32, 48, 64};
    int ndd = 4;
    if (best_delta_d && *best_delta_d != 0) {
        if ((rc = check_blocks(*best_delta_d, eps0))) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ix->timing = timing;
            return rc;
        }
        dds[0] = *best_delta_d;
        ndd = 1;
    }
    TuneCfg best = saved;
    float best_t = INFINITY;
    auto consider = [&](const TuneCfg &c) -> int {
        float t = 0.f;
        const int r = time_cfg(c, &t);
        if (r == ADSX_OK && t < best_t) {
            best_t = t;
            best = c;
        }
        return r;
    };
    for (int di = 0; di < ndd && rc == ADSX_OK; ++di) {
        if (ndd > 1 && dds[di] > ix->Dp) continue;
        rc = consider({dds[di], ADSX_SCHED_QUERY, saved.G, saved.tpi, 48});
        if (rc == ADSX_OK) rc = consider({dds[di], ADSX_SCHED_CLUSTER, 0, 2, 48});
    }
    const TuneCfg base = best;
    if (rc == ADSX_OK && base.sched == ADSX_SCHED_CLUSTER) {
        // queries per item (0: chosen per batch), then tiles per item
        const int Gs[4] = {4, 8, 16, 32}, tpis[3] = {1, 2, 4};
        for (int gi = 0; gi < 4 && rc == ADSX_OK; ++gi)
            if (Gs[gi] != base.G) rc = consider({base.dd, base.sched, Gs[gi], base.tpi, base.ip});
        const TuneCfg b2 = best;
        for (int ti = 0; ti < 3 && rc == ADSX_OK; ++ti)
            if (tpis[ti] != b2.tpi) rc = consider({b2.dd, b2.sched, b2.G, tpis[ti], b2.ip});
    } else if (rc == ADSX_OK) {
        const int ips[2] = {24, 96};
        for (int ii = 0; ii < 2 && rc == ADSX_OK; ++ii)
            rc = consider({base.dd, base.sched, base.G, base.tpi, ips[ii]});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ix->timing = timing;
    if (rc) {
        apply_cfg(ix, saved);
        return rc;
    }
    apply_cfg(ix, best);
    ix->tuned_delta_d = best.dd;
    if (best_delta_d) *best_delta_d = best.dd;
    if (best_items_per_sm) *best_items_per_sm = best.ip;
    if (best_ms) *best_ms = best_t;
    return ADSX_OK;
}

int adsx_scan_config(const adsx_index *index, int32_t *delta_d, int32_t *schedule,
                     int32_t *queries_per_item, int32_t *tiles_per_item, int32_t *items_per_sm)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    if (!ix) return fail(ADSX_EINVAL, "index is NULL");
    if (delta_d) *delta_d = ix->tuned_delta_d;
    if (schedule) *schedule = ix->sched;
    if (queries_per_item) *queries_per_item = ix->cm_G;
    if (tiles_per_item) *tiles_per_item = ix->cm_tpi;
    if (items_per_sm) *items_per_sm = ix->items_per_sm;
    return ADSX_OK;
}

int adsx_set_scan_schedule(adsx_index *index, int32_t schedule, int32_t queries_per_item,
                           int32_t tiles_per_item)
{
    Index *ix = reinterpret_cast<Index *>(index);
    if (!ix) return fail(ADSX_EINVAL, "index is NULL");
    if (schedule != ADSX_SCHED_AUTO && schedule != ADSX_SCHED_QUERY &&
        schedule != ADSX_SCHED_CLUSTER)
        return fail(ADSX_EINVAL, "unknown scan schedule %d", schedule);
    if (queries_per_item < -1 || queries_per_item > adsx::CM_MAX_G)
        return fail(ADSX_EINVAL, "queries_per_item out of range (-1..%d)", adsx::CM_MAX_G);
    if (tiles_per_item < 0 || tiles_per_item > 64)
        return fail(ADSX_EINVAL, "tiles_per_item out of range (0..64)");
    ix->sched = schedule;
    if (queries_per_item) ix->cm_G = queries_per_item < 0 ? 0 : queries_per_item;
    if (tiles_per_item) ix->cm_tpi = tiles_per_item;
    return ADSX_OK;
}

int adsx_set_query_rotation(adsx_index *index, int32_t mode)
{
    Index *ix = reinterpret_cast<Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (mode != ADSX_ROT_FP32 && mode != ADSX_ROT_TENSOR)
        return fail(ADSX_EINVAL, "unknown query rotation mode %d", mode);
    if (mode == ADSX_ROT_TENSOR && !ix->rot_ok)
        return fail(ADSX_EINVAL, "tensor-core rotation needs a dense P and a padded D <= 1024");
    ix->rot_tc = mode == ADSX_ROT_TENSOR;
    return ADSX_OK;
}

int adsx_set_stage_timing(adsx_index *index, int32_t enable)
{
    Index *ix = reinterpret_cast<Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (enable && !ix->ev[0]) {
        for (cudaEvent_t &e : ix->ev) CK(cudaEventCreate(&e), "create event");
        for (cudaEvent_t &e : ix->kev) CK(cudaEventCreate(&e), "create event");
    }
    ix->timing = enable != 0;
    return ADSX_OK;
}

int adsx_stage_ms(const adsx_index *index, float *ms)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (!ms) return fail(ADSX_EINVAL, "ms is NULL");
    if (!ix->timed_once || !ix->ev[0]) return fail(ADSX_EINVAL, "no timed search has run");
    CK(cudaEventSynchronize(ix->ev[4]), "event sync");
    for (int i = 0; i < 4; ++i) CK(cudaEventElapsedTime(&ms[i], ix->ev[i], ix->ev[i + 1]), "elapsed");
    return ADSX_OK;
}

int adsx_scan_kernel_ms(const adsx_index *index, float *ms, int32_t *launches)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    if (!ms) return fail(ADSX_EINVAL, "ms is NULL");
    if (!ix->timed_once || !ix->ev[0]) return fail(ADSX_EINVAL, "no timed search has run");
    CK(cudaEventSynchronize(ix->ev[4]), "event sync");
    float tot = 0.f;
    for (int i = 0; i < ix->nkev; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ix->kev[2 * i], ix->kev[2 * i + 1]), "elapsed");
        tot += t;
    }
    *ms = tot;
    if (launches) *launches = ix->nkev;
    return ADSX_OK;
}

int adsx_stream_status(const adsx_index *index, void *stream)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    int rc = check_index(ix);
    if (rc) return rc;
    CK(cudaStreamSynchronize((cudaStream_t)stream), "sync");
    unsigned err = 0;
    CK(cudaMemcpy(&err, ix->err, sizeof err, cudaMemcpyDeviceToHost), "read error word");
    if (err) {
        cudaMemset(ix->err, 0, sizeof(unsigned));
        if (err & (adsx::ERR_BATCH_ARGS | adsx::ERR_OUT_RANGE))
            return fail(ADSX_EINVAL, "device-side argument check failed (error word 0x%x)", err);
        return fail(ADSX_ETIMEOUT, "a bounded device wait gave up (error word 0x%x)", err);
    }
    return ADSX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- graph search
// HNSW+ (Sec. 4) on a kNN proximity graph over an FP32 L2 or cosine index; kernels in
// graph.cu.  The graph owns its device memory and, once a search has run, the
// per-warp scratch of the visited test (reused by later searches).
struct Graph {
    int64_t N = 0;
    int32_t degree = 0, nlist = 0, device = 0, n_ce = 1;
    int32_t *nbr = nullptr;      // N x degree
    int64_t *entry = nullptr;    // nlist x n_ce
    int64_t *vbase = nullptr;    // N
    int32_t *vstride = nullptr;  // N
    unsigned *bitmap = nullptr;  // warps x bm_words (all zero between queries)
    int32_t *vlist = nullptr;    // warps x vcap
    unsigned long long *qnext = nullptr;  // the search's query counter
    int64_t bm_words = 0, vcap = 0;
    int32_t warps = 0;           // warps the scratch holds
};

extern "C" {

int adsx_free_graph(adsx_graph *graph)
{
    Graph *g = reinterpret_cast<Graph *>(graph);
    if (!g) return ADSX_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->nbr);
    cudaFree(g->entry);
    cudaFree(g->vbase);
    cudaFree(g->vstride);
    cudaFree(g->bitmap);
    cudaFree(g->vlist);
    cudaFree(g->qnext);
    delete g;
    return ADSX_OK;
}

int adsx_build_graph(const adsx_index *index, const float *X, int32_t degree, int32_t nprobe,
                     int32_t entries_per_cluster, void *stream, adsx_graph **out)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    if (!out) return fail(ADSX_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_index(ix);
    if (rc) return rc;
    if (ix->storage != ADSX_F32 || (ix->metric != ADSX_L2 && ix->metric != ADSX_COSINE))
        return fail(ADSX_EINVAL, "graph search needs an FP32 L2 or cosine index");
    if (!X) return fail(ADSX_EINVAL, "X is NULL");
    if (degree < 1 || degree > ADSX_MAX_DEGREE)
        return fail(ADSX_EINVAL, "degree out of range (1..%d)", ADSX_MAX_DEGREE);
    if (nprobe < 1 || nprobe > ix->nlist || nprobe > ADSX_MAX_NPROBE)
        return fail(ADSX_EINVAL, "nprobe out of range (1..min(nlist, %d))", ADSX_MAX_NPROBE);
    if (entries_per_cluster < 1 || entries_per_cluster > ADSX_MAX_CLUSTER_ENTRIES)
        return fail(ADSX_EINVAL, "entries_per_cluster out of range (1..%d)", ADSX_MAX_CLUSTER_ENTRIES);
    cudaStream_t s = (cudaStream_t)stream;
    Graph *g = new Graph();
    g->n_ce = entries_per_cluster;
    g->N = ix->N;
    g->degree = degree;
    g->nlist = ix->nlist;
    g->device = ix->device;
    auto cleanup = [&](int r) {
        adsx_free_graph(reinterpret_cast<adsx_graph *>(g));
        return r;
    };
    cudaError_t e;
#define GCK(call, what)                                          \
    do {                                                         \
        e = (call);                                              \
        if (e != cudaSuccess) return cleanup(cuda_fail(e, what)); \
    } while (0)
    GCK(cudaMalloc(&g->nbr, sizeof(int32_t) * (size_t)g->N * degree), "alloc graph");
    GCK(cudaMalloc(&g->entry, sizeof(int64_t) * (size_t)g->nlist * g->n_ce), "alloc graph");
    GCK(cudaMalloc(&g->vbase, sizeof(int64_t) * (size_t)g->N), "alloc graph");
    GCK(cudaMalloc(&g->vstride, sizeof(int32_t) * (size_t)g->N), "alloc graph");
    {
        // Each vertex's degree nearest others among its nprobe nearest
        // clusters: the library's exact IVF search with every vertex as a
        // query, in chunks (its centroid-distance matrix is chunk x nlist).
        const int Kk = degree + 1;
        const int64_t chunk = 65536;
        int64_t *knn = nullptr;
        float *kd = nullptr;
        GCK(cudaMalloc(&knn, sizeof(int64_t) * (size_t)std::min(chunk, g->N) * Kk), "alloc kNN");
        e = cudaMalloc(&kd, sizeof(float) * (size_t)std::min(chunk, g->N) * Kk);
        if (e != cudaSuccess) {
            cudaFree(knn);
            return cleanup(cuda_fail(e, "alloc kNN"));
        }
        for (int64_t r0 = 0; r0 < g->N && rc == 0; r0 += chunk) {
            const int64_t n = std::min(chunk, g->N - r0);
            rc = search_impl(index, X + r0 * ix->D, n, Kk, nprobe, INFINITY, 32, knn, kd, nullptr,
                             stream, 0);
            if (rc == 0) {
                e = adsx::launch_knn_to_graph(knn, n, r0, Kk, degree, g->nbr + r0 * degree, s);
                if (e != cudaSuccess) rc = cuda_fail(e, "graph rows");
            }
        }
        cudaStreamSynchronize(s);
        cudaFree(knn);
        cudaFree(kd);
        if (rc) return cleanup(rc);
    }
    GCK(adsx::launch_vertex_map(ix->off, ix->nlist, ix->ids, ix->Dp, g->vbase, g->vstride, s), "vertex map");
    {
        float *mind = nullptr;
        GCK(cudaMalloc(&mind, sizeof(float) * (size_t)std::max<int64_t>(g->N, 1)), "alloc entry scratch");
        e = adsx::launch_cluster_entries(static_cast<const float *>(ix->data), ix->off, ix->ids, ix->cents,
                                         ix->nlist, ix->Dp, g->n_ce, mind, g->entry, s);
        const cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(mind);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "cluster entries"));
    }
#undef GCK
    *out = reinterpret_cast<adsx_graph *>(g);
    return ADSX_OK;
}

int adsx_graph_export(const adsx_graph *graph, int32_t *neighbors, int64_t *entries)
{
    const Graph *g = reinterpret_cast<const Graph *>(graph);
    if (!g) return fail(ADSX_EINVAL, "graph is NULL");
    cudaSetDevice(g->device);
    cudaError_t e = cudaSuccess;
    if (neighbors)
        e = cudaMemcpy(neighbors, g->nbr, sizeof(int32_t) * (size_t)g->N * g->degree, cudaMemcpyDefault);
    if (e == cudaSuccess && entries)
        e = cudaMemcpy(entries, g->entry, sizeof(int64_t) * (size_t)g->nlist * g->n_ce, cudaMemcpyDefault);
    return e == cudaSuccess ? ADSX_OK : cuda_fail(e, "graph export");
}

int adsx_graph_info(const adsx_graph *graph, int64_t *N, int32_t *degree, int32_t *nlist,
                    int32_t *entries_per_cluster)
{
    const Graph *g = reinterpret_cast<const Graph *>(graph);
    if (!g) return fail(ADSX_EINVAL, "graph is NULL");
    if (N) *N = g->N;
    if (degree) *degree = g->degree;
    if (nlist) *nlist = g->nlist;
    if (entries_per_cluster) *entries_per_cluster = g->n_ce;
    return ADSX_OK;
}

int adsx_search_graph(const adsx_index *index, const adsx_graph *graph, const float *Qv,
                      int64_t nq, int32_t K, int32_t ef, int32_t n_entry, int32_t decoupled,
                      float eps0, int32_t delta_d, int64_t *ids, float *dists,
                      int64_t *dims_read, void *stream)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    Graph *g = const_cast<Graph *>(reinterpret_cast<const Graph *>(graph));
    int rc = check_index(ix);
    if (rc) return rc;
    if (!g || g->N != ix->N || g->nlist != ix->nlist) return fail(ADSX_EINVAL, "graph does not match the index");
    if (ix->storage != ADSX_F32 || (ix->metric != ADSX_L2 && ix->metric != ADSX_COSINE))
        return fail(ADSX_EINVAL, "graph search needs an FP32 L2 or cosine index");
    if (nq < 0 || (nq > 0 && (!Qv || !ids || !dists))) return fail(ADSX_EINVAL, "bad query arguments");
    if (ef < 1 || ef > ADSX_MAX_EF) return fail(ADSX_EINVAL, "ef out of range (1..%d)", ADSX_MAX_EF);
    if (K < 1 || K > ef) return fail(ADSX_EINVAL, "K out of range (1..ef)");
    if (decoupled != 0 && decoupled != 1) return fail(ADSX_EINVAL, "decoupled must be 0 or 1");
    if (n_entry < 1 || n_entry > ADSX_MAX_GRAPH_ENTRIES || n_entry > ix->nlist)
        return fail(ADSX_EINVAL, "n_entry out of range (1..min(nlist, %d))", ADSX_MAX_GRAPH_ENTRIES);
    if (delta_d == 0) delta_d = ix->tuned_delta_d;
    if ((rc = check_blocks(delta_d, eps0))) return rc;
    if (nq == 0) return ADSX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int max_iter = 4 * ef;
    // Algorithm 1 steps per DCO (the test off: one full-width step)
    const int gnblk = ix->Dp / adsx::BLK;
    int gdb = delta_d / adsx::BLK;
    const bool gtest = !isinf(eps0) && gdb < gnblk;
    if (!gtest) gdb = gnblk;
    const int nst = (gnblk + gdb - 1) / gdb;
    // per-warp scratch of the visited test, kept with the graph (grown,
    // never shrunk: a search uses the first `warps` slots)
    int32_t warps = 0;
    {
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ix->device);
        warps = adsx::graph_search_resident_warps(ix->Dp, ef, K, nst, nsm);
        if (warps <= 0) return fail(ADSX_EINVAL, "graph search: ef and D need more shared memory than an SM has");
        const int64_t bm_words = (g->N + 31) / 32;
        // visited ids are distinct: never more than N of them
        const int64_t vcap = std::min<int64_t>(1 + (int64_t)ADSX_MAX_GRAPH_ENTRIES * ADSX_MAX_CLUSTER_ENTRIES +
                                                   (int64_t)max_iter * g->degree,
                                               g->N);
        if (g->warps < warps || g->bm_words != bm_words || g->vcap < vcap || !g->qnext) {
            cudaStreamSynchronize(s);
            cudaFree(g->bitmap);
            cudaFree(g->vlist);
            cudaFree(g->qnext);
            g->bitmap = nullptr;
            g->vlist = nullptr;
            g->qnext = nullptr;
            g->warps = 0;
            cudaError_t e = cudaMalloc(&g->bitmap, sizeof(unsigned) * (size_t)warps * bm_words);
            if (e == cudaSuccess) e = cudaMalloc(&g->vlist, sizeof(int32_t) * (size_t)warps * vcap);
            if (e == cudaSuccess) e = cudaMalloc(&g->qnext, sizeof(unsigned long long));
            if (e == cudaSuccess) e = cudaMemset(g->bitmap, 0, sizeof(unsigned) * (size_t)warps * bm_words);
            if (e != cudaSuccess) {
                cudaFree(g->bitmap);
                cudaFree(g->vlist);
                cudaFree(g->qnext);
                g->bitmap = nullptr;
                g->vlist = nullptr;
                g->qnext = nullptr;
                return cuda_fail(e, "alloc graph search scratch");
            }
            g->warps = warps;
            g->bm_words = bm_words;
            g->vcap = vcap;
        }
    }
    Scratch sc(s);
    Buf<float> q, od;
    Buf<int64_t> oi, odims;
    float *qrot = nullptr, *ftab = nullptr;
    int32_t *probes = nullptr;
    const int nblk = ix->Dp / adsx::BLK;
    CK(stage_in(sc, Qv, (size_t)nq * ix->D, q), "stage queries");
    CK(stage_out(sc, ids, (size_t)nq * K, oi), "stage ids");
    CK(stage_out(sc, dists, (size_t)nq * K, od), "stage dists");
    CK(stage_out(sc, dims_read, (size_t)nq, odims), "stage dims");
    CK(sc.get(&qrot, (size_t)nq * ix->Dp), "alloc q'");
    CK(sc.get(&probes, (size_t)nq * n_entry), "alloc probes");
    CK(sc.get(&ftab, (size_t)nblk + 1), "alloc test factors");
    CK(rotate_queries(ix, q.dev, nq, qrot, sc), "rotate");
    CK(queries_before_probe(ix, qrot, nq, s), "normalise queries");
    CK(probe_queries(ix, qrot, nq, n_entry, probes, nullptr, sc), "entry clusters");
    adsx::GraphArgs a;
    a.data = static_cast<const float *>(ix->data);
    a.vbase = g->vbase;
    a.vstride = g->vstride;
    a.nbr = g->nbr;
    a.degree = g->degree;
    a.entry = g->entry;
    a.n_ce = g->n_ce;
    a.qrot = qrot;
    a.probes = probes;
    a.n_entry = n_entry;
    a.ftab = ftab;
    a.nq = nq;
    a.D = ix->D;
    a.Dp = ix->Dp;
    a.nblk = nblk;
    a.db = gdb;
    a.test_on = gtest ? 1 : 0;
    a.nst = nst;
    a.K = K;
    a.ef = ef;
    a.max_iter = max_iter;
    a.pp = decoupled;
    a.metric = ix->metric;
    a.out_ids = oi.dev;
    a.out_d2 = od.dev;
    a.out_dims = odims.dev;
    a.bitmap = g->bitmap;
    a.bm_words = g->bm_words;
    a.vlist = g->vlist;
    a.vcap = g->vcap;
    a.warps = warps;
    a.qnext = g->qnext;
    CK(adsx::launch_test_factors(ftab, nblk, ix->D, a.test_on ? eps0 : 0.f, s, 0), "test factors");
    CK(adsx::launch_graph_search(a, s), "graph search");
    CK(copy_back(oi, s), "copy back");
    CK(copy_back(od, s), "copy back");
    CK(copy_back(odims, s), "copy back");
    return finish(s, oi.host || od.host || odims.host, "graph search");
}

}  // extern "C"
