// noalloc.cu -- adsx_search_noalloc: the search pipeline of adsx_search with
// every temporary buffer carved from one fixed, file-scope device array
// instead of the stream-ordered allocator.
//
// Who needs it: callers that must not allocate device memory on the query
// path -- for example a serving process whose GPU memory is reserved up front
// by another allocator or a fixed budget, where cudaMalloc/cudaMallocAsync
// would fail, or would take a lock or synchronise and stall other work.
//
// The array is a static __device__ object, so every GPU that loads this
// library holds ADSX_NOALLOC_SCRATCH_BYTES of it until the process exits.  In
// host code the array's name is only a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) on the first call made on that device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "adsx_internal.cuh"

namespace {

constexpr int MAX_DEVICES = 64;

// The shared scratch of adsx_search_noalloc.  Every call uses it, and it keeps
// whatever the last call left in it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ADSX_NOALLOC_SCRATCH_BYTES];

int nerr(int code, const std::string &msg)
{
    adsx::set_last_error(msg);
    return code;
}

// Device (or managed) memory that lives on `device`: the kernels read and
// write these buffers directly.
bool is_device_ptr_on(const void *p, int device)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

// Device address of the scratch array in the current context, looked up on
// every call (a cheap runtime query): a cached address would dangle after
// the context is destroyed and re-created (cudaDeviceReset).
int scratch_base(int device, unsigned char **out)
{
    if (device < 0 || device >= MAX_DEVICES) return nerr(ADSX_EINVAL, "device id out of range");
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return nerr(ADSX_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    }
    *out = static_cast<unsigned char *>(p);
    return ADSX_OK;
}

// Bump carving of the fixed array, 256-byte aligned pieces.
struct Carver {
    unsigned char *base;
    size_t used = 0;
    template <typename T>
    T *take(size_t count)
    {
        size_t bytes = (std::max<size_t>(count * sizeof(T), 1) + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

}  // namespace

extern "C" int adsx_search_noalloc(const adsx_index *index, const float *Qv, int64_t nq,
                                   int32_t K, int32_t nprobe, float eps0, int32_t delta_d,
                                   int64_t *ids, float *dists, int64_t *dims_read, void *stream)
{
    const adsx::Index *ix = reinterpret_cast<const adsx::Index *>(index);
    if (!ix) return nerr(ADSX_EINVAL, "index is NULL");
    if (ix->metric != ADSX_L2) return nerr(ADSX_EINVAL, "adsx_search_noalloc supports L2 indexes only");
    cudaError_t e = cudaSetDevice(ix->device);
    if (e != cudaSuccess) return nerr(ADSX_ECUDA, cudaGetErrorString(e));
    if (nq < 0) return nerr(ADSX_EINVAL, "nq < 0");
    if (K < 1 || K > ADSX_MAX_K) return nerr(ADSX_EINVAL, "K out of range");
    if (nprobe < 1 || nprobe > ix->nlist || nprobe > ADSX_MAX_NPROBE)
        return nerr(ADSX_EINVAL, "nprobe out of range");
    if (delta_d == 0) delta_d = ix->tuned_delta_d;   // as adsx_search: the tuned step
    if (delta_d < 16 || delta_d % 16) return nerr(ADSX_EINVAL, "delta_d must be a positive multiple of 16");
    if (!(eps0 >= 0.f)) return nerr(ADSX_EINVAL, "eps0 must be >= 0");
    if (nq == 0) return ADSX_OK;
    if (!is_device_ptr_on(Qv, ix->device) || !is_device_ptr_on(ids, ix->device) ||
        !is_device_ptr_on(dists, ix->device) ||
        (dims_read && !is_device_ptr_on(dims_read, ix->device)))
        return nerr(ADSX_EINVAL, "adsx_search_noalloc takes device pointers of the index's GPU only");

    const int Dp = ix->Dp, nblk = Dp / adsx::BLK;
    adsx::ScanArgs a;
    if (!adsx::fill_uniform_scan(a, ix, nq, K, nprobe, eps0, delta_d, 0))
        return nerr(ADSX_EINVAL, "too many queries");

    // Size check before touching the array.
    auto rup = [](size_t b) { return (std::max<size_t>(b, 1) + 255) & ~size_t(255); };
    // the centroid distances share their region with the partial sums of a
    // tensor-core query rotation (used one after the other)
    const size_t rot_part =
        ix->rot_tc ? (size_t)adsx::tc_rot_scratch_floats(ix, std::min<int64_t>(nq, 1024)) * 4 : 0;
    const size_t dist_bytes = std::max<size_t>((size_t)nq * ix->nlist * 4, rot_part);
    const size_t split_bytes = (size_t)adsx::tf32_split_words(nq, Dp) * 4;
    size_t need = rup((size_t)nq * Dp * 4) + rup((size_t)nq * 4) + rup(split_bytes) + rup(dist_bytes) +
                  rup((size_t)nq * nprobe * 4) + rup((size_t)(nblk + 1) * 4) + rup(4) +
                  (ix->rot_tc ? rup((size_t)nq * 4) : 0);
    if (a.S > 1) need += rup((size_t)nq * 4) + 2 * rup((size_t)a.n_items * K * 4);
    if (need > (size_t)ADSX_NOALLOC_SCRATCH_BYTES)
        return nerr(ADSX_EINVAL, "adsx_search_noalloc: this call needs " + std::to_string(need) +
                                     " bytes of scratch, above the fixed maximum of " +
                                     std::to_string((long long)ADSX_NOALLOC_SCRATCH_BYTES) +
                                     " (split the batch)");

    unsigned char *base = nullptr;
    int rc = scratch_base(ix->device, &base);
    if (rc) return rc;
    Carver cv{base};
    float *qrot = cv.take<float>((size_t)nq * Dp);
    float *qn = cv.take<float>((size_t)nq);
    uint32_t *qs = cv.take<uint32_t>(split_bytes / 4);
    float *dist = cv.take<float>(dist_bytes / 4);
    int32_t *probes = cv.take<int32_t>((size_t)nq * nprobe);
    float *ftab = cv.take<float>((size_t)nblk + 1);
    unsigned *counter = cv.take<unsigned>(1);
    a.qrot = qrot;
    a.probes = probes;
    a.ftab = ftab;
    a.work_counter = counter;
    a.out_ids = ids;
    a.out_d2 = dists;
    a.out_dims = dims_read;
    cudaStream_t s = (cudaStream_t)stream;
    // The array keeps the previous call's contents: clear what must start
    // from a known value.
    if (a.S > 1) {
        a.r2g = cv.take<unsigned>((size_t)nq);
        a.part_d = cv.take<float>((size_t)a.n_items * K);
        a.part_i = cv.take<int32_t>((size_t)a.n_items * K);
        e = cudaMemsetAsync(a.r2g, 0xff, sizeof(unsigned) * nq, s);
        if (e == cudaSuccess && dims_read) e = cudaMemsetAsync(dims_read, 0, sizeof(int64_t) * nq, s);
        if (e != cudaSuccess) return nerr(ADSX_ECUDA, cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        if (ix->rot_tc)
            e = adsx::rotate_queries_tc(ix, Qv, nq, qrot, dist, (int64_t)(dist_bytes / 4),
                                        cv.take<int32_t>((size_t)nq), s);
        else
            e = adsx::rotate_rows(ix, Qv, nq, qrot, s);
    }
    if (e == cudaSuccess) e = adsx::launch_row_sqnorm(qrot, nq, Dp, Dp, qn, s);
    if (e == cudaSuccess) e = adsx::launch_tf32_split(qrot, nq, Dp, Dp, qs, s);
    if (e == cudaSuccess)
        e = adsx::launch_tc_gemm(qs, nq, ix->cents_split, Dp, dist, ix->nlist, ix->nlist, qn,
                                 ix->cnorm, ix->err, s);
    if (e == cudaSuccess)
        e = adsx::launch_select_nprobe(dist, nq, ix->nlist, nprobe, probes, nullptr, s);
    if (e == cudaSuccess)
        e = adsx::launch_test_factors(ftab, nblk, ix->D, a.test_on ? eps0 : 0.f, s);
    if (e == cudaSuccess) e = adsx::launch_ads_scan(a, adsx::ads_scan_grid(a, ix->device), s);
    if (e == cudaSuccess) e = adsx::launch_finalize_topk(a, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nerr(ADSX_ECUDA, std::string("adsx_search_noalloc: ") + cudaGetErrorString(e));
    }
    return ADSX_OK;
}
