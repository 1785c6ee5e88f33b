// persist.cu -- adsx_save_index / adsx_load_index: an index written to a
// file and read back (the paper stores P at index time, Sec. 6.1
// "Implementation"; here the whole built index is kept, so that a process
// can search without repeating the rotation of the data and the layout).
//
// File format (native byte order; the reading host must match the writer's):
//   8 bytes   "ADSXIDX1"
//   header    a fixed block of int64 fields (FileHeader below)
//   arrays    in a fixed order, each as raw bytes of the size the header
//             implies: P or the Kac walk, centroids and their norms, the
//             dim-blocked data, the FP32 rows and norms (16-bit storage),
//             the raw norms (inner product), ids, CSR and tile offsets, and
//             the digits of P for the tensor-core rotation when present
//   8 bytes   FNV-1a hash of every byte after the magic
// A file that is short, has another magic, fields out of the library's
// limits or a wrong hash is rejected with ADSX_EINVAL.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "adsx_internal.cuh"

using adsx::Index;

namespace {

constexpr char MAGIC[8] = {'A', 'D', 'S', 'X', 'I', 'D', 'X', '1'};

struct FileHeader {
    int64_t N, D, Dp, nlist, storage, metric, kac_L, total_tiles, max_tiles;
    int64_t tuned_delta_d, items_per_sm, sched, cm_G, cm_tpi;
    int64_t has_P, rot_ok, rot_b, rot_T, rot_Lmax, rot_floats;
    int64_t rot_boff[16];
};

int perr(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    adsx::set_last_error(buf);
    return code;
}

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n)
    {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

size_t elem_bytes(int64_t storage) { return storage == ADSX_F32 ? 4 : 2; }

// The arrays of an index, in file order: device pointer slot and byte size.
struct Part {
    void **dev;
    size_t bytes;
};

std::vector<Part> parts_of(Index *ix, const FileHeader &h)
{
    std::vector<Part> p;
    const size_t N = (size_t)h.N, Dp = (size_t)h.Dp, nl = (size_t)h.nlist;
    if (h.has_P) p.push_back({(void **)&ix->P, sizeof(float) * Dp * Dp});
    if (h.kac_L > 0) {
        const size_t cnt = (size_t)h.kac_L * 2 * (size_t)(h.D / 2);
        p.push_back({(void **)&ix->kac_pairs, sizeof(int32_t) * cnt});
        p.push_back({(void **)&ix->kac_cs, sizeof(float) * cnt});
    }
    p.push_back({(void **)&ix->cents, sizeof(float) * nl * Dp});
    p.push_back({(void **)&ix->cnorm, sizeof(float) * nl});
    p.push_back({(void **)&ix->data, elem_bytes(h.storage) * N * Dp});
    if (h.storage != ADSX_F32) {
        p.push_back({(void **)&ix->rows32, sizeof(float) * N * Dp});
        p.push_back({(void **)&ix->norms, sizeof(float) * N});
    }
    if (h.metric == ADSX_IP) p.push_back({(void **)&ix->onorm, sizeof(float) * N});
    p.push_back({(void **)&ix->ids, sizeof(int32_t) * N});
    p.push_back({(void **)&ix->off, sizeof(int64_t) * (nl + 1)});
    p.push_back({(void **)&ix->tile_off, sizeof(int32_t) * (nl + 1)});
    if (h.rot_ok) {
        p.push_back({(void **)&ix->rot_B, sizeof(float) * (size_t)h.rot_floats});
        p.push_back({(void **)&ix->rot_F, sizeof(int32_t) * Dp});
    }
    return p;
}

constexpr size_t CHUNK = (size_t)64 << 20;   // bytes moved per host buffer fill

// Where the digits of P for the tensor-core rotation sit: per level
// L = 2..Lmax a Dp x (digit pairs of L) Dp matrix, one after another.
int64_t rot_layout(int64_t Dp, int64_t T, int64_t Lmax, int64_t *boff)
{
    int64_t total = 0;
    for (int L = 0; L < 16; ++L) boff[L] = 0;
    for (int64_t L = 2; L <= Lmax; ++L) {
        const int64_t lo = L - T > 1 ? L - T : 1, hi = L - 1 < T ? L - 1 : T;
        boff[L] = total;
        total += (hi - lo + 1) * Dp * Dp;
    }
    return total;
}

template <class T>
bool to_host(std::vector<T> &v, const T *dev, size_t n)
{
    v.resize(n);
    return cudaMemcpy(v.data(), dev, sizeof(T) * n, cudaMemcpyDeviceToHost) == cudaSuccess;
}

// The index arrays that kernels use as indexes, checked after a load: CSR
// and tile offsets consistent with each other, ids a permutation's range,
// every Kac-walk layer a set of distinct dims.  Returns the problem or "".
std::string check_indexes(Index *ix)
{
    const int64_t nl = ix->nlist;
    if (!to_host(ix->h_off, ix->off, (size_t)nl + 1)) return "copy offsets";
    if (ix->h_off[0] != 0 || ix->h_off[(size_t)nl] != ix->N) return "inconsistent CSR offsets";
    std::vector<int32_t> t;
    if (!to_host(t, ix->tile_off, (size_t)nl + 1)) return "copy tile offsets";
    int64_t mx = 0;
    if (t[0] != 0) return "inconsistent tile offsets";
    for (int64_t c = 0; c < nl; ++c) {
        const int64_t n = ix->h_off[(size_t)c + 1] - ix->h_off[(size_t)c];
        if (n < 0) return "inconsistent CSR offsets";
        if ((int64_t)t[(size_t)c + 1] - t[(size_t)c] != (n + 31) / 32) return "inconsistent tile offsets";
        mx = (n + 31) / 32 > mx ? (n + 31) / 32 : mx;
    }
    if (t[(size_t)nl] != ix->total_tiles || mx != ix->max_tiles) return "inconsistent tile counts";
    std::vector<int32_t> ids;
    if (!to_host(ids, ix->ids, (size_t)ix->N)) return "copy ids";
    for (int32_t id : ids)
        if (id < 0 || (int64_t)id >= ix->N) return "id out of range";
    if (ix->kac_L > 0) {
        const size_t m = (size_t)(ix->D / 2);
        std::vector<int32_t> pr;
        if (!to_host(pr, ix->kac_pairs, (size_t)ix->kac_L * 2 * m)) return "copy Kac walk";
        std::vector<int32_t> stamp((size_t)ix->D, -1);
        for (int32_t l = 0; l < ix->kac_L; ++l)
            for (size_t k = 0; k < 2 * m; ++k) {
                const int32_t i = pr[(size_t)l * 2 * m + k];
                if (i < 0 || i >= ix->D || stamp[(size_t)i] == l) return "malformed Kac walk";
                stamp[(size_t)i] = l;
            }
    }
    return "";
}

}  // namespace

extern "C" int adsx_save_index(const adsx_index *index, const char *path, void *stream)
{
    const Index *ix = reinterpret_cast<const Index *>(index);
    if (!ix || !ix->off) return perr(ADSX_EINVAL, "index is NULL or freed");
    if (!path) return perr(ADSX_EINVAL, "path is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return perr(ADSX_ECUDA, "sync: %s", cudaGetErrorString(e));
    FileHeader h;
    memset(&h, 0, sizeof h);
    h.N = ix->N;
    h.D = ix->D;
    h.Dp = ix->Dp;
    h.nlist = ix->nlist;
    h.storage = ix->storage;
    h.metric = ix->metric;
    h.kac_L = ix->kac_L;
    h.total_tiles = ix->total_tiles;
    h.max_tiles = ix->max_tiles;
    h.tuned_delta_d = ix->tuned_delta_d;
    h.items_per_sm = ix->items_per_sm;
    h.sched = ix->sched;
    h.cm_G = ix->cm_G;
    h.cm_tpi = ix->cm_tpi;
    h.has_P = ix->P != nullptr;
    h.rot_ok = ix->rot_ok;
    h.rot_b = ix->rot_b;
    h.rot_T = ix->rot_T;
    h.rot_Lmax = ix->rot_Lmax;
    int64_t boff[16];
    h.rot_floats = ix->rot_ok ? rot_layout(ix->Dp, ix->rot_T, ix->rot_Lmax, boff) : 0;
    for (int i = 0; i < 16; ++i) h.rot_boff[i] = ix->rot_boff[i];

    FILE *f = fopen(path, "wb");
    if (!f) return perr(ADSX_EINVAL, "cannot open %s for writing", path);
    Fnv fnv;
    bool ok = fwrite(MAGIC, 1, 8, f) == 8 && fwrite(&h, sizeof h, 1, f) == 1;
    fnv.add(&h, sizeof h);
    Index *mx = const_cast<Index *>(ix);
    std::vector<unsigned char> buf;
    for (const Part &p : parts_of(mx, h)) {
        for (size_t o = 0; ok && o < p.bytes; o += CHUNK) {
            const size_t n = p.bytes - o < CHUNK ? p.bytes - o : CHUNK;
            buf.resize(n);
            e = cudaMemcpy(buf.data(), static_cast<unsigned char *>(*p.dev) + o, n,
                           cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                fclose(f);
                return perr(ADSX_ECUDA, "copy index to host: %s", cudaGetErrorString(e));
            }
            fnv.add(buf.data(), n);
            ok = fwrite(buf.data(), 1, n, f) == n;
        }
    }
    ok = ok && fwrite(&fnv.h, sizeof fnv.h, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return perr(ADSX_EINVAL, "writing %s failed", path);
    return ADSX_OK;
}

extern "C" int adsx_load_index(const char *path, void *stream, adsx_index **out)
{
    if (!out) return perr(ADSX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!path) return perr(ADSX_EINVAL, "path is NULL");
    FILE *f = fopen(path, "rb");
    if (!f) return perr(ADSX_EINVAL, "cannot open %s", path);
    char magic[8];
    FileHeader h;
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, MAGIC, 8) != 0 || fread(&h, sizeof h, 1, f) != 1) {
        fclose(f);
        return perr(ADSX_EINVAL, "%s is not an adsx index file", path);
    }
    // the header's fields within the library's limits
    const bool sane =
        h.N >= 1 && h.N < ((int64_t)1 << 31) && h.D >= 1 && h.D <= ADSX_MAX_D &&
        h.Dp == (h.D + 15) / 16 * 16 && h.nlist >= 1 && h.nlist <= ADSX_MAX_NLIST && h.nlist <= h.N &&
        (h.storage == ADSX_F32 || h.storage == ADSX_BF16 || h.storage == ADSX_F16) &&
        (h.metric == ADSX_L2 || h.metric == ADSX_IP || h.metric == ADSX_COSINE) &&
        h.kac_L >= 0 && h.kac_L <= ADSX_MAX_KAC_LAYERS && (h.has_P == 0 || h.has_P == 1) &&
        (h.has_P == 1) == (h.kac_L == 0) &&
        h.total_tiles >= 0 && h.max_tiles >= 0 && h.rot_floats >= 0 &&
        h.rot_floats <= (int64_t)64 * h.Dp * h.Dp && (h.rot_ok == 0 || h.rot_ok == 1) &&
        h.rot_T >= 0 && h.rot_T <= 15 && h.rot_Lmax >= 0 && h.rot_Lmax < 16 &&
        h.sched >= ADSX_SCHED_AUTO && h.sched <= ADSX_SCHED_CLUSTER && h.cm_G >= 0 &&
        h.cm_G <= adsx::CM_MAX_G && h.cm_tpi >= 1 && h.cm_tpi <= 64 && h.tuned_delta_d >= 16 &&
        h.tuned_delta_d <= ADSX_MAX_D &&
        h.tuned_delta_d % 16 == 0 && h.items_per_sm >= 1 && h.items_per_sm <= 1024;
    bool rot_sane = sane;
    if (sane) {
        // the digit layout is a function of Dp alone
        int rb = 0, rT = 0, rL = 0;
        adsx::tc_rot_params((int)h.Dp, &rb, &rT, &rL);
        int64_t boff[16];
        if (h.rot_ok) {
            const int64_t total = rot_layout(h.Dp, h.rot_T, h.rot_Lmax, boff);
            rot_sane = h.has_P == 1 && rT > 0 && h.rot_b == rb && h.rot_T == rT && h.rot_Lmax == rL &&
                       h.rot_floats == total;
            for (int i = 0; i < 16 && rot_sane; ++i) rot_sane = h.rot_boff[i] == boff[i];
        } else {
            rot_sane = h.rot_floats == 0;
        }
    }
    if (!sane || !rot_sane) {
        fclose(f);
        return perr(ADSX_EINVAL, "%s: header fields out of range", path);
    }
    Index *ix = new Index();
    ix->N = h.N;
    ix->D = (int32_t)h.D;
    ix->Dp = (int32_t)h.Dp;
    ix->nlist = (int32_t)h.nlist;
    ix->storage = (int32_t)h.storage;
    ix->metric = (int32_t)h.metric;
    ix->kac_L = (int32_t)h.kac_L;
    ix->total_tiles = (int32_t)h.total_tiles;
    ix->max_tiles = (int32_t)h.max_tiles;
    ix->tuned_delta_d = (int32_t)h.tuned_delta_d;
    ix->items_per_sm = (int32_t)h.items_per_sm;
    ix->sched = (int32_t)h.sched;
    ix->cm_G = (int32_t)h.cm_G;
    ix->cm_tpi = (int32_t)h.cm_tpi;
    ix->rot_ok = h.rot_ok != 0;
    ix->rot_tc = false;
    ix->rot_b = (int32_t)h.rot_b;
    ix->rot_T = (int32_t)h.rot_T;
    ix->rot_Lmax = (int32_t)h.rot_Lmax;
    for (int i = 0; i < 16; ++i) ix->rot_boff[i] = h.rot_boff[i];
    cudaGetDevice(&ix->device);
    auto fail_free = [&](int code, const std::string &msg) {
        fclose(f);
        adsx_free_index(reinterpret_cast<adsx_index *>(ix));
        return perr(code, "%s", msg.c_str());
    };
    cudaError_t e = cudaMalloc((void **)&ix->err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ix->err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return fail_free(ADSX_ECUDA, std::string("alloc: ") + cudaGetErrorString(e));
    ix->bytes = sizeof(unsigned);
    Fnv fnv;
    fnv.add(&h, sizeof h);
    std::vector<unsigned char> buf;
    for (const Part &p : parts_of(ix, h)) {
        e = cudaMalloc(p.dev, p.bytes > 16 ? p.bytes : 16);
        if (e != cudaSuccess)
            return fail_free(e == cudaErrorMemoryAllocation ? ADSX_ENOMEM : ADSX_ECUDA,
                             std::string("alloc: ") + cudaGetErrorString(e));
        ix->bytes += (int64_t)p.bytes;
        for (size_t o = 0; o < p.bytes; o += CHUNK) {
            const size_t n = p.bytes - o < CHUNK ? p.bytes - o : CHUNK;
            buf.resize(n);
            if (fread(buf.data(), 1, n, f) != n)
                return fail_free(ADSX_EINVAL, std::string(path) + " is truncated");
            fnv.add(buf.data(), n);
            e = cudaMemcpy(static_cast<unsigned char *>(*p.dev) + o, buf.data(), n,
                           cudaMemcpyHostToDevice);
            if (e != cudaSuccess)
                return fail_free(ADSX_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
        }
    }
    uint64_t stored = 0;
    if (fread(&stored, sizeof stored, 1, f) != 1 || stored != fnv.h)
        return fail_free(ADSX_EINVAL, std::string(path) + ": checksum mismatch");
    fclose(f);
    const std::string bad = check_indexes(ix);
    if (!bad.empty()) {
        adsx_free_index(reinterpret_cast<adsx_index *>(ix));
        return perr(ADSX_EINVAL, "%s: %s", path, bad.c_str());
    }
    // the centroids' TF32 halves for the centroid GEMM, derived, not stored
    const size_t sw = (size_t)adsx::tf32_split_words(ix->nlist, ix->Dp);
    e = cudaMalloc((void **)&ix->cents_split, sizeof(uint32_t) * sw);
    if (e == cudaSuccess) {
        ix->bytes += (int64_t)(sizeof(uint32_t) * sw);
        e = adsx::launch_tf32_split(ix->cents, ix->nlist, ix->Dp, ix->Dp, ix->cents_split, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        adsx_free_index(reinterpret_cast<adsx_index *>(ix));
        return perr(e == cudaErrorMemoryAllocation ? ADSX_ENOMEM : ADSX_ECUDA, "split centroids: %s",
                    cudaGetErrorString(e));
    }
    (void)stream;
    *out = reinterpret_cast<adsx_index *>(ix);
    return ADSX_OK;
}
