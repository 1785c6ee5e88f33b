// select.cu -- top-nprobe cluster selection per query (Sec. 2.2.2: probe the
// N_probe clusters whose centroids are nearest to the query), ordered by
// (squared centroid distance, cluster id).
//
// One warp per query row, several per block, no block barriers.  When the
// centroid GEMM has written the tile summary (four smallest entries of every
// 128-column tile of the row, adsx_internal.cuh) and nprobe <= 64, the row
// is mostly not read at all: the nprobe-th smallest summary word bounds the
// nprobe-th smallest distance, a tile whose fourth word lies above the bound
// contributes exactly its summary words below it (their exact values read
// one by one), and only the other tiles are read whole (select_by_summary).
// Else, for nprobe <= 64, a bound-and-gather path over the whole row is
// taken (see the kernel); otherwise, or when ties overflow it, a radix
// select runs: the row's distances become order-preserving 32-bit keys (bit
// patterns of non-negative floats), re-read from the row (an L2 hit: the
// warp has just read it) on every pass, so a warp needs shared memory only
// for its winners and a histogram; the row's smallest and largest key give
// the high bits every key shares, and radix passes of up to 8 bits over the
// remaining bits (warp-aggregated shared-memory histograms) find the exact
// key T of the nprobe-th smallest distance and how many keys equal to T are
// needed (or stop early when a digit's bin is needed whole).  Keys below T
// and the needed keys equal to T (ascending cluster id) are gathered by
// ballot in index order, and the warp bitonic-sorts the nprobe winners as
// 64-bit (key, id) words.
#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int MAXW = 8;                 // warps per block (fewer for large nprobe)
constexpr unsigned FULL = 0xffffffffu;

// Bitonic sort of n (a power of two) entries of `v` by the warp.
template <typename K>
__device__ __forceinline__ void warp_sort(K *v, int n, int lane)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < n; i += 32) {
                const int j = i ^ stride;
                if (j > i) {
                    const K x = v[i], y = v[j];
                    if ((x > y) == ((i & size) == 0)) {
                        v[i] = y;
                        v[j] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// One warp's shared-memory region: winners (P2 x 8 bytes, at least the
// 128 of the bound-and-gather path) and a 256-bin histogram.
constexpr int FAST_CAP = 128;   // candidate capacity of the bound-and-gather path (nprobe <= 64)
__host__ __device__ inline size_t sel_bytes(int P2)
{
    return ((size_t)(P2 > FAST_CAP ? P2 : FAST_CAP) * 8 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t warp_region(int P2)
{
    return sel_bytes(P2) + 1024;
}

// The sorted (key, id) words sel[0 .. c) padded to a power of two, sorted,
// and the first nprobe written out.
__device__ __forceinline__ void emit_sorted(unsigned long long *sel, unsigned c, int nprobe,
                                            int lane, int32_t *prow, float *drow)
{
    int n2 = 32;
    while (n2 < (int)c) n2 <<= 1;
    for (int i = (int)c + lane; i < n2; i += 32) sel[i] = ~0ull;
    __syncwarp();
    warp_sort(sel, n2, lane);
    for (int p = lane; p < nprobe; p += 32) {
        const unsigned long long v = sel[p];
        prow[p] = (int32_t)(v & 0xffffffffu);
        if (drow) drow[p] = __uint_as_float((unsigned)(v >> 32));
    }
    __syncwarp();
}

// nprobe <= 64 from the tile summary `srow` (ntiles x 4 words of this row).
// Each lane keeps the four smallest words of its tiles; the nprobe-th
// smallest of those 128 words, pb, is at least the packed word of the
// nprobe-th smallest distance (a subset's order statistic), so with
// tb = pb & ~127 every distance among the nprobe smallest has a key
// <= Tb = tb | 127.  A tile whose fourth word has (word & ~127) > tb holds
// no other key <= Tb than those of its summary words with (word & ~127) <= tb,
// whose exact keys are read from the row; every other tile is read whole.
// Everything <= Tb is gathered and sorted by (key, id): the exact answer.
// Returns false (nothing written) when the summary holds fewer than nprobe
// entries or more than FAST_CAP keys reach the bound.
__device__ bool select_by_summary(const float *__restrict__ row, const unsigned *__restrict__ srow,
                                  int ntiles, int nlist, int nprobe, unsigned long long *sel,
                                  int lane, int32_t *prow, float *drow)
{
    const unsigned below = (1u << lane) - 1u;
    unsigned t0 = ~0u, t1 = ~0u, t2 = ~0u, t3 = ~0u;
    uint4 w0 = make_uint4(~0u, ~0u, ~0u, ~0u);      // this lane's first tile, kept for the gather
    for (int t = lane; t < ntiles; t += 32) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(srow) + t);
        if (t == lane) w0 = w;
        keep4(w.x, t0, t1, t2, t3);
        keep4(w.y, t0, t1, t2, t3);
        keep4(w.z, t0, t1, t2, t3);
        keep4(w.w, t0, t1, t2, t3);
    }
    // tb = (nprobe-th smallest of the 128 kept words) & ~127, bit by bit from
    // the top: bit b of tb is 0 iff at least nprobe words lie at or below
    // the prefix found so far with bit b clear and every lower bit set.
    unsigned tb = 0u;
    for (int b = 31; b >= 7; --b) {
        const unsigned x = tb | ((1u << b) - 1u);
        const unsigned n = (t0 <= x) + (t1 <= x) + (t2 <= x) + (t3 <= x);
        if (__reduce_add_sync(FULL, n) < (unsigned)nprobe) tb |= 1u << b;
    }
    if (tb == (~0u & ~SUMMARY_LOW)) return false;   // fewer than nprobe summary entries
    const unsigned Tb = tb | SUMMARY_LOW;
    unsigned c = 0;
    for (int g0 = 0; g0 < ntiles && c <= (unsigned)FAST_CAP; g0 += 32) {
        const int t = g0 + lane;
        uint4 w = w0;
        if (g0 > 0) w = t < ntiles ? __ldg(reinterpret_cast<const uint4 *>(srow) + t)
                                   : make_uint4(~0u, ~0u, ~0u, ~0u);
        const bool whole = t < ntiles && (w.w & ~SUMMARY_LOW) <= tb;
        const unsigned e4[4] = {w.x, w.y, w.z, w.w};
        // the exact values of the summary words below the bound, loaded together
        float xv[4];
        unsigned needm = 0u;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const bool need = !whole && (e4[e] & ~SUMMARY_LOW) <= tb;   // padding never passes
            needm |= (need ? 1u : 0u) << e;
            xv[e] = need ? __ldg(row + t * SUMMARY_TILE + (int)(e4[e] & SUMMARY_LOW)) : 0.f;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned k = dist_key(xv[e]);
            const bool take = ((needm >> e) & 1u) && k <= Tb;
            const unsigned bt = __ballot_sync(FULL, take);
            const unsigned at = c + __popc(bt & below);
            if (take && at < (unsigned)FAST_CAP)
                sel[at] = ((unsigned long long)k << 32) |
                          (unsigned)(t * SUMMARY_TILE + (int)(e4[e] & SUMMARY_LOW));
            c += __popc(bt);
        }
        // tiles that may hold more keys <= Tb than their summary shows, two
        // at a time
        unsigned wm = __ballot_sync(FULL, whole);
        while (wm) {
            const int ta = g0 + __ffs(wm) - 1;
            wm &= wm - 1u;
            int tz = -1;
            if (wm) {
                tz = g0 + __ffs(wm) - 1;
                wm &= wm - 1u;
            }
            constexpr int U = SUMMARY_TILE / 32;
            float x[2 * U];
#pragma unroll
            for (int u = 0; u < 2 * U; ++u) {
                const int tt = u < U ? ta : tz;
                const int col = tt * SUMMARY_TILE + (u % U) * 32 + lane;
                x[u] = (tt >= 0 && col < nlist) ? __ldg(row + col) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 2 * U; ++u) {
                const int tt = u < U ? ta : tz;
                const int col = tt * SUMMARY_TILE + (u % U) * 32 + lane;
                const unsigned k = dist_key(x[u]);
                const bool take = tt >= 0 && col < nlist && k <= Tb;
                const unsigned bt = __ballot_sync(FULL, take);
                const unsigned at = c + __popc(bt & below);
                if (take && at < (unsigned)FAST_CAP)
                    sel[at] = ((unsigned long long)k << 32) | (unsigned)col;
                c += __popc(bt);
            }
        }
    }
    if (c > (unsigned)FAST_CAP) {
        __syncwarp();
        return false;
    }
    emit_sorted(sel, c, nprobe, lane, prow, drow);
    return true;
}

__global__ void __launch_bounds__(MAXW * 32, 3) select_nprobe_kernel(
    const float *__restrict__ dist, int64_t nq, int nlist, int pstride, int P2, int W,
    int32_t *__restrict__ probes, float *__restrict__ pd2, const int32_t *__restrict__ nprobe_q,
    const unsigned *__restrict__ summary, int ntiles)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *base = smraw + warp_region(P2) * warp;
    unsigned long long *sel = reinterpret_cast<unsigned long long *>(base);
    unsigned *hist = reinterpret_cast<unsigned *>(base + sel_bytes(P2));
    const unsigned below = (1u << lane) - 1u;

    for (int64_t q = (int64_t)blockIdx.x * W + warp; q < nq; q += (int64_t)gridDim.x * W) {
        int nprobe = pstride;
        if (nprobe_q) {                     // per-query count, clamped to [1, pstride]
            nprobe = nprobe_q[q];
            nprobe = nprobe < 1 ? 1 : (nprobe > pstride ? pstride : nprobe);
        }
        const float *row = dist + q * nlist;
        if (summary && nprobe <= 64 &&
            select_by_summary(row, summary + (size_t)q * ntiles * 4, ntiles, nlist, nprobe, sel,
                              lane, probes + q * pstride, pd2 ? pd2 + q * pstride : nullptr))
            continue;
        unsigned kmin = 0xffffffffu, kmax = 0u;
        // nprobe <= 64: the nprobe-th smallest of the 128 lane-wise four
        // smallest keys bounds the nprobe-th smallest key from above (it is
        // the nprobe-th of a subset), so gathering every key up to it and
        // sorting those by (key, id) gives the exact answer.
        const bool fast = nprobe <= 64;
        unsigned t0 = 0xffffffffu, t1 = 0xffffffffu, t2 = 0xffffffffu, t3 = 0xffffffffu;
        if ((nlist & 3) == 0) {
            // 16-byte loads, eight in flight per lane before any use
            const float4 *r4 = reinterpret_cast<const float4 *>(row);
            const int n4 = nlist >> 2;
            for (int i0 = lane; i0 < n4; i0 += 32 * 8) {
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + 32 * u < n4) v[u] = __ldg(r4 + i0 + 32 * u);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 32 * u;
                    if (i < n4) {
                        const uint4 k4 = make_uint4(dist_key(v[u].x), dist_key(v[u].y),
                                                    dist_key(v[u].z), dist_key(v[u].w));
                        kmin = min(min(kmin, min(k4.x, k4.y)), min(k4.z, k4.w));
                        kmax = max(max(kmax, max(k4.x, k4.y)), max(k4.z, k4.w));
                        if (fast) {
                            keep4(k4.x, t0, t1, t2, t3);
                            keep4(k4.y, t0, t1, t2, t3);
                            keep4(k4.z, t0, t1, t2, t3);
                            keep4(k4.w, t0, t1, t2, t3);
                        }
                    }
                }
            }
        } else {
            for (int i0 = lane; i0 < nlist; i0 += 32 * 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + 32 * u < nlist) v[u] = __ldg(row + i0 + 32 * u);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 32 * u;
                    if (i < nlist) {
                        const unsigned k = dist_key(v[u]);
                        kmin = k < kmin ? k : kmin;
                        kmax = k > kmax ? k : kmax;
                        if (fast) keep4(k, t0, t1, t2, t3);
                    }
                }
            }
        }
        kmin = __reduce_min_sync(FULL, kmin);
        kmax = __reduce_max_sync(FULL, kmax);
        __syncwarp();
        if (fast) {
            hist[lane * 4 + 0] = t0;
            hist[lane * 4 + 1] = t1;
            hist[lane * 4 + 2] = t2;
            hist[lane * 4 + 3] = t3;
            __syncwarp();
            warp_sort(hist, 128, lane);
            const unsigned Tb = hist[nprobe - 1];
            // gather every key <= Tb (any order: sorted below), the row read
            // again 8 x 32 keys at a time
            unsigned c = 0;
            for (int i0 = 0; i0 < nlist && c <= (unsigned)FAST_CAP; i0 += 32 * 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 32 * u + lane;
                    v[u] = i < nlist ? __ldg(row + i) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 32 * u + lane;
                    const unsigned k = dist_key(v[u]);
                    const bool take = i < nlist && k <= Tb;
                    const unsigned bt = __ballot_sync(FULL, take);
                    const unsigned at = c + __popc(bt & below);
                    if (take && at < (unsigned)FAST_CAP)
                        sel[at] = ((unsigned long long)k << 32) | (unsigned)i;
                    c += __popc(bt);
                }
            }
            if (c <= (unsigned)FAST_CAP) {
                emit_sorted(sel, c, nprobe, lane, probes + q * pstride,
                            pd2 ? pd2 + q * pstride : nullptr);
                continue;
            }
            __syncwarp();                   // too many ties: the radix path below
        }

        // Radix select over the bits below the common prefix of all keys.
        unsigned prefix = kmin, rem = (unsigned)nprobe;
        int cut = -1;     // >= 0: every key whose bits above `cut` are <= prefix's is taken
        if (kmin != kmax) {
            const int hb = 31 - __clz(kmin ^ kmax);             // highest differing bit
            unsigned mask = hb == 31 ? 0u : ~((2u << hb) - 1u);  // bits already fixed
            prefix = kmin & mask;
            for (int top = hb; top >= 0; top -= 8) {
                const int shift = top >= 7 ? top - 7 : 0;
                const unsigned dmask = (2u << (top - shift)) - 1u;  // <= 8 bits
#pragma unroll
                for (int j = 0; j < 8; ++j) hist[lane * 8 + j] = 0u;
                __syncwarp();
                for (int i0 = 0; i0 < nlist; i0 += 32) {
                    const int i = i0 + lane;
                    unsigned bin = 256u;                        // no vote
                    if (i < nlist) {
                        const unsigned u = dist_key(__ldg(row + i));
                        if ((u & mask) == prefix) bin = (u >> shift) & dmask;
                    }
                    // lanes with the same digit merge into one atomic
                    const unsigned peers = __match_any_sync(FULL, bin);
                    if (bin < 256u && lane == __ffs(peers) - 1)
                        atomicAdd(&hist[bin], (unsigned)__popc(peers));
                }
                __syncwarp();
                // the bin holding the rem-th key: each lane owns 8 bins, a
                // shuffle scan gives the counts before them
                unsigned h[8], own = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    h[j] = hist[lane * 8 + j];
                    own += h[j];
                }
                unsigned incl = own;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                unsigned cum = incl - own, bin = 0, nrem = 0, cnt = 0;
                const bool found = cum < rem && incl >= rem;
                if (found) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (cum + h[j] >= rem) {
                            bin = (unsigned)(lane * 8 + j);
                            nrem = rem - cum;
                            cnt = h[j];
                            break;
                        }
                        cum += h[j];
                    }
                }
                const int src = __ffs(__ballot_sync(FULL, found)) - 1;
                bin = __shfl_sync(FULL, bin, src);
                rem = __shfl_sync(FULL, nrem, src);
                cnt = __shfl_sync(FULL, cnt, src);
                prefix |= bin << shift;
                mask |= dmask << shift;
                __syncwarp();
                if (shift == 0) break;
                if (cnt == rem) {       // the whole bin is needed: no further digits
                    cut = shift;
                    break;
                }
            }
        }
        const unsigned T = prefix;          // key of the nprobe-th smallest distance
        const unsigned need_eq = rem;       // keys equal to T still needed (>= 1)

        // Gather in index order: keys below T, and the first need_eq keys == T.
        unsigned nsel = 0, eq_seen = 0;
        for (int i0 = 0; i0 < nlist; i0 += 32) {
            const int i = i0 + lane;
            const unsigned u = i < nlist ? dist_key(__ldg(row + i)) : 0xffffffffu;
            const bool lt = i < nlist && (cut >= 0 ? (u >> cut) <= (T >> cut) : u < T);
            const bool eq = i < nlist && cut < 0 && u == T;
            const unsigned be = __ballot_sync(FULL, eq);
            const bool take = lt || (eq && eq_seen + __popc(be & below) < need_eq);
            const unsigned bt = __ballot_sync(FULL, take);
            if (take) sel[nsel + __popc(bt & below)] = ((unsigned long long)u << 32) | (unsigned)i;
            nsel += __popc(bt);
            eq_seen += __popc(be);
        }
        for (int i = (int)nsel + lane; i < P2; i += 32) sel[i] = ~0ull;
        __syncwarp();
        warp_sort(sel, P2, lane);
        for (int p = lane; p < nprobe; p += 32) {
            const unsigned long long v = sel[p];
            probes[q * pstride + p] = (int32_t)(v & 0xffffffffu);
            if (pd2) pd2[q * pstride + p] = __uint_as_float((unsigned)(v >> 32));
        }
        __syncwarp();                       // before the next row reuses the region
    }
}

}  // namespace

cudaError_t launch_select_nprobe(const float *dist, int64_t nq, int nlist, int nprobe,
                                 int32_t *probes, float *probe_d2, cudaStream_t s,
                                 const int32_t *nprobe_q, const unsigned *summary)
{
    if (nq <= 0) return cudaSuccess;
    int P2 = 1;
    while (P2 < nprobe) P2 <<= 1;
    const size_t per = warp_region(P2);
    int W = (int)((48u << 10) / per);
    W = W > MAXW ? MAXW : (W < 1 ? 1 : W);
    const size_t smem = per * W;
    cudaError_t e = cudaFuncSetAttribute(select_nprobe_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (nq + W - 1) / W;
    if (grid > 152 * 8) grid = 152 * 8;
    const int ntiles = (nlist + SUMMARY_TILE - 1) / SUMMARY_TILE;
    select_nprobe_kernel<<<(unsigned)grid, W * 32, smem, s>>>(dist, nq, nlist, nprobe, P2, W, probes,
                                                              probe_d2, nprobe_q, summary, ntiles);
    return cudaGetLastError();
}

}  // namespace adsx
