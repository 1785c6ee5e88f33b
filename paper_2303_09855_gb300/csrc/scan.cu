// scan.cu -- the IVF+ candidate scan: Algorithm 1 (ADSampling) as the DCO of
// every member of a query's probed clusters (Sec. 4), against the query's
// current K-th distance (Sec. 2.2.2).  The same kernel, instantiated with a
// fixed threshold per query and every cluster as a probe slot, is the linear
// scan of the verification protocol (Sec. 6.2.5): its decisions come from
// exactly the accumulation, test and recheck code of a search.
//
// ads_scan_kernel is persistent and warp-centric.  A work item is (query q,
// split s): the probe slots s, s+S, s+2S, ... of q, or with more splits than
// slots every js-th tile of one slot (S = 1 unless there are too few queries
// to fill the GPU).  Each warp claims items from a global
// counter and owns, in shared memory, the item's q', a pending ring and a
// candidate buffer; nothing is shared between warps, so no locks.
//   1. Members are visited cluster by cluster in probe order, 32 per tile.
//      Each 16-dim block of a member is split over NL lanes (4 for FP32, 2
//      for 16-bit storage; 16 bytes each), so one load instruction of the
//      warp reads whole blocks of 32/NL members -- a contiguous 512-byte run
//      of the dim-blocked layout -- and a shuffle transpose gives every lane
//      the complete partial distance of one member.
//   2. The squared test S_d > r^2 f(d) (Sec. 3.2) rejects.  While at least
//      DENSE_MIN members of a tile are live, the tile advances as a whole
//      (all live members sit at the same block: contiguous loads, broadcast
//      query reads); then a ballot compacts the survivors into the warp's
//      pending ring (next-block offset, block stride, blocks done, CSR row,
//      S).  Whenever 32 are pending they advance one delta_d step each (NL
//      lanes per candidate again, all loads issued before the arithmetic)
//      and are re-tested, so lanes stay busy after compaction.
//   3. Candidates reaching d = D with S_D <= r^2 are appended to the warp's
//      candidate buffer (capacity C = 2 * next_pow2(K)).  When it fills, or
//      first holds K entries, it is bitonic-sorted by (distance, id) and cut
//      to K; r^2 becomes the K-th distance (the KNN set's maximum, Sec. 2.2.2).
//      With S > 1, r^2 is also published per query with atomicMin and read
//      back at each tile, so every split prunes with the best known bound.
//   4. At the end the buffer is sorted: with S = 1 the warp writes the final
//      top-K; otherwise its list goes to a partial buffer that
//      finalize_topk_kernel merges per query.
// Every returned distance is exact (d = D); any r used is the K-th of a set
// of exact candidate distances, so it is never below the exact K-th distance
// of all candidates -- the bracket property the tests check.
#include <float.h>

#include "scan_common.cuh"

namespace adsx {
namespace {

using namespace scan;

constexpr int WARPS = 4;
constexpr int THREADS = WARPS * 32;
constexpr int RING = 128;                 // per-warp pending ring (power of 2)
// Live members that keep a tile stepping as a whole (measured on the
// SIFT-shaped benchmark: 16-20 best; 8 and 32 -- never dense -- about 8% slower).
#ifndef ADSX_DENSE_MIN
#define ADSX_DENSE_MIN 20
#endif
constexpr int DENSE_MIN = ADSX_DENSE_MIN;

__host__ __device__ inline int align4(int x) { return (x + 3) & ~3; }

// Per-warp shared-memory region, in 4-byte words.
struct WarpCarve {
    int qv, ed, ei, pof, pst, pb, pp, pS, words;
    __host__ __device__ WarpCarve(int Dp, int C)
    {
        int o = 0;
        qv = o; o = align4(o + Dp);
        ed = o; o = align4(o + C);
        ei = o; o = align4(o + C);
        pof = o; o += 2 * RING;             // 8-byte aligned (o is a multiple of 4)
        pst = o; o += RING;
        pb = o; o += RING;
        pp = o; o += RING;
        pS = o; o += RING;
        words = o;
    }
};

template <typename T, bool IP, bool FIXED>
struct Warp {
    const ScanArgs *a;
    float *qv;
    float *ed;
    int *ei;
    // pending ring: element offset of the candidate's next block, its block
    // stride (16 * cluster size), blocks done, CSR row, partial distance
    long long *pof;
    int *pst, *pb, *pp;
    float *pS;
    const float *ftab;         // test factors (shared memory)
    int lane;
    int64_t q;
    int K, C, S;               // this item's K, buffer capacity, splits of its query
    int head, cnt;             // pending ring (warp-uniform)
    int count;                 // candidate buffer fill (warp-uniform)
    float r2;                  // this warp's K-th key (warp-uniform; squared distance, or
                               // -<o,q> for inner products)
    float qn;                  // ||q|| (inner-product indexes)
    unsigned dims;             // per lane, dims sampled by this item
};

// Sorts the candidate buffer by (distance, id), keeps the first K and sets
// r^2 to the K-th distance once K are held.
template <typename T, bool IP, bool FIXED>
__device__ void compact(Warp<T, IP, FIXED> &w)
{
    const int C = w.C, K = w.K;
    for (int k = w.count + w.lane; k < C; k += 32) {
        w.ed[k] = INFINITY;
        w.ei[k] = 0x7fffffff;
    }
    __syncwarp();
    for (int size = 2; size <= C; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = w.lane; i < C; i += 32) {
                const int j = i ^ stride;
                if (j > i) {
                    const float di = w.ed[i], dj = w.ed[j];
                    const int ii = w.ei[i], ij = w.ei[j];
                    const bool up = (i & size) == 0;
                    if (pair_less(dj, ij, di, ii) == up) {
                        w.ed[i] = dj;
                        w.ei[i] = ij;
                        w.ed[j] = di;
                        w.ei[j] = ii;
                    }
                }
            }
            __syncwarp();
        }
    }
    if (w.count > K) w.count = K;
    if (w.count == K) {
        const float r2 = w.ed[K - 1];
        if (r2 < w.r2) {
            w.r2 = r2;
            if (w.S > 1 && w.lane == 0) atomicMin(w.a->r2g + w.q, key_to_ord(r2));
        }
    }
    __syncwarp();
}

template <typename T, bool IP, bool FIXED>
__device__ __forceinline__ float current_r2(const Warp<T, IP, FIXED> &w)
{
    float r2 = w.r2;
    if (!FIXED && w.S > 1) {
        const unsigned g = *((volatile const unsigned *)(w.a->r2g + w.q));
        if (g != 0xffffffffu) r2 = fminf(r2, ord_to_key(g));
    }
    return r2;
}

// 16-bit storage: exact FP32 distance of every lane with `need` (the
// shared recheck, with the query from the warp's shared memory).
template <typename T, bool IP, bool FIXED>
__device__ __forceinline__ float recheck_exact(const Warp<T, IP, FIXED> &w, bool need, int pos, float S)
{
    return scan::recheck_rows(w.a->rows32, w.a->Dp, w.qv, need, pos, S, w.lane);
}

// Fixed-threshold mode: the decision of candidate `pos` (CSR row) for the
// item's query, by original id.
template <typename T, bool IP, bool FIXED>
__device__ __forceinline__ void record_decision(const Warp<T, IP, FIXED> &w, int pos, int dec,
                                                int dims)
{
    const ScanArgs &a = *w.a;
    const int64_t o = w.q * a.N + a.ids[pos];
    a.decisions[o] = (uint8_t)dec;
    if (a.dec_dims) a.dec_dims[o] = dims;
}

// Appends the lanes with `surv` to the pending ring (lane order).
template <typename T, bool IP, bool FIXED>
__device__ __forceinline__ void enqueue(Warp<T, IP, FIXED> &w, bool surv, float S, int blk, int pos,
                                        long long off, int st)
{
    const unsigned sm = __ballot_sync(FULL, surv);
    if (surv) {
        const int idx = (w.head + w.cnt + __popc(sm & ((1u << w.lane) - 1u))) & (RING - 1);
        w.pof[idx] = off;
        w.pst[idx] = st;
        w.pb[idx] = blk;
        w.pp[idx] = pos;
        w.pS[idx] = S;
    }
    w.cnt += __popc(sm);
}

// After a candidate has `blk` blocks accumulated in S: the exact compare at
// d = D (Case 3), else the hypothesis test (Case 1 reject / Case 2 continue).
// `pos` is the candidate's CSR row, `off` the element offset of its block
// `blk` and `st` its block stride.  Returns whether the candidate continues;
// with `push` it is also queued.
template <typename T, bool IP, bool FIXED>
__device__ __forceinline__ bool after_step(Warp<T, IP, FIXED> &w, bool valid, float S, int blk, int pos,
                                           long long off, int st, float r2, bool push)
{
    const ScanArgs &a = *w.a;
    const bool fin = valid && blk >= a.nblk;
    // Squared threshold on the stored vectors: r^2 itself (L2, cosine), or
    // for inner products the per-object 2 - 2 r / (||o|| ||q||) on the
    // normalised vectors, r = -r2 the K-th largest inner product held
    // (Sec. 8, extension (1)); a negative threshold rejects at once.
    float thr = r2, onq = 0.f;
    if (IP && valid) {
        onq = a.onorm[pos] * w.qn;
        thr = 2.f + 2.f * r2 / onq;
    }
    bool surv = false;
    if (valid && !fin) {
        if (a.test_on && S > thr * w.ftab[blk]) {
            const int d = blk * BLK;
            w.dims += (unsigned)(d < a.D ? d : a.D);
            if constexpr (FIXED) record_decision(w, pos, 0, d < a.D ? d : a.D);
        } else {
            surv = true;
        }
    }
    if (fin) w.dims += (unsigned)a.D;
    if (push) enqueue(w, surv, S, blk, pos, off, st);
    bool cand = fin;
    if constexpr (Roundoff<T>::u > 0.f) {
        // S is a sum over rounded coordinates x~ with |x~ - x| <= u|x|, so
        // ||x~ - q|| <= ||x - q|| + u||x||: a candidate with S_D <= r^2 has
        // sqrt(S~) <= r + u||x||.  Only those are recomputed exactly in FP32;
        // the low precision moves reject decisions only, never a result.
        bool need = false;
        if (fin) {
            need = !(thr < INFINITY);
            if (!need && thr >= 0.f) {
                const float bound = (sqrtf(thr) + Roundoff<T>::u * a.norms[pos]) * 1.0001f;
                need = sqrtf(S) <= bound;
            }
        }
        S = recheck_exact(w, need, pos, S);
        cand = need;
    }
    if constexpr (FIXED) {
        // positive iff the (exact FP32) distance at d = D is <= r^2
        if (fin) record_decision(w, pos, (cand && S <= r2) ? 1 : 2, a.D);
        return surv;
    }
    // Case 3 positives into the candidate buffer; the key is the squared
    // distance, or -<o,q> = -||o|| ||q|| (1 - S/2) for inner products.
    const float key = IP ? -(onq * fmaf(-0.5f, S, 1.f)) : S;
    const bool want = cand && key <= r2;
    const unsigned wm = __ballot_sync(FULL, want);
    if (wm) {
        const int nw = __popc(wm);
        if (w.count + nw > w.C) compact(w);
        if (want) {
            const int k = w.count + __popc(wm & ((1u << w.lane) - 1u));
            w.ed[k] = key;
            w.ei[k] = a.ids[pos];
        }
        w.count += nw;
        __syncwarp();
        if (w.count >= w.K && w.r2 == INFINITY) compact(w);
    }
    __syncwarp();
    return surv;
}

// One step of a dense tile: blocks [b0, b1) of the live members among
// m0 .. m0+31 of a cluster laid out from `cb` (block stride n*16); member
// m0 + g + (32/NL) k is loaded iff bit owner_lane(g, k) of `live` is set.
// Returns, on lane l, the step's partial distance of member m0 + own_slot(l)
// (meaningless if that member is dead: its loads are skipped, its sum unused).
template <typename T>
__device__ __forceinline__ float tile_step(const T *cb, int64_t stride, int m0, int b0, int b1,
                                           unsigned live, const float *qv, int lane)
{
    constexpr int NL = Split<T>::NL, NG = 32 / NL, PW = BLK / NL;
    typedef typename Split<T>::V V;
    const int g = lane / NL, jo = (lane % NL) * PW;
    const T *x = cb + (int64_t)b0 * stride + (int64_t)(m0 + g) * BLK + jo;
    bool ok[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) ok[k] = (live >> owner_lane<NL>(g, k)) & 1u;
    float2 p[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) p[k] = make_float2(0.f, 0.f);
    int b = b0;
    for (; b + 2 <= b1; b += 2, x += 2 * stride) {
        V v[2 * NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            zero_piece(v[k]);
            zero_piece(v[NL + k]);
            if (ok[k]) {
                v[k] = ld_piece(x + k * NG * BLK);
                v[NL + k] = ld_piece(x + stride + k * NG * BLK);
            }
        }
        const QPiece<NL> q0 = ld_qpiece<NL>(qv + b * BLK + jo);
        const QPiece<NL> q1 = ld_qpiece<NL>(qv + (b + 1) * BLK + jo);
#pragma unroll
        for (int k = 0; k < NL; ++k)
            p[k] = add_piece(v[NL + k], q1, add_piece(v[k], q0, p[k], T()), T());
    }
    if (b < b1) {
        V v[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            zero_piece(v[k]);
            if (ok[k]) v[k] = ld_piece(x + k * NG * BLK);
        }
        const QPiece<NL> q0 = ld_qpiece<NL>(qv + b * BLK + jo);
#pragma unroll
        for (int k = 0; k < NL; ++k) p[k] = add_piece(v[k], q0, p[k], T());
    }
    return group_sum<NL>(p, lane);
}

// Advances the first nb (<= 32) pending candidates by one delta_d step each,
// NL lanes per candidate, then tests them (after_step) one per lane.
template <typename T, bool IP, bool FIXED>
__device__ __forceinline__ void process_pending(Warp<T, IP, FIXED> &w, int nb)
{
    constexpr int NL = Split<T>::NL, NG = 32 / NL, PW = BLK / NL;
    typedef typename Split<T>::V V;
    const ScanArgs &a = *w.a;
    const int g = w.lane / NL, jo = (w.lane % NL) * PW, mine = own_slot<NL>(w.lane);
    const T *data = static_cast<const T *>(a.data) + jo;
    const T *x[NL];
    int st[NL], bk[NL], kb[NL];
    long long off_own = 0;
    int st_own = 0, e_own = 0, kmax = 0;
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        const int t = g + NG * k;
        long long off = 0;
        int s = 0, blk = 0, e = 0;
        if (t < nb) {
            const int idx = (w.head + t) & (RING - 1);
            off = w.pof[idx];
            s = w.pst[idx];
            blk = w.pb[idx];
            e = blk + a.db < a.nblk ? blk + a.db : a.nblk;
        }
        x[k] = data + off;
        st[k] = s;
        bk[k] = blk;
        kb[k] = e - blk;
        kmax = kb[k] > kmax ? kb[k] : kmax;
        if (t == mine) {
            off_own = off + (long long)(e - blk) * s;
            st_own = s;
            e_own = e;
        }
    }
    const bool valid = mine < nb;
    float S = 0.f;
    int pos = 0;
    if (valid) {
        const int idx = (w.head + mine) & (RING - 1);
        S = w.pS[idx];
        pos = w.pp[idx];
    }
    __syncwarp();
    w.head = (w.head + nb) & (RING - 1);
    w.cnt -= nb;
    const float r2 = current_r2(w);
    float2 p[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) p[k] = make_float2(0.f, 0.f);
    for (int s = 0; s < kmax; s += 2) {
        V v[2 * NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            zero_piece(v[k]);
            zero_piece(v[NL + k]);
            if (s < kb[k]) v[k] = ld_piece(x[k]);
            if (s + 1 < kb[k]) v[NL + k] = ld_piece(x[k] + st[k]);
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            if (s < kb[k])
                p[k] = add_piece(v[k], ld_qpiece<NL>(w.qv + (bk[k] + s) * BLK + jo), p[k], T());
            if (s + 1 < kb[k])
                p[k] = add_piece(v[NL + k], ld_qpiece<NL>(w.qv + (bk[k] + s + 1) * BLK + jo), p[k],
                                 T());
            x[k] += 2 * st[k];
        }
    }
    S += group_sum<NL>(p, w.lane);
    after_step(w, valid, S, e_own, pos, off_own, st_own, r2, true);
}

// Resident blocks per SM the register budget is sized for (FP32 storage;
// 16-bit storage).  Measured on the SIFT-shaped 1M x 128 benchmark (FP32) and
// the GIST-shaped 1M x 960 one (16-bit): 5 beats 4 and 6 for both.
#ifndef ADSX_SCAN_MINBLOCKS
#define ADSX_SCAN_MINBLOCKS 5
#endif
#ifndef ADSX_SCAN_MINBLOCKS_H
#define ADSX_SCAN_MINBLOCKS_H 5
#endif
template <typename T> struct MinBlocks { static constexpr int value = ADSX_SCAN_MINBLOCKS_H; };
template <> struct MinBlocks<float> { static constexpr int value = ADSX_SCAN_MINBLOCKS; };

template <typename T, bool IP, bool FIXED>
__global__ void __launch_bounds__(THREADS, MinBlocks<T>::value) ads_scan_kernel(ScanArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WarpCarve wc(a.Dp, a.C);
    float *base = reinterpret_cast<float *>(smraw) + (size_t)warp * wc.words;
    __shared__ float s_ftab[256];
    for (int b = threadIdx.x; b <= a.nblk && b < 256; b += THREADS) s_ftab[b] = a.ftab[b];
    __syncthreads();
    Warp<T, IP, FIXED> w;
    w.a = &a;
    w.ftab = s_ftab;
    w.qv = base + wc.qv;
    w.ed = base + wc.ed;
    w.ei = reinterpret_cast<int *>(base + wc.ei);
    w.pof = reinterpret_cast<long long *>(base + wc.pof);
    w.pst = reinterpret_cast<int *>(base + wc.pst);
    w.pb = reinterpret_cast<int *>(base + wc.pb);
    w.pp = reinterpret_cast<int *>(base + wc.pp);
    w.pS = base + wc.pS;
    w.lane = lane;
    const int n_items = a.n_items_dev ? *a.n_items_dev : a.n_items;

    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(a.work_counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_items) break;
        int64_t q;
        int s, S;
        if (a.items) {                       // batched: planned (query, split, splits)
            const int2 it = a.items[item];
            q = it.x;
            s = it.y >> 16;
            S = it.y & 0xffff;
        } else {
            q = item / a.S;
            s = item - (int)q * a.S;
            S = a.S;
        }
        const int K = a.Kq ? a.Kq[q] : a.K;
        const int nprobe = a.nprobe_q ? a.nprobe_q[q] : a.nprobe;
        int C = 1;
        {
            int Kp = 1;
            while (Kp < K) Kp <<= 1;
            const int need = 2 * Kp > K + 32 ? 2 * Kp : K + 32;
            while (C < need) C <<= 1;
        }
        w.q = q;
        w.K = K;
        w.C = C;
        w.S = S;
        for (int i = lane; i < a.Dp; i += 32) w.qv[i] = a.qrot[q * a.Dp + i];
        w.head = w.cnt = 0;
        w.count = 0;
        w.r2 = FIXED ? a.r2fixed[q] : INFINITY;
        w.qn = IP ? a.qnorm[q] : 1.f;
        w.dims = 0u;
        __syncwarp();

        // With S <= nprobe, split s owns the probe slots s, s + S, ... (the
        // split holding the nearest cluster finds a tight r early and shares
        // it).  With S > nprobe (e.g. nlist = 1, a linear scan), split s works
        // on slot s % nprobe alone, taking every js-th 32-member tile of it
        // from tile s / nprobe, js being the number of splits on that slot.
        // (Two inlined copies: the common one has constant tile steps.)
        const int pstride = a.probe_stride ? a.probe_stride : a.nprobe;
        auto scan_slot = [&](int p, int j0, int js) {
            const int c = FIXED ? p : a.probes[q * pstride + p];
            const int o = (int)a.off[c];
            const int n = (int)(a.off[c + 1] - o);
            const T *cb = static_cast<const T *>(a.data) + (int64_t)o * a.Dp;
            const int64_t stride = (int64_t)n * BLK;
            const long long cbase = (long long)o * a.Dp;
            for (int m0 = j0 * 32; m0 < n; m0 += 32 * js) {
                // The tile advances step by step while at least DENSE_MIN of
                // its members are live (all at the same block, contiguous
                // loads); the rest go to the pending ring.
                const int m = m0 + own_slot<Split<T>::NL>(lane);
                bool live = m < n;
                unsigned lm = __ballot_sync(FULL, live);
                float Sd = 0.f;
                int blk = 0;
                for (;;) {
                    const float r2 = current_r2(w);
                    const int e = blk + a.db < a.nblk ? blk + a.db : a.nblk;
                    Sd += tile_step(cb, stride, m0, blk, e, lm, w.qv, lane);
                    blk = e;
                    const long long off = cbase + blk * stride + (long long)m * BLK;
                    live = after_step(w, live, Sd, blk, o + m, off, (int)stride, r2, false);
                    lm = __ballot_sync(FULL, live);
                    if (lm == 0u) break;
                    if (__popc(lm) < DENSE_MIN) {
                        enqueue(w, live, Sd, blk, o + m, off, (int)stride);
                        break;
                    }
                }
                while (w.cnt >= 32) process_pending(w, 32);
            }
        };
        if (S <= nprobe) {
            for (int p = s; p < nprobe; p += S) scan_slot(p, 0, 1);
        } else {
            const int p0 = s % nprobe;
            scan_slot(p0, s / nprobe, (S - 1 - p0) / nprobe + 1);
        }
        while (w.cnt > 0) process_pending(w, w.cnt < 32 ? w.cnt : 32);
        if constexpr (FIXED) continue;       // decisions only, no KNN set
        compact(w);

        unsigned long long wd = w.dims;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) wd += __shfl_xor_sync(FULL, wd, off);
        if (S == 1) {
            const int64_t ob = a.out_off ? a.out_off[q] : q * (int64_t)K;
            if (a.out_off && (ob < 0 || ob + K > a.out_total)) {
                if (lane == 0) atomicOr(a.err, ERR_OUT_RANGE);
                continue;
            }
            for (int k = lane; k < K; k += 32) {
                const bool has = k < w.count;
                a.out_ids[ob + k] = has ? (int64_t)w.ei[k] : (int64_t)-1;
                a.out_d2[ob + k] = out_value(a.metric, has ? w.ed[k] : 0.f, has);
            }
            if (lane == 0 && a.out_dims) a.out_dims[q] = (int64_t)wd;
        } else {
            const int64_t pbase = (int64_t)item * (a.Kmax ? a.Kmax : a.K);
            for (int k = lane; k < K; k += 32) {
                a.part_d[pbase + k] = k < w.count ? w.ed[k] : INFINITY;
                a.part_i[pbase + k] = k < w.count ? w.ei[k] : 0x7fffffff;
            }
            if (lane == 0 && a.out_dims) atomicAdd((unsigned long long *)(a.out_dims + q), wd);
        }
        __syncwarp();
    }
}

// Merges the S_q sorted partial lists of each split query into its final
// top-K (queries with one item were written by the scan itself).
__global__ void __launch_bounds__(256) finalize_topk_kernel(ScanArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Tmax = a.finalize_T;
    float *sd = reinterpret_cast<float *>(smraw);
    int *si = reinterpret_cast<int *>(sd + Tmax);
    for (int64_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        int64_t first;
        int S;
        if (a.items) {
            first = a.item_first[q];
            S = a.items[first].y & 0xffff;
        } else {
            first = q * a.S;
            S = a.S;
        }
        if (S <= 1) continue;                 // uniform per block
        const int K = a.Kq ? a.Kq[q] : a.K;
        int T = 1;
        while (T < S * K) T <<= 1;
        for (int i = threadIdx.x; i < T; i += blockDim.x) {
            const int s = i / K, k = i - s * K;
            const bool in = s < S;
            const int64_t src = (first + s) * (int64_t)(a.Kmax ? a.Kmax : a.K) + k;
            sd[i] = in ? a.part_d[src] : INFINITY;
            si[i] = in ? a.part_i[src] : 0x7fffffff;
        }
        __syncthreads();
        for (int size = 2; size <= T; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < T; i += blockDim.x) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const float di = sd[i], dj = sd[j];
                        const int ii = si[i], ij = si[j];
                        const bool up = (i & size) == 0;
                        if (pair_less(dj, ij, di, ii) == up) {
                            sd[i] = dj;
                            si[i] = ij;
                            sd[j] = di;
                            si[j] = ii;
                        }
                    }
                }
                __syncthreads();
            }
        }
        const int64_t ob = a.out_off ? a.out_off[q] : q * (int64_t)K;
        if (a.out_off && (ob < 0 || ob + K > a.out_total)) {
            if (threadIdx.x == 0) atomicOr(a.err, ERR_OUT_RANGE);
            __syncthreads();
            continue;
        }
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const bool has = sd[k] != INFINITY || si[k] != 0x7fffffff;
            a.out_ids[ob + k] = has ? (int64_t)si[k] : (int64_t)-1;
            a.out_d2[ob + k] = out_value(a.metric, sd[k], has);
        }
        __syncthreads();
    }
}

// f(d) per step: ADSampling's (d/D)(1+eps0/sqrt d)^2 (Sec. 3.2), or 1 for
// PDScanning (reject as soon as the partial distance exceeds r, Sec. 6.1).
__global__ void test_factor_kernel(float *ftab, int nblk, int D, float eps0, int pd)
{
    for (int b = threadIdx.x; b <= nblk; b += blockDim.x)
        ftab[b] = (b == 0) ? 0.f : (pd ? 1.f : test_factor(b, D, eps0));
}

}  // namespace

size_t scan_smem_bytes(const ScanArgs &a)
{
    return (size_t)WarpCarve(a.Dp, a.C).words * 4 * WARPS;
}

int scan_items_target(int device, int items_per_sm)
{
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    return nsm * items_per_sm;   // default 48: about one item per resident warp slot
}

// The instantiation a launch runs: storage type, inner-product thresholds,
// fixed-threshold mode (L2 / cosine only).
typedef void (*ScanKernel)(ScanArgs);
template <typename T>
static ScanKernel scan_kernel_for(const ScanArgs &a)
{
    if (a.decisions) return ads_scan_kernel<T, false, true>;
    return a.metric == ADSX_IP ? ads_scan_kernel<T, true, false> : ads_scan_kernel<T, false, false>;
}
static ScanKernel scan_kernel_for_args(const ScanArgs &a)
{
    if (a.storage == ADSX_F32) return scan_kernel_for<float>(a);
    if (a.storage == ADSX_BF16) return scan_kernel_for<__nv_bfloat16>(a);
    return scan_kernel_for<__half>(a);
}

int ads_scan_grid(const ScanArgs &a, int device)
{
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    size_t smem = scan_smem_bytes(a);
    const ScanKernel k = scan_kernel_for_args(a);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, THREADS, smem);
    if (per < 1) per = 1;
    int64_t g = (int64_t)nsm * per;
    const int64_t need = ((int64_t)a.n_items + WARPS - 1) / WARPS;
    if (g > need) g = need;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_test_factors(float *ftab, int nblk, int D, float eps0, cudaStream_t s, int pd)
{
    test_factor_kernel<<<1, 256, 0, s>>>(ftab, nblk, D, eps0, pd);
    return cudaGetLastError();
}

cudaError_t launch_ads_scan(const ScanArgs &a, int grid, cudaStream_t s)
{
    if (a.n_items <= 0) return cudaSuccess;
    size_t smem = scan_smem_bytes(a);
    const ScanKernel k = scan_kernel_for_args(a);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize_topk(const ScanArgs &a, cudaStream_t s)
{
    if (a.nq <= 0 || (!a.items && a.S <= 1)) return cudaSuccess;
    // a split query has S_q * next_pow2(K_q) <= 16384 entries (the planner's cap)
    int Tmax = 1;
    while (Tmax < (a.items ? 16384 : a.S * a.K)) Tmax <<= 1;
    ScanArgs b = a;
    b.finalize_T = Tmax;
    size_t smem = (size_t)Tmax * 8;
    cudaError_t e = cudaFuncSetAttribute(finalize_topk_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = a.nq < 152 * 8 ? a.nq : 152 * 8;
    finalize_topk_kernel<<<(unsigned)grid, 256, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace adsx
