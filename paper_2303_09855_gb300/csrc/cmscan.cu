// cmscan.cu -- the cluster-major schedule of the IVF+ candidate scan (Sec. 4
// with Algorithm 1 DCOs), for large query batches.
//
// The query-major scan (scan.cu) gives each warp one query and reads every
// probed cluster once per query that probes it.  On a large batch each
// cluster is probed by many queries (about nq * nprobe / nlist), so here the
// work is grouped by cluster instead: a work item is (cluster c, up to G of
// the queries that probe c), and one warp loads each Delta_d step of a
// 32-member tile of c ONCE into registers and tests it against all of its
// queries.  One load instruction of the warp then feeds G queries' FMAs.
//
// The running threshold r of a query cannot be shared between the warps
// that serve it without a global KNN set, so the probe ranks are processed
// in rounds: round 0 scans each query's nearest R0 clusters in full (no r is
// known yet, so the test is off) and gives every query its K-th distance r
// among them; each following round scans a range of probe ranks against the
// r of the rounds before it, appending every candidate that reaches d = D
// with S_D <= r^2 to a per-query list; cm_merge_kernel then merges the list
// into the query's top-K and tightens r.  A fixed r per round is a
// valid threshold (the K-th of a subset of exact candidate distances is
// never below the exact K-th of all of them), so every returned distance is
// exact and the bracket property of the query-major scan holds; and as r is
// fixed within a round, the result does not depend on the schedule.
//
// Every partial distance is accumulated with the shared per-candidate code
// of scan_common.cuh, in the same order as the query-major kernel, so both
// schedules compute the same FP32 value of S_d for every (query, candidate,
// step); with a fixed threshold (the verification protocol of Sec. 6.2.5)
// their decisions are identical.
//
// Within an item, each tile's first step is dense (one load of the step's
// blocks feeds every query of the item); each later step is loaded once,
// staged in shared memory, and only the (query, member) pairs still live are
// computed, one per lane, so that candidates ADSampling has rejected cost
// nothing more.
//
// A query whose list overflows its capacity in some round is flagged and,
// after the last round, searched again by the query-major kernel.
#include <float.h>

#include "scan_common.cuh"

namespace adsx {
namespace {

using namespace scan;

constexpr int CM_WARPS = 4;
// Percentage of live (slot, member) pairs of a tile from which a step is
// computed densely rather than pair by pair.
#ifndef ADSX_CM_DENSE_PCT
#define ADSX_CM_DENSE_PCT 35
#endif
constexpr int CM_DENSE_PCT = ADSX_CM_DENSE_PCT;
constexpr int CM_THREADS = CM_WARPS * 32;
// Resident blocks per SM the register allocation is bounded for (4 warps
// each).  The scan is latency-bound, so occupancy pays for a few spilled
// registers: measured on the SIFT-shaped 1M x 128 benchmark (10k queries,
// nprobe 64, K 100), scan kernel ms per search for 4 / 5 / 6 / 7 / 8 blocks:
// FP32 4.56 / 4.05 / 3.75 / 4.05 / 5.29 (118 / 96 / 80 / 72 / 64 registers),
// BF16 storage 5.60 (at 5) / 5.18 / 4.96 / 5.25 (6 / 7 / 8); with the live
// state in registers, FP32 at 6: 3.72 (FDScanning 4.04), BF16 at 7: 5.24.
#ifndef ADSX_CM_MINBLOCKS
#define ADSX_CM_MINBLOCKS 6
#endif
#ifndef ADSX_CM_MINBLOCKS_H
#define ADSX_CM_MINBLOCKS_H 7
#endif
template <typename T> struct CmMinBlocks { static constexpr int value = ADSX_CM_MINBLOCKS_H; };
template <> struct CmMinBlocks<float> { static constexpr int value = ADSX_CM_MINBLOCKS; };

// Member-block row of the staged tile step in shared memory: the 16 dims of
// one member as NL 16-byte pieces (FP32: 4, 16-bit: 2), piece j stored in
// column j ^ swz(member).  A 128-bit shared load serves eight lanes at a
// time; the eight members a pass gives eight consecutive lanes of one slot
// are own_slot(l) for eight consecutive l -- members 0, 16, 8, 24, 1, 17, 9,
// 25 and so on (FP32), 0, 16, 1, 17, ... (16-bit) -- whose unswizzled pieces
// would share banks; the swizzle spreads them over all 32 banks.
template <typename T> struct Stage {
    static constexpr int ROW = 32;               // bytes per member-block row
    __device__ static int swz(int m) { return (m >> 4) & 1; }
};
template <> struct Stage<float> {
    static constexpr int ROW = 64;
    __device__ static int swz(int m) { return (m >> 3) & 3; }
};

// Per-warp shared memory: query slots and their thresholds; the slots' live
// masks while a sparse step runs; per (slot, tile lane) the partial distance
// S_d; the live (slot, lane) pairs of a sparse step; and the tile's current
// step, staged member by member.
struct CmCarve {
    int qg, r2, live, S, pa, stile, bytes;
    __host__ __device__ CmCarve(int G, int db, int row)
    {
        int o = 0;
        qg = o; o += 4 * G;
        r2 = o; o += 4 * G;
        live = o; o += 4 * G;
        S = o; o += 4 * 32 * G;
        pa = o; o += 2 * 32 * G;
        o = (o + 15) & ~15;
        // the staged tile step of a sparse pass, or (dense steps) the step's
        // dims of every slot's query
        stile = o;
        o += db * 32 * row > G * db * 16 * 4 ? db * 32 * row : G * db * 16 * 4;
        bytes = (o + 15) & ~15;
    }
};

__device__ __forceinline__ float4 ldg4(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}
template <int NL>
__device__ __forceinline__ QPiece<NL> ld_qpiece_ro(const float *q)
{
    QPiece<NL> r;
    r.a = ldg4(q);
    if constexpr (NL == 2) r.b = ldg4(q + 4);
    return r;
}

// One member's step sum computed by one lane, in the order the NL-lane
// layout produces it: a chain pair (even, odd dims) per piece over the step's
// blocks, each pair summed, then the pieces combined as group_sum does --
// (P0 + P1) + (P2 + P3) for FP32, P0 + P1 for 16-bit storage -- which IEEE
// addition, being commutative, makes the same value on every lane.
//   row: the member's block rows in the staged tile (stride 32 rows per
//   block); mt: the member within the tile; q: the query's dims of the
//   step's first block.
template <typename T, int DB>
__device__ __forceinline__ float member_step_sum(const unsigned char *row, int mt, const float *q,
                                                 int nb)
{
    constexpr int NL = Split<T>::NL, PW = BLK / NL;
    constexpr int RB = 32 * Stage<T>::ROW;       // bytes between a member's block rows
    float2 p[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) p[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < DB; ++b) {
        if (b < nb) {
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const typename Split<T>::V v = *reinterpret_cast<const typename Split<T>::V *>(
                    row + b * RB + ((j ^ Stage<T>::swz(mt)) * 16));
                p[j] = add_piece(v, ld_qpiece_ro<NL>(q + b * BLK + j * PW), p[j], T());
            }
        }
    }
    if constexpr (NL == 4)
        return ((p[0].x + p[0].y) + (p[1].x + p[1].y)) + ((p[2].x + p[2].y) + (p[3].x + p[3].y));
    else
        return (p[0].x + p[0].y) + (p[1].x + p[1].y);
}

// One warp per item.  Each 32-member tile takes its first step densely: the
// step's blocks are loaded once into registers in the NL-lane layout of the
// query-major scan, and every query slot of the item computes its partial
// distances from them (two slots at a time: their FMA chains and shuffles
// interleave).  With the test off (FDScanning) every member stays live and
// the later steps run the same way.  With the test on, each later step of
// the tile is staged once in shared memory and only the live (slot, member)
// pairs are computed, one pair per lane, 32 pairs per pass whatever their
// query: the pairs that ADSampling has rejected cost nothing more.
template <typename T, int DB, bool FIXED>
__global__ void __launch_bounds__(CM_THREADS, CmMinBlocks<T>::value) cm_scan_kernel(CmArgs a)
{
    constexpr int NL = Split<T>::NL, NG = 32 / NL, PW = BLK / NL;
    constexpr int ROW = Stage<T>::ROW, RB = 32 * ROW;
    typedef typename Split<T>::V V;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float s_ftab[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const CmCarve cc(a.G, a.db, ROW);
    unsigned char *base = smraw + (size_t)warp * cc.bytes;
    int *qg = reinterpret_cast<int *>(base + cc.qg);
    float *r2g = reinterpret_cast<float *>(base + cc.r2);
    unsigned *live = reinterpret_cast<unsigned *>(base + cc.live);
    float *Sv = reinterpret_cast<float *>(base + cc.S);
    unsigned short *pa = reinterpret_cast<unsigned short *>(base + cc.pa);
    unsigned char *stile = base + cc.stile;
    for (int b = threadIdx.x; b <= a.nblk && b < 256; b += CM_THREADS) s_ftab[b] = a.ftab[b];
    __syncthreads();

    const int gi = lane / NL, jo = (lane % NL) * PW;
    const int own = own_slot<NL>(lane);
    const int n_items = *a.n_items;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(a.work_counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_items) break;
        const int2 it = a.items[item];
        const int c = it.x;
        const int64_t o = a.off[c];
        const int n = (int)(a.off[c + 1] - o);
        // item = (query group, chunk of tpi tiles) of cluster c
        const int tiles = (n + 31) >> 5, chunks = (tiles + a.tpi - 1) / a.tpi;
        const int qgi = it.y / chunks, tc = it.y - qgi * chunks;
        const int q0 = a.coff[c] + qgi * a.G;
        const int ngq = a.coff[c + 1] - q0 < a.G ? a.coff[c + 1] - q0 : a.G;
        const int mb = tc * a.tpi * 32;
        const int me = mb + a.tpi * 32 < n ? mb + a.tpi * 32 : n;
        for (int g = lane; g < ngq; g += 32) {
            const int q = a.qlist[q0 + g];
            qg[g] = q;
            r2g[g] = FIXED ? a.r2fixed[q] : a.r2[q];
        }
        __syncwarp();
        // dims sampled in this item by slots lane and lane + 32
        unsigned dga = 0u, dgb = 0u;
        const unsigned long long slots = ngq >= 64 ? ~0ull : (1ull << ngq) - 1ull;
        const T *cb = static_cast<const T *>(a.data) + o * a.Dp;
        const int64_t stride = (int64_t)n * BLK;
        for (int m0 = mb; m0 < me; m0 += 32) {
            // The tile's live state, in registers: la / lb are the live
            // members of slots lane and lane + 32 (bit l: member
            // own_slot(l)); am holds the slots for which this lane's own
            // member is live.
            const bool mine = m0 + own < n;
            const unsigned vm = __ballot_sync(FULL, mine);
            unsigned la = lane < ngq ? vm : 0u, lb = lane + 32 < ngq ? vm : 0u;
            unsigned long long am = mine ? slots : 0ull;
            int blk = 0;
            for (;;) {
                const unsigned U = __ballot_sync(FULL, am != 0ull);   // members live for some slot
                if (U == 0u) break;
                const int L = (int)__reduce_add_sync(FULL, (unsigned)(__popc(la) + __popc(lb)));
                // bit g: slot g has a live member
                const unsigned long long sl =
                    ((unsigned long long)__ballot_sync(FULL, lb != 0u) << 32) |
                    __ballot_sync(FULL, la != 0u);
                const int e = blk + a.db < a.nblk ? blk + a.db : a.nblk;
                const int nb = e - blk;
                const bool fin = e >= a.nblk;
                const float fe = s_ftab[e];
                const unsigned dstep = (unsigned)(e * BLK < a.D ? e * BLK : a.D);
                // Every pair live when the step starts samples its width: a
                // pair stopped at d_j has sampled the widths of steps 1..j.
                const unsigned width = dstep - (unsigned)(blk * BLK);
                dga += (unsigned)__popc(la) * width;
                dgb += (unsigned)__popc(lb) * width;
                // A step is dense -- every slot against every member, the
                // step's blocks loaded once into registers -- while enough
                // pairs are live (always the first step, and every step with
                // the test off); else only the live pairs are computed, one
                // per lane, from the step staged in shared memory.
                const bool dense = blk == 0 || !a.test_on || 100 * L >= CM_DENSE_PCT * 32 * ngq;
                const T *x = cb + (int64_t)blk * stride + (int64_t)(m0 + gi) * BLK + jo;
                if (dense) {
                    // this step's blocks of the tile: loaded once for every query
                    // (16-bit storage: converted to FP32 once, not per query)
                    typename Unpacked<T>::U v[DB][NL];
#pragma unroll
                    for (int b = 0; b < DB; ++b) {
#pragma unroll
                        for (int k = 0; k < NL; ++k) {
                            V w;
                            zero_piece(w);
                            if (b < nb && ((U >> owner_lane<NL>(gi, k)) & 1u))
                                w = ld_piece(x + b * stride + k * NG * BLK);
                            v[b][k] = unpack_piece(w, T());
                        }
                    }
                    // this step's dims of every slot's query, staged in the
                    // (idle) tile buffer: the slot loop reads them from shared
                    // memory (the same values, so the same sums)
                    constexpr int QW = DB * BLK;
                    float *qs = reinterpret_cast<float *>(stile);
                    {
                        const int per = nb * (BLK / 4);             // float4 per slot
                        for (int i = lane; i < ngq * per; i += 32) {
                            const int g = i / per, c = i - g * per;
                            reinterpret_cast<float4 *>(qs + g * QW)[c] =
                                ldg4(a.qrot + (int64_t)qg[g] * a.Dp + blk * BLK + 4 * c);
                        }
                        __syncwarp();
                    }
                    const int pos = (int)o + m0 + own;
                    // slot g's live mask loses the members m (lane g % 32 holds it)
                    auto drop = [&](int g, unsigned m) {
                        const unsigned cm = lane == (g & 31) ? m : 0u;
                        if (g < 32) la &= ~cm;
                        else lb &= ~cm;
                    };
                    auto finish = [&](int g, float st, const float *qv) {
                        float S = (blk == 0 ? 0.f : Sv[g * 32 + lane]) + st;
                        const bool alive = (am >> g) & 1ull;
                        const float r2 = r2g[g];
                        if (!fin) {
                            if (a.test_on) {
                                // Case 1 / Case 2 of Algorithm 1 (squared test, Sec. 3.2)
                                const bool rej = alive && S > r2 * fe;
                                const unsigned rmk = __ballot_sync(FULL, rej);
                                if (rmk) {
                                    if (rej) am &= ~(1ull << g);
                                    drop(g, rmk);
                                    if (FIXED && rej) {
                                        const int64_t off = (int64_t)qg[g] * a.N + a.ids[pos];
                                        a.decisions[off] = 0;
                                        if (a.dec_dims) a.dec_dims[off] = (int)dstep;
                                    }
                                }
                            }
                            Sv[g * 32 + lane] = S;
                            return;
                        }
                        // Case 3: the exact compare at d = D
                        bool cand = alive;
                        if (Roundoff<T>::u > 0.f && !a.defer_recheck) {
                            // 16-bit storage: only candidates with sqrt(S~) <= r + u ||x||
                            // can have S_D <= r^2; their exact FP32 distance comes from
                            // the FP32 row copy
                            bool need = false;
                            if (alive) {
                                need = !(r2 < INFINITY);
                                if (!need && r2 >= 0.f) {
                                    const float bound =
                                        (sqrtf(r2) + Roundoff<T>::u * a.norms[pos]) * 1.0001f;
                                    need = sqrtf(S) <= bound;
                                }
                            }
                            S = recheck_rows(a.rows32, a.Dp, qv, need, pos, S, lane);
                            cand = need;
                        }
                        const bool posv = cand && S <= r2;
                        if constexpr (FIXED) {
                            if (alive) {
                                const int64_t off = (int64_t)qg[g] * a.N + a.ids[pos];
                                a.decisions[off] = posv ? 1 : 2;
                                if (a.dec_dims) a.dec_dims[off] = a.D;
                            }
                        } else {
                            const unsigned pm = __ballot_sync(FULL, posv);
                            if (pm) {
                                const int q = qg[g];
                                unsigned b0 = 0u;
                                if (lane == 0) b0 = atomicAdd(a.app_n + q, (unsigned)__popc(pm));
                                b0 = __shfl_sync(FULL, b0, 0);
                                if (posv) {
                                    const unsigned idx = b0 + __popc(pm & below);
                                    if (idx < (unsigned)a.cap) {
                                        a.app_d[(int64_t)q * a.cap + idx] = S;
                                        a.app_i[(int64_t)q * a.cap + idx] =
                                            a.defer_recheck ? pos : a.ids[pos];
                                    }
                                }
                            }
                        }
                        am &= ~(1ull << g);
                        drop(g, ~0u);
                    };
                    // ---- dense step: the live slots, two at a time, every
                    // member, from registers
                    for (int g = 0; g < ngq; g += 2) {
                        const bool two = g + 1 < ngq;
                        const unsigned s2 = (unsigned)(sl >> g) & (two ? 3u : 1u);
                        if (s2 == 0u) continue;
                        const float *qv0 = a.qrot + (int64_t)qg[g] * a.Dp;
                        const float *qv1 = two ? a.qrot + (int64_t)qg[g + 1] * a.Dp : qv0;
                        float2 p0[NL], p1[NL];
#pragma unroll
                        for (int k = 0; k < NL; ++k) {
                            p0[k] = make_float2(0.f, 0.f);
                            p1[k] = make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int b = 0; b < DB; ++b) {
                            if (b < nb) {
                                const QPiece<NL> qa = ld_qpiece<NL>(qs + g * QW + b * BLK + jo);
                                const QPiece<NL> qb =
                                    ld_qpiece<NL>(qs + (two ? g + 1 : g) * QW + b * BLK + jo);
#pragma unroll
                                for (int k = 0; k < NL; ++k) {
                                    p0[k] = add_piece_u(v[b][k], qa, p0[k]);
                                    p1[k] = add_piece_u(v[b][k], qb, p1[k]);
                                }
                            }
                        }
                        const float s0 = group_sum<NL>(p0, lane);
                        const float s1 = group_sum<NL>(p1, lane);
                        if (s2 & 1u) finish(g, s0, qv0);
                        if (s2 & 2u) finish(g + 1, s1, qv1);
                    }
                } else {
                    // ---- sparse step: the tile's step staged in shared
                    // memory, then the live (slot, member) pairs, one per
                    // lane, 32 per pass whatever their query
                    if (lane < ngq) live[lane] = la;
                    if (lane + 32 < ngq) live[lane + 32] = lb;
#pragma unroll
                    for (int b = 0; b < DB; ++b)
#pragma unroll
                        for (int k = 0; k < NL; ++k)
                            if (b < nb && ((U >> owner_lane<NL>(gi, k)) & 1u))
                                *reinterpret_cast<V *>(
                                    stile + b * RB + (gi + NG * k) * ROW +
                                    (((lane % NL) ^ Stage<T>::swz(gi + NG * k)) * 16)) =
                                    ld_piece(x + b * stride + k * NG * BLK);
                    __syncwarp();
                    int npr = 0;
                    for (int g = 0; g < ngq; ++g) {
                        const unsigned lv = live[g];
                        if ((lv >> lane) & 1u)
                            pa[npr + __popc(lv & below)] = (unsigned short)((g << 5) | lane);
                        npr += __popc(lv);
                    }
                    __syncwarp();
                    for (int p0 = 0; p0 < npr; p0 += 32) {
                        const bool valid = p0 + lane < npr;
                        const int pr = valid ? pa[p0 + lane] : 0;
                        const int g = pr >> 5, l = pr & 31;
                        const int mt = own_slot<NL>(l);             // member within the tile
                        const int pos = (int)o + m0 + mt;
                        const float *qv = a.qrot + (int64_t)qg[g] * a.Dp;
                        float S = 0.f;
                        if (valid)
                            S = Sv[g * 32 + l] +
                                member_step_sum<T, DB>(stile + mt * ROW, mt, qv + blk * BLK, nb);
                        const float r2 = valid ? r2g[g] : 0.f;
                        bool out = false;                           // continues to the next step
                        if (!fin) {
                            if (valid) {
                                if (S > r2 * fe) {
                                    if constexpr (FIXED) {
                                        const int64_t off = (int64_t)qg[g] * a.N + a.ids[pos];
                                        a.decisions[off] = 0;
                                        if (a.dec_dims) a.dec_dims[off] = (int)dstep;
                                    }
                                } else {
                                    out = true;
                                    Sv[g * 32 + l] = S;
                                }
                            }
                        } else {
                            bool cand = valid;
                            if constexpr (Roundoff<T>::u > 0.f) {
                                bool need = false;
                                if (valid) {
                                    need = !(r2 < INFINITY);
                                    if (!need && r2 >= 0.f) {
                                        const float bound =
                                            (sqrtf(r2) + Roundoff<T>::u * a.norms[pos]) * 1.0001f;
                                        need = sqrtf(S) <= bound;
                                    }
                                }
                                S = recheck_rows(a.rows32, a.Dp, qv, need, pos, S, lane);
                                cand = need;
                            }
                            const bool posv = cand && S <= r2;
                            if constexpr (FIXED) {
                                if (valid) {
                                    const int64_t off = (int64_t)qg[g] * a.N + a.ids[pos];
                                    a.decisions[off] = posv ? 1 : 2;
                                    if (a.dec_dims) a.dec_dims[off] = a.D;
                                }
                            } else if (posv) {
                                const int q = qg[g];
                                const unsigned idx = atomicAdd(a.app_n + q, 1u);
                                if (idx < (unsigned)a.cap) {
                                    a.app_d[(int64_t)q * a.cap + idx] = S;
                                    a.app_i[(int64_t)q * a.cap + idx] = a.ids[pos];
                                }
                            }
                        }
                        // the pairs that stop here, per slot (a slot's pairs
                        // are consecutive): live bits cleared by the slot's
                        // lowest lane
                        const unsigned grp = __match_any_sync(FULL, valid ? g : -1);
                        const unsigned dead = __reduce_or_sync(grp, valid && !out ? 1u << l : 0u);
                        if (valid && dead && lane == __ffs(grp) - 1) live[g] &= ~dead;
                        __syncwarp();
                    }
                    // the registers again from the shared masks
                    la = lane < ngq ? live[lane] : 0u;
                    lb = lane + 32 < ngq ? live[lane + 32] : 0u;
                    am = 0ull;
                    for (int g = 0; g < ngq; ++g)
                        am |= (unsigned long long)((live[g] >> lane) & 1u) << g;
                }
                __syncwarp();
                blk = e;
            }
        }
        if (a.out_dims) {
            if (lane < ngq)
                atomicAdd(reinterpret_cast<unsigned long long *>(a.out_dims + qg[lane]),
                          (unsigned long long)dga);
            if (lane + 32 < ngq)
                atomicAdd(reinterpret_cast<unsigned long long *>(a.out_dims + qg[lane + 32]),
                          (unsigned long long)dgb);
        }
        __syncwarp();
    }
}

// ---- round planning, every round in one pass: the (query, probe rank)
// pairs of each round grouped by cluster.  cnt[r][c] counts them;
// cm_plan_offsets (one block per round) turns the counts into offsets of each
// cluster's query list and of its work items (one per G queries and chunk of
// tpi 32-member tiles, so that large clusters are shared among warps);
// cm_plan_scatter fills the lists and the items.
__device__ __forceinline__ int cm_round_of(const CmRounds &R, int p)
{
    int r = 0;
    while (r + 1 < R.n && p >= R.lo[r + 1]) ++r;
    return r;
}

__global__ void cm_plan_count_kernel(const int32_t *__restrict__ probes, int64_t nq, int pstride,
                                     CmRounds R, int nlist, int *__restrict__ cnt)
{
    const int w = R.lo[R.n] - R.lo[0];
    const int64_t total = nq * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / w;
        const int p = R.lo[0] + (int)(i - q * w);
        atomicAdd(cnt + (size_t)cm_round_of(R, p) * nlist + probes[q * pstride + p], 1);
    }
}

// One block per round: exclusive prefix sums of cnt (-> coff) and of
// ceil(cnt / G) * chunks (-> ioff), the item total, and the cursors cleared.
__device__ __forceinline__ int cm_chunks(const int64_t *off, int c, int tpi)
{
    const int tiles = (int)((off[c + 1] - off[c] + 31) >> 5);
    return (tiles + tpi - 1) / tpi;
}

__global__ void __launch_bounds__(1024) cm_plan_offsets_kernel(const int *__restrict__ cnt_all,
                                                               const int64_t *__restrict__ off,
                                                               int nlist, int G, int tpi,
                                                               int *__restrict__ coff_all,
                                                               int *__restrict__ ioff_all,
                                                               int *__restrict__ cur_all,
                                                               int *__restrict__ n_items)
{
    __shared__ int s_a[32], s_b[32];
    const int r = blockIdx.x;
    const int *cnt = cnt_all + (size_t)r * nlist;
    int *coff = coff_all + (size_t)r * (nlist + 1);
    int *ioff = ioff_all + (size_t)r * nlist;
    int *cur = cur_all + (size_t)r * nlist;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (nlist + 1023) / 1024;
    const int c0 = t * per, c1 = c0 + per < nlist ? c0 + per : nlist;
    int sa = 0, sb = 0;
    for (int c = c0; c < c1; ++c) {
        sa += cnt[c];
        sb += (cnt[c] + G - 1) / G * cm_chunks(off, c, tpi);
    }
    int xa = sa, xb = sb;                 // inclusive warp scans
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int ya = __shfl_up_sync(FULL, xa, d), yb = __shfl_up_sync(FULL, xb, d);
        if (lane >= d) {
            xa += ya;
            xb += yb;
        }
    }
    if (lane == 31) {
        s_a[warp] = xa;
        s_b[warp] = xb;
    }
    __syncthreads();
    if (warp == 0) {
        int ya = s_a[lane], yb = s_b[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int za = __shfl_up_sync(FULL, ya, d), zb = __shfl_up_sync(FULL, yb, d);
            if (lane >= d) {
                ya += za;
                yb += zb;
            }
        }
        s_a[lane] = ya;
        s_b[lane] = yb;
    }
    __syncthreads();
    int ea = xa - sa + (warp > 0 ? s_a[warp - 1] : 0);
    int eb = xb - sb + (warp > 0 ? s_b[warp - 1] : 0);
    for (int c = c0; c < c1; ++c) {
        coff[c] = ea;
        ioff[c] = eb;
        cur[c] = 0;
        ea += cnt[c];
        eb += (cnt[c] + G - 1) / G * cm_chunks(off, c, tpi);
    }
    if (t == 1023) {
        coff[nlist] = ea;
        n_items[r] = eb;
    }
}

__global__ void cm_plan_scatter_kernel(const int32_t *__restrict__ probes, int64_t nq, int pstride,
                                       CmRounds R, int nlist, int G, int tpi,
                                       const int64_t *__restrict__ off,
                                       const int *__restrict__ coff_all,
                                       const int *__restrict__ ioff_all, int *__restrict__ cur_all,
                                       int *__restrict__ qlist, int2 *__restrict__ items)
{
    const int w = R.lo[R.n] - R.lo[0];
    const int64_t total = nq * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / w;
        const int p = R.lo[0] + (int)(i - q * w);
        const int r = cm_round_of(R, p);
        const int c = probes[q * pstride + p];
        const int slot = atomicAdd(cur_all + (size_t)r * nlist + c, 1);
        qlist[nq * (R.lo[r] - R.lo[0]) + coff_all[(size_t)r * (nlist + 1) + c] + slot] = (int)q;
        if (slot % G == 0) {
            const int ch = cm_chunks(off, c, tpi), first = (slot / G) * ch;
            int2 *it = items + R.ibase[r] + ioff_all[(size_t)r * nlist + c] + first;
            for (int t = 0; t < ch; ++t) it[t] = make_int2(c, first + t);
        }
    }
}

// Per query (one warp each): the top-K so far (ids / keys, -1 padded, sorted
// by (distance, id)) and the candidates the round appended merge into the
// new top-K; r^2 becomes the K-th key (+inf while fewer than K are known).
// The appended (key, id) pairs -- 64-bit words, key bits above id, which
// orders non-negative keys as (distance, id) -- are sorted by a warp bitonic
// network in shared memory; every entry of either list then lands at its
// index plus its rank in the other list (the two lists hold distinct ids),
// and the first K are kept.  A long list is first cut, in global memory, to
// the keys whose distance is at most the K-th smallest of both lists; the
// shared memory holds T >= 2K of them.  A list beyond its capacity, or one
// whose cut still exceeds T (ties at the K-th distance), flags the query.
// With `final_pass` the keys are written as the values the search returns.
constexpr int MERGE_WARPS = 4;

__device__ __forceinline__ unsigned below_mask(int lane) { return (1u << lane) - 1u; }

__device__ __forceinline__ unsigned long long mkey(float d, int id)
{
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)id;
}

// entries of the sorted a[0..n) below x
__device__ __forceinline__ int rank_below(const unsigned long long *a, int n, unsigned long long x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Appended distance bits a lane keeps in registers (keys lane + 32 j): lists
// of up to 32 * MERGE_RK entries are read from global memory once.
constexpr int MERGE_RK = 16;

// Calls f(h, valid) on every lane for each distance bit pattern h (the high
// word of a key) of e[0..ne) and of the appended list -- from the registers
// hv when `inreg`, else from gd 8 x 32 at a time -- with warp-uniform control
// flow (f may use warp collectives).
template <typename F>
__device__ __forceinline__ void visit_hi(const unsigned long long *e, int ne, const float *gd,
                                         int na, const unsigned (&hv)[MERGE_RK], bool inreg,
                                         int lane, F f)
{
    for (int i0 = 0; i0 < ne; i0 += 32) {
        const int i = i0 + lane;
        f(i < ne ? (unsigned)(e[i] >> 32) : 0u, i < ne);
    }
    if (inreg) {
#pragma unroll
        for (int j = 0; j < MERGE_RK; ++j)
            if (32 * j < na) f(hv[j], lane + 32 * j < na);
    } else {
        for (int i0 = 0; i0 < na; i0 += 32 * 8) {
            unsigned h[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + 32 * u + lane;
                h[u] = i < na ? __float_as_uint(__ldg(gd + i)) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + 32 * u < na) f(h[u], i0 + 32 * u + lane < na);
        }
    }
}

// The distance bits of the K-th smallest key among e[0..ne) and the
// appended list (distances gd[0..na), their bits in hv when `inreg`): a radix
// select over the bits below the prefix all of them share, 8 bits per pass,
// with a 256-bin histogram in shared memory (lane l owns bins 8l .. 8l+7 for
// the scan); lanes voting for the same bin merge into one atomic.
__device__ __forceinline__ unsigned select_hi(const unsigned long long *e, int ne,
                                              const float *gd, int na,
                                              const unsigned (&hv)[MERGE_RK], bool inreg, int K,
                                              unsigned *hist, int lane)
{
    unsigned lo = 0xffffffffu, hi = 0u;
    visit_hi(e, ne, gd, na, hv, inreg, lane, [&](unsigned h, bool v) {
        if (v) {
            lo = min(lo, h);
            hi = max(hi, h);
        }
    });
    lo = __reduce_min_sync(FULL, lo);
    hi = __reduce_max_sync(FULL, hi);
    if (lo == hi) return lo;
    const int hb = 31 - __clz(lo ^ hi);                  // highest differing bit
    unsigned pmask = hb == 31 ? 0u : ~((2u << hb) - 1u);  // bits already fixed
    unsigned prefix = lo & pmask;
    unsigned kk = (unsigned)K;
    for (int top = hb; top >= 0; top -= 8) {
        const int shift = top >= 7 ? top - 7 : 0;
        const unsigned dmask = (2u << (top - shift)) - 1u;   // <= 8 bits
#pragma unroll
        for (int j = 0; j < 8; ++j) hist[lane * 8 + j] = 0u;
        __syncwarp();
        visit_hi(e, ne, gd, na, hv, inreg, lane, [&](unsigned h, bool v) {
            const unsigned bin = v && (h & pmask) == prefix ? (h >> shift) & dmask : 256u;
            const unsigned peers = __match_any_sync(FULL, bin);
            if (bin < 256u && lane == __ffs(peers) - 1) atomicAdd(hist + bin, (unsigned)__popc(peers));
        });
        __syncwarp();
        unsigned c[8], sum = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            c[j] = hist[8 * lane + j];
            sum += c[j];
        }
        unsigned incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += y;
        }
        const unsigned excl = incl - sum;
        const unsigned hit = __ballot_sync(FULL, excl < kk && kk <= incl);
        const int src = __ffs(hit) - 1;
        unsigned bin = 0u, before = 0u;
        if (lane == src) {
            unsigned acc = excl;
            bool found = false;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!found && acc + c[j] >= kk) {
                    found = true;
                    bin = 8u * lane + j;
                    before = acc;
                }
                acc += c[j];
            }
        }
        bin = __shfl_sync(FULL, bin, src);
        before = __shfl_sync(FULL, before, src);
        prefix |= bin << shift;
        pmask |= dmask << shift;
        kk -= before;
        __syncwarp();
        if (shift == 0) break;
    }
    return prefix;
}

__global__ void __launch_bounds__(MERGE_WARPS * 32, 8) cm_merge_kernel(CmMergeArgs m)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = m.K;
    unsigned long long *ak = reinterpret_cast<unsigned long long *>(smraw) +
                             (size_t)warp * (m.T + K + 128);
    unsigned long long *ek = ak + m.T;
    unsigned *hist = reinterpret_cast<unsigned *>(ek + K);
    const unsigned long long NONE = ~0ull;
    for (int64_t q = (int64_t)blockIdx.x * MERGE_WARPS + warp; q < m.nq;
         q += (int64_t)gridDim.x * MERGE_WARPS) {
        unsigned na = m.app_n ? m.app_n[q] : 0u;
        if (na > (unsigned)m.cap) {
            if (lane == 0) m.ovf[q] = 1;
            na = (unsigned)m.cap;
        }
        int64_t *ids = m.ids + q * K;
        float *dk = m.d2 + q * K;
        if (na == 0u && !m.final_pass) {
            if (lane == 0) m.r2[q] = ids[K - 1] >= 0 ? dk[K - 1] : INFINITY;
            continue;
        }
        int ne = 0;                                   // existing entries (a prefix)
        for (int k0 = 0; k0 < K; k0 += 32) {
            const int k = k0 + lane;
            const bool has = k < K && ids[k] >= 0;
            if (k < K) ek[k] = has ? mkey(dk[k], (int)ids[k]) : NONE;
            ne += __popc(__ballot_sync(FULL, has));
        }
        const float *gd = m.app_d + q * m.cap;
        const int32_t *gi = m.app_i + q * m.cap;
        auto akey = [&](int i) { return mkey(gd[i], gi[i]); };
        if (na > 64u && ne + (int)na > K) {
            // many appended: keep only the keys whose distance is at most the
            // K-th smallest of both lists (ties kept), then sort those
            const int n = (int)na;
            const bool inreg = n <= 32 * MERGE_RK;
            unsigned hv[MERGE_RK];
#pragma unroll
            for (int j = 0; j < MERGE_RK; ++j) {
                const int i = lane + 32 * j;
                hv[j] = inreg && i < n ? __float_as_uint(__ldg(gd + i)) : 0u;
            }
            const unsigned th = select_hi(ek, ne, gd, n, hv, inreg, K, hist, lane);
            int kept = 0;
            for (int i0 = 0; i0 < n; i0 += 32 * 8) {
                unsigned long long v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 32 * u + lane;
                    v[u] = i < n ? akey(i) : NONE;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (i0 + 32 * u >= n) break;
                    const bool keep = i0 + 32 * u + lane < n && (unsigned)(v[u] >> 32) <= th;
                    const unsigned km = __ballot_sync(FULL, keep);
                    const int at = kept + __popc(km & below_mask(lane));
                    if (keep && at < m.T) ak[at] = v[u];
                    kept += __popc(km);
                }
            }
            if (kept > m.T) {
                // ties at the K-th distance beyond the sort capacity: the
                // query is searched again (query-major); its list is dropped
                if (lane == 0) {
                    m.ovf[q] = 1;
                    if (m.app_n) m.app_n[q] = 0u;
                }
                __syncwarp();
                continue;
            }
            na = (unsigned)kept;
            ne = rank_below(ek, ne, (unsigned long long)(th + 1u) << 32);
        } else {
            for (int i = lane; i < (int)na; i += 32) ak[i] = akey(i);
        }
        __syncwarp();
        int T = 32;
        while (T < (int)na) T <<= 1;
        for (int i = (int)na + lane; i < T; i += 32) ak[i] = NONE;
        __syncwarp();
        for (int size = 2; size <= T; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = lane; i < T; i += 32) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const unsigned long long x = ak[i], y = ak[j];
                        const bool up = (i & size) == 0;
                        if ((y < x) == up) {
                            ak[i] = y;
                            ak[j] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        const int total = ne + (int)na < K ? ne + (int)na : K;
        unsigned long long kth = NONE;
        auto put = [&](int pos, unsigned long long key) {
            const int id = (int)(key & 0xffffffffu);
            const float d = __uint_as_float((unsigned)(key >> 32));
            ids[pos] = id;
            dk[pos] = m.final_pass ? out_value(m.metric, d, true) : d;
            if (pos == K - 1) kth = key;
        };
        // reads of ids / dk are done (ek holds them); positions are distinct
        __syncwarp();
        for (int k = lane; k < ne; k += 32) {
            const int pos = k + rank_below(ak, (int)na, ek[k]);
            if (pos < K) put(pos, ek[k]);
        }
        for (int j = lane; j < (int)na; j += 32) {
            const int pos = j + rank_below(ek, ne, ak[j]);
            if (pos < K) put(pos, ak[j]);
        }
        for (int k = total + lane; k < K; k += 32) {
            ids[k] = -1;
            dk[k] = m.final_pass ? out_value(m.metric, 0.f, false) : INFINITY;
        }
        // the lane that placed the K-th entry publishes r^2
        const unsigned km = __ballot_sync(FULL, kth != NONE);
        if (km) {
            if (lane == __ffs(km) - 1) m.r2[q] = __uint_as_float((unsigned)(kth >> 32));
        } else if (lane == 0) {
            m.r2[q] = INFINITY;
        }
        if (lane == 0 && m.app_n) m.app_n[q] = 0u;
        __syncwarp();
    }
}

// Round 0 of a 16-bit search: per query (one warp) the list holds every
// member of the nearest cluster with its approximate distance a_i = sqrt(S~_i)
// and CSR row.  The exact distance e_i differs from a_i by at most
// ||y~_i - y_i|| <= u ||y_i||, so B, the K-th smallest of a_i + u ||y_i||, is at
// least the exact K-th distance, and only members with a_i <= B + u ||y_i||
// can be among the K nearest.  B is taken as the K-th smallest of the lanes'
// four smallest bounds (the K-th of a subset: never below the K-th of all,
// so still valid); with K > 128 every member is kept.  The kept members get
// their exact FP32 distances from the FP32 rows (recheck_rows, the same
// arithmetic as every other recheck) and their ids; the list is compacted.
__global__ void __launch_bounds__(MERGE_WARPS * 32) cm_recheck0_kernel(CmRecheck0Args r)
{
    __shared__ unsigned s_w[MERGE_WARPS][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned *w4 = s_w[warp];
    for (int64_t q = (int64_t)blockIdx.x * MERGE_WARPS + warp; q < r.nq;
         q += (int64_t)gridDim.x * MERGE_WARPS) {
        unsigned na = r.app_n[q];
        if (na > (unsigned)r.cap) na = (unsigned)r.cap;   // the merge flags the overflow
        const int n = (int)na;
        float *gd = r.app_d + q * r.cap;
        int32_t *gi = r.app_i + q * r.cap;
        float B = INFINITY;
        if (n > r.K && r.K <= 128) {
            // each lane's four smallest bounds a_i + u ||y_i|| (as float bits:
            // non-negative floats order like their bit patterns)
            unsigned t0 = ~0u, t1 = ~0u, t2 = ~0u, t3 = ~0u;
            for (int i0 = 0; i0 < n; i0 += 32 * 8) {
                float sd[8];
                int pr[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int i = i0 + 32 * k + lane;
                    sd[k] = i < n ? gd[i] : 0.f;
                    pr[k] = i < n ? gi[i] : 0;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (i0 + 32 * k + lane < n) {
                        unsigned x = __float_as_uint(sqrtf(sd[k]) + r.u * r.norms[pr[k]]);
                        unsigned m;
                        m = min(t0, x); x = max(t0, x); t0 = m;
                        m = min(t1, x); x = max(t1, x); t1 = m;
                        m = min(t2, x); x = max(t2, x); t2 = m;
                        t3 = min(t3, x);
                    }
                }
            }
            w4[lane * 4 + 0] = t0;
            w4[lane * 4 + 1] = t1;
            w4[lane * 4 + 2] = t2;
            w4[lane * 4 + 3] = t3;
            __syncwarp();
            for (int size = 2; size <= 128; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = lane; i < 128; i += 32) {
                        const int j = i ^ stride;
                        if (j > i) {
                            const unsigned x = w4[i], y = w4[j];
                            if ((x > y) == ((i & size) == 0)) {
                                w4[i] = y;
                                w4[j] = x;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            const unsigned kb = w4[r.K - 1];
            B = kb == ~0u ? INFINITY : __uint_as_float(kb) * 1.0001f;
            __syncwarp();
        }
        // keep (in list order, compacted in place) the members that can be
        // among the K nearest, then their exact distances, 32 at a time
        int kept = 0;
        const float *qv = r.qrot + q * r.Dp;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            float sd = 0.f;
            int pr = 0;
            bool keep = false;
            if (i < n) {
                sd = gd[i];
                pr = gi[i];
                keep = !(B < INFINITY) ||
                       sqrtf(sd) <= (B + r.u * r.norms[pr]) * 1.0001f;
            }
            const unsigned km = __ballot_sync(FULL, keep);
            // exact FP32 distances of the kept members of this chunk
            const float S = recheck_rows(r.rows32, r.Dp, qv, keep, pr, sd, lane);
            __syncwarp();                     // the chunk is read before it is written
            if (keep) {
                const int at = kept + __popc(km & below_mask(lane));
                gd[at] = S;
                gi[at] = r.ids[pr];
            }
            kept += __popc(km);
        }
        __syncwarp();
        if (lane == 0 && r.app_n[q] <= (unsigned)r.cap) r.app_n[q] = (unsigned)kept;
    }
}

// Items (query, one split) of the queries whose lists overflowed, for a
// query-major re-run.
__global__ void cm_overflow_items_kernel(const int *__restrict__ ovf, int64_t nq,
                                         int2 *__restrict__ items, int *__restrict__ n_items)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x)
        if (ovf[q]) items[atomicAdd(n_items, 1)] = make_int2((int)q, (0 << 16) | 1);
}

// Probe slot p of every query is cluster p (the fixed-threshold scan of all
// clusters).
__global__ void cm_all_clusters_kernel(int32_t *__restrict__ probes, int64_t nq, int nlist)
{
    const int64_t total = nq * nlist;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        probes[i] = (int32_t)(i % nlist);
}

typedef void (*CmKernel)(CmArgs);

template <typename T, bool FIXED>
CmKernel cm_kernel_db(int db)
{
    switch (db) {
    case 1: return cm_scan_kernel<T, 1, FIXED>;
    case 2: return cm_scan_kernel<T, 2, FIXED>;
    case 3: return cm_scan_kernel<T, 3, FIXED>;
    default: return cm_scan_kernel<T, 4, FIXED>;
    }
}

template <typename T>
CmKernel cm_kernel_t(const CmArgs &a)
{
    return a.decisions ? cm_kernel_db<T, true>(a.db) : cm_kernel_db<T, false>(a.db);
}

CmKernel cm_kernel_for(const CmArgs &a)
{
    if (a.storage == ADSX_F32) return cm_kernel_t<float>(a);
    if (a.storage == ADSX_BF16) return cm_kernel_t<__nv_bfloat16>(a);
    return cm_kernel_t<__half>(a);
}

unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

size_t cm_smem_bytes(int G, int db, int storage)
{
    const int row = storage == ADSX_F32 ? Stage<float>::ROW : Stage<__half>::ROW;
    return (size_t)CmCarve(G, db, row).bytes * CM_WARPS;
}

cudaError_t launch_cm_plan(const int32_t *probes, int64_t nq, int pstride, const CmRounds &R,
                           int nlist, int G, int tpi, const int64_t *off, CmPlan &pl,
                           cudaStream_t s)
{
    if (R.n < 1 || R.n > CM_MAX_ROUNDS) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(pl.cnt, 0, sizeof(int) * (size_t)R.n * nlist, s);
    if (e != cudaSuccess) return e;
    const int64_t work = nq * (int64_t)(R.lo[R.n] - R.lo[0]);
    cm_plan_count_kernel<<<grid_for(work, 256), 256, 0, s>>>(probes, nq, pstride, R, nlist, pl.cnt);
    cm_plan_offsets_kernel<<<R.n, 1024, 0, s>>>(pl.cnt, off, nlist, G, tpi, pl.coff, pl.ioff, pl.cur,
                                                pl.n_items);
    cm_plan_scatter_kernel<<<grid_for(work, 256), 256, 0, s>>>(probes, nq, pstride, R, nlist, G, tpi,
                                                                off, pl.coff, pl.ioff, pl.cur,
                                                                pl.qlist, pl.items);
    return cudaGetLastError();
}

cudaError_t launch_cm_scan(const CmArgs &a, int device, cudaStream_t s)
{
    if (a.db < 1 || a.db > CM_MAX_DB || a.G < 1 || a.G > CM_MAX_G || a.tpi < 1)
        return cudaErrorInvalidValue;
    const CmKernel k = cm_kernel_for(a);
    const size_t smem = cm_smem_bytes(a.G, a.db, a.storage);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, CM_THREADS, smem);
    if (per < 1) per = 1;
    int64_t grid = (int64_t)nsm * per;
    const int64_t need = ((int64_t)a.items_cap + CM_WARPS - 1) / CM_WARPS;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(a.work_counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)grid, CM_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cm_merge(const CmMergeArgs &m, cudaStream_t s)
{
    if (m.nq <= 0) return cudaSuccess;
    CmMergeArgs b = m;
    // the sort capacity: every list of at most 64 or whose merge cannot
    // exceed K (na <= K) fits, and the cut of a longer one (K plus ties)
    int T = 128;
    while (T < 2 * m.K) T <<= 1;
    b.T = T;
    // per warp: appended keys, existing keys, a 256-bin histogram
    const size_t smem = (size_t)(T + m.K + 128) * 8 * MERGE_WARPS;
    cudaError_t e = cudaFuncSetAttribute(cm_merge_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (m.nq + MERGE_WARPS - 1) / MERGE_WARPS;
    if (grid > 152 * 16) grid = 152 * 16;
    cm_merge_kernel<<<(unsigned)grid, MERGE_WARPS * 32, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_cm_recheck0(const CmRecheck0Args &r, cudaStream_t s)
{
    if (r.nq <= 0) return cudaSuccess;
    int64_t grid = (r.nq + MERGE_WARPS - 1) / MERGE_WARPS;
    if (grid > 152 * 16) grid = 152 * 16;
    cm_recheck0_kernel<<<(unsigned)grid, MERGE_WARPS * 32, 0, s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_cm_overflow_items(const int *ovf, int64_t nq, int2 *items, int *n_items,
                                     cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(n_items, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    cm_overflow_items_kernel<<<grid_for(nq, 256), 256, 0, s>>>(ovf, nq, items, n_items);
    return cudaGetLastError();
}

cudaError_t launch_cm_all_clusters(int32_t *probes, int64_t nq, int nlist, cudaStream_t s)
{
    cm_all_clusters_kernel<<<grid_for(nq * nlist, 256), 256, 0, s>>>(probes, nq, nlist);
    return cudaGetLastError();
}

}  // namespace adsx
