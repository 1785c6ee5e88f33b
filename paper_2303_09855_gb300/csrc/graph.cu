// graph.cu -- graph-based search with ADSampling DCOs (HNSW+, Sec. 4): the
// greedy beam search HNSW runs on its base layer (Sec. 2.2.1), each DCO
// being Algorithm 1 against the largest distance of the result set R.
//
// The proximity graph is a kNN graph of fixed degree <= 32 (one neighbour per
// lane) over the vectors of an FP32 index, read in place from its
// dim-blocked layout through a per-vertex address map.  HNSW's upper layers
// only find a start vertex; here each query starts from the entry vertices
// of its n_entry nearest clusters (per cluster, the member nearest to the
// centroid, then farthest-point samples: a k-means cluster can hold several
// mutually unreachable parts of a kNN graph).
//
// graph_search_kernel: one warp per query, persistent, as many warps as fit
// on the SMs, each taking the next query from a counter (HNSW+; with pp set,
// HNSW++ of Sec. 5.1: an exact K-set R1 gives the DCO threshold and the
// output, the beam keeps each DCO's observed distance).  R (capacity ef) is a
// sorted array of (distance, id) with an "expanded" flag; the search set S is
// R's unexpanded entries (an entry evicted from R cannot matter again).  The
// start vertices (32 list positions at a time), then each expansion's
// neighbours, form batches of one vertex per lane: they pass an exact visited
// test (a per-warp bitmap over all vertices, its set bits cleared after the
// query), the fresh ones run Algorithm 1 against r = R's largest distance,
// fixed for the batch (the next step's blocks prefetched into L2 while a
// step's test is pending), and the accepted ones are sorted by a warp
// bitonic network and merged into R by rank.  Each iteration expands R's
// first unexpanded entry.
#include <climits>

#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int GW = 4;                       // warps per block
constexpr unsigned FULL = 0xffffffffu;

// Asks L2 for the line holding p (a global address); no register result.
__device__ __forceinline__ void prefetch_l2(const float *p)
{
    asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tprefetch.global.L2 [ga];\n\t}"
                 :: "l"(p));
}

__device__ __forceinline__ bool pless(float d1, int i1, float d2, int i2)
{
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

// The least t >= 0 with fl(t f) >= S (f > 0), i.e. the least threshold under
// which the squared test "S > t f" passes: fl(t f) does not decrease as t
// grows, so the correctly rounded S / f is moved to the boundary (in practice
// one float step at most; the loops are bounded).
__device__ __forceinline__ float pass_bound(float S, float f)
{
    float t = __fdiv_rn(S, f);
    for (int it = 0; it < 64 && __fmul_rn(t, f) < S; ++it) t = nextafterf(t, INFINITY);
    for (int it = 0; it < 64 && t > 0.f; ++it) {
        const float pt = nextafterf(t, 0.f);
        if (__fmul_rn(pt, f) >= S) t = pt;
        else break;
    }
    return t;
}

// number of entries of the sorted (d, i)[0..n) that precede (x, xi)
__device__ __forceinline__ int rank_in(const float *d, const int *i, int n, float x, int xi)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pless(d[mid], i[mid], x, xi)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Row r of a chunk of kNN lists is vertex row0 + r: its neighbours are the
// listed ids other than itself, -1 padded.
__global__ void knn_to_graph_kernel(const int64_t *__restrict__ knn, int64_t N, int64_t row0,
                                    int Kk, int degree, int32_t *__restrict__ nbr)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        for (int j = 0; j < Kk && k < degree; ++j) {
            const int64_t v = knn[r * Kk + j];
            if (v >= 0 && v != row0 + r) nbr[r * degree + k++] = (int32_t)v;
        }
        for (; k < degree; ++k) nbr[r * degree + k] = -1;
    }
}

// vbase[id] = element offset of the vertex's block 0, vstride[id] = 16 n_c.
__global__ void vertex_map_kernel(const int64_t *__restrict__ off, int nlist,
                                  const int32_t *__restrict__ ids, int Dp,
                                  int64_t *__restrict__ vbase, int32_t *__restrict__ vstride)
{
    for (int c = blockIdx.x; c < nlist; c += gridDim.x) {
        const int64_t o = off[c], n = off[c + 1] - o;
        for (int64_t m = threadIdx.x; m < n; m += blockDim.x) {
            const int32_t id = ids[o + m];
            vbase[id] = o * Dp + m * BLK;
            vstride[id] = (int32_t)(n * BLK);
        }
    }
}

// One warp per cluster, E start vertices chosen by farthest-point sampling:
// entry 0 is the member nearest to the (rotated) centroid; entry e is the
// member whose distance to the nearest of entries 0..e-1 is largest (ties by
// id; -1 once every member coincides with a chosen one, or for an empty
// cluster).  mind[o + m] keeps member m's distance to the chosen set.
__global__ void cluster_entry_kernel(const float *__restrict__ data, const int64_t *__restrict__ off,
                                     const int32_t *__restrict__ ids, const float *__restrict__ cents,
                                     int nlist, int Dp, int E, float *__restrict__ mind,
                                     int64_t *__restrict__ entry)
{
    const int lane = threadIdx.x & 31;
    const int nblk = Dp / BLK;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nlist; c += nw) {
        const int64_t o = off[c], n = off[c + 1] - o;
        const float *cb = data + o * Dp;
        const float *cq = cents + c * Dp;
        float best = INFINITY;
        int bid = INT_MAX;
        int64_t bm = 0;
        for (int64_t m = lane; m < n; m += 32) {
            float S = 0.f;
            for (int b = 0; b < nblk; ++b) S = accum_block_f32(cb + b * n * BLK + m * BLK, cq + b * BLK, S);
            const int id = ids[o + m];
            if (pless(S, id, best, bid)) {
                best = S;
                bid = id;
                bm = m;
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const float ob = __shfl_xor_sync(FULL, best, s);
            const int oi = __shfl_xor_sync(FULL, bid, s);
            const int64_t om = __shfl_xor_sync(FULL, bm, s);
            if (pless(ob, oi, best, bid)) {
                best = ob;
                bid = oi;
                bm = om;
            }
        }
        if (lane == 0) entry[c * E] = n > 0 ? (int64_t)bid : -1;
        bool done = n == 0;
        for (int e = 1; e < E; ++e) {
            float far = -1.f;
            int fid = INT_MAX;
            int64_t fm = 0;
            if (!done) {
                const float *xs = cb + bm * BLK;            // the entry chosen last
                for (int64_t m = lane; m < n; m += 32) {
                    float S = 0.f;
                    for (int b = 0; b < nblk; ++b)
                        S = accum_block_f32(cb + b * n * BLK + m * BLK, xs + b * n * BLK, S);
                    const float md = e == 1 ? S : fminf(mind[o + m], S);
                    mind[o + m] = md;
                    const int id = ids[o + m];
                    if (md > far || (md == far && id < fid)) {
                        far = md;
                        fid = id;
                        fm = m;
                    }
                }
            }
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const float of = __shfl_xor_sync(FULL, far, s);
                const int oi = __shfl_xor_sync(FULL, fid, s);
                const int64_t om = __shfl_xor_sync(FULL, fm, s);
                if (of > far || (of == far && oi < fid)) {
                    far = of;
                    fid = oi;
                    fm = om;
                }
            }
            done = done || !(far > 0.f);
            if (lane == 0) entry[c * E + e] = done ? (int64_t)-1 : (int64_t)fid;
            bm = fm;
        }
    }
}

// One warp's shared memory: the query, the beam R (two buffers of distance,
// id and expanded flag), the exact K-set R1 of HNSW++ (two buffers), two
// 32-entry staging areas for sorted additions, and each lane's partial
// distance after every Algorithm 1 step of the current batch (nst steps).
__host__ __device__ __forceinline__ size_t graph_warp_bytes(int Dp, int ef, int K, int nst)
{
    const size_t cap = (size_t)ef + 32, cap1 = (size_t)K + 32;
    return (((size_t)Dp * 4 + cap * 4 * 6 + cap1 * 4 * 4 + 32 * 8 * 2 + (size_t)nst * 32 * 4) +
            15) & ~(size_t)15;
}

// Ascending bitonic sort of one 64-bit key per lane.
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long key, int lane)
{
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, key, stride);
            const bool lower = (lane & stride) == 0;
            const bool up = (lane & size) == 0;
            key = (lower == up) ? (o < key ? o : key) : (o > key ? o : key);
        }
    }
    return key;
}

__device__ __forceinline__ unsigned long long dkey(float d, int id)
{
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)id;   // d >= 0
}

// Merges the sorted (cd, ci[, cx])[0..n) and the sorted additions (ad, ai)[0..na)
// into (nd, ni[, nx]), keeping the first `keep`; additions get flag 0.  Returns
// the new count.  Entries are distinct, so every position is written once.
__device__ __forceinline__ int warp_merge(const float *cd, const int *ci, const int *cx, int n,
                                          const float *ad, const int *ai, int na, float *nd,
                                          int *ni, int *nx, int keep, int lane)
{
    for (int k = lane; k < n; k += 32) {
        const int pos = k + rank_in(ad, ai, na, cd[k], ci[k]);
        if (pos < keep) {
            nd[pos] = cd[k];
            ni[pos] = ci[k];
            if (nx) nx[pos] = cx[k];
        }
    }
    if (lane < na) {
        const int pos = lane + rank_in(cd, ci, n, ad[lane], ai[lane]);
        if (pos < keep) {
            nd[pos] = ad[lane];
            ni[pos] = ai[lane];
            if (nx) nx[pos] = 0;
        }
    }
    __syncwarp();
    return n + na < keep ? n + na : keep;
}

// Stages the lanes' keys with `take` sorted into (ad, ai); returns their count.
__device__ __forceinline__ int stage_sorted(bool take, float d, int id, float *ad, int *ai,
                                            int lane)
{
    const int na = __popc(__ballot_sync(FULL, take));
    if (na) {
        const unsigned long long key = warp_sort32(take ? dkey(d, id) : ~0ull, lane);
        if (lane < na) {
            ad[lane] = __uint_as_float((unsigned)(key >> 32));
            ai[lane] = (int)(key & 0xffffffffu);
        }
        __syncwarp();
    }
    return na;
}

__global__ void __launch_bounds__(GW * 32) graph_search_kernel(GraphArgs g)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int cap = g.ef + 32, cap1 = g.K + 32;
    unsigned char *base = smraw + graph_warp_bytes(g.Dp, g.ef, g.K, g.nst) * warp;
    float *qv = reinterpret_cast<float *>(base);
    float *rd = qv + g.Dp, *nd = rd + cap;
    int *ri = reinterpret_cast<int *>(nd + cap), *ni = ri + cap;
    int *rx = ni + cap, *nx = rx + cap;
    float *kd = reinterpret_cast<float *>(nx + cap), *kd2 = kd + cap1;
    int *ki = reinterpret_cast<int *>(kd2 + cap1), *ki2 = ki + cap1;
    float *ad = reinterpret_cast<float *>(ki2 + cap1);
    int *ai = reinterpret_cast<int *>(ad + 32);
    float *ad1 = reinterpret_cast<float *>(ai + 32);
    int *ai1 = reinterpret_cast<int *>(ad1 + 32);
    float *sst = reinterpret_cast<float *>(ai1 + 32);     // nst x 32 partial distances
    const int64_t gw = (int64_t)blockIdx.x * GW + warp;
    if (gw >= g.warps) return;
    unsigned *bm = g.bitmap + gw * g.bm_words;
    int32_t *vl = g.vlist + gw * g.vcap;

    // queries are taken one at a time from a shared counter: search lengths
    // vary, so a static split would leave warps idle at the end
    auto next_query = [&]() {
        unsigned long long t = 0ull;
        if (lane == 0) t = atomicAdd(g.qnext, 1ull);
        return (int64_t)__shfl_sync(FULL, t, 0);
    };
    for (int64_t q = next_query(); q < g.nq; q = next_query()) {
        for (int i = lane; i < g.Dp; i += 32) qv[i] = g.qrot[q * g.Dp + i];
        __syncwarp();
        unsigned long long dims = 0ull;
        int vcount = 0, nR = 0, n1 = 0;
        // One batch of up to 32 vertices (one per lane, in list order; fresh
        // ones only), with the outcome of the paper's order: each vertex's
        // DCO faces the threshold as it stands after the vertices before it.
        // All DCOs first run side by side against the threshold at the
        // batch's start (an upper bound of every later one), recording S_d
        // after each step; a threshold that only shrinks can only move a
        // decision to an earlier rejection, which the recorded S_d settle
        // exactly (the same FP32 comparison).  So the decisions are then
        // replayed in list order: each vertex knows the least threshold under
        // which it is positive, the vertices that enter the set giving the
        // threshold (R for HNSW+, R1 for HNSW++) are found one after another
        // in registers, and each vertex is finally decided against the
        // threshold of its turn.  The dims counted are those of the paper's
        // order.
        auto dco_batch = [&](int v, bool fresh) {
            const bool full0 = nR == g.ef;
            const float rmax0 = full0 ? rd[nR - 1] : INFINITY;
            const int rid0 = full0 ? ri[nR - 1] : INT_MAX;
            float th = g.pp ? (n1 == g.K ? kd[n1 - 1] : INFINITY) : rmax0;
            // Algorithm 1 against th (squared test of Sec. 3.2), S_d recorded
            float S = 0.f;
            int blk = 0, nst = 0;
            bool alive = fresh;
            const float *x = g.data + (fresh ? g.vbase[v] : 0);
            const int64_t st = fresh ? g.vstride[v] : 0;
            while (__ballot_sync(FULL, alive)) {
                if (alive) {
                    const int e2 = blk + g.db < g.nblk ? blk + g.db : g.nblk;
                    // the next step's blocks head for L2 while this step's
                    // test is pending (wasted only if the test rejects)
                    const int e3 = e2 + g.db < g.nblk ? e2 + g.db : g.nblk;
                    for (int b = e2; b < e3; ++b) prefetch_l2(x + b * st);
                    for (int b = blk; b < e2; ++b) S = accum_block_f32(x + b * st, qv + b * BLK, S);
                    blk = e2;
                    sst[nst * 32 + lane] = S;
                    ++nst;
                    if (blk >= g.nblk || (g.test_on && S > th * g.ftab[blk])) alive = false;
                }
            }
            // the decision against threshold t from the recorded steps:
            // 0 rejected at d < D, 1 positive (d = D, S_D <= t), 2 negative
            // at d = D; dstep the dims, sdec S_d where Algorithm 1 stopped
            int dec = 0, dstep = 0;
            float sdec = 0.f;
            auto decide = [&](float t) {
                int b2 = 0;
                for (int k = 0; k < nst; ++k) {
                    b2 = b2 + g.db < g.nblk ? b2 + g.db : g.nblk;
                    const float Sk = sst[k * 32 + lane];
                    if (b2 >= g.nblk) {
                        dec = Sk <= t ? 1 : 2;
                        dstep = g.D;
                        sdec = Sk;
                        return;
                    }
                    if (g.test_on && Sk > t * g.ftab[b2]) {
                        dec = 0;
                        dstep = b2 * BLK < g.D ? b2 * BLK : g.D;
                        sdec = Sk;
                        return;
                    }
                }
            };
            // tpos: the smallest threshold under which this vertex is positive
            // (every recorded step passes and S_D <= t): the larger of S_D
            // and, per earlier step, the least t with fl(t f) >= S_d; +inf if
            // th already rejects it (a smaller threshold rejects it too)
            float tpos = INFINITY, sD = 0.f;
            if (fresh) {
                decide(th);
                if (dec == 1) {
                    sD = sdec;
                    tpos = sdec;
                    int b2 = 0;
                    for (int k = 0; k + 1 < nst; ++k) {
                        b2 = b2 + g.db < g.nblk ? b2 + g.db : g.nblk;
                        tpos = fmaxf(tpos, pass_bound(sst[k * 32 + lane], g.ftab[b2]));
                    }
                }
            }
            // Replay in list order.  T is the set that gives the threshold (R
            // for HNSW+, R1 for HNSW++, C entries at most); E holds the keys of
            // this batch's vertices that entered it so far, sorted, lane e the
            // e-th; thk is the C-th smallest key of T and E (~0: T and E hold
            // fewer), the threshold for the vertices after the last one that
            // entered.  The first vertex still positive under thk with a key
            // below it enters next; each vertex keeps the thk of its turn.
            const int C = g.pp ? g.K : g.ef;
            const int nT = g.pp ? n1 : nR;
            const float *Td = g.pp ? kd : rd;
            const int *Ti = g.pp ? ki : ri;
            unsigned long long thk = nT == C ? dkey(Td[C - 1], Ti[C - 1]) : ~0ull;
            unsigned long long E = ~0ull, mythk = thk;
            const unsigned long long mykey = dkey(sD, v);
            int m = 0;
            unsigned settled = 0u;
            for (;;) {
                const float thd = thk == ~0ull ? INFINITY : __uint_as_float((unsigned)(thk >> 32));
                const bool enter = fresh && !((settled >> lane) & 1u) && thd >= tpos && mykey < thk;
                const unsigned em = __ballot_sync(FULL, enter);
                if (!em) break;
                const int j = __ffs(em) - 1;
                settled |= (j == 31) ? FULL : ((2u << j) - 1u);
                const unsigned long long kj = __shfl_sync(FULL, mykey, j);
                const int p = __popc(__ballot_sync(FULL, lane < m && E < kj));
                const unsigned long long up = __shfl_up_sync(FULL, E, 1);
                if (lane == p) E = kj;
                else if (lane > p && lane <= m) E = up;
                ++m;
                if (nT + m >= C) {
                    // the C smallest of T and E: the ts smallest of E and the
                    // C - ts smallest of T, ts the largest t <= min(m, C) with
                    // E[t-1] below T[C-t] (or T shorter than C - t + 1)
                    const int t = lane + 1, hi_t = m < C ? m : C;
                    const bool P = t <= hi_t && (C - t >= nT || E < dkey(Td[C - t], Ti[C - t]));
                    const int ts = __popc(__ballot_sync(FULL, P));
                    const unsigned long long ea = __shfl_sync(FULL, E, ts > 0 ? ts - 1 : 0);
                    const unsigned long long k1 = ts > 0 ? ea : 0ull;
                    const unsigned long long k2 =
                        C - ts - 1 >= 0 ? dkey(Td[C - ts - 1], Ti[C - ts - 1]) : 0ull;
                    thk = k1 > k2 ? k1 : k2;
                }
                if (lane > j) mythk = thk;
            }
            // every vertex's own outcome, against the threshold of its turn
            if (fresh)
                decide(mythk == ~0ull ? INFINITY : __uint_as_float((unsigned)(mythk >> 32)));
            // the entered keys join T (a bounded set fed one at a time ends
            // as the smallest of all it was offered)
            if (m > 0) {
                float *sd_ = g.pp ? ad1 : ad;
                int *si_ = g.pp ? ai1 : ai;
                if (lane < m) {
                    sd_[lane] = __uint_as_float((unsigned)(E >> 32));
                    si_[lane] = (int)(E & 0xffffffffu);
                }
                __syncwarp();
                if (!g.pp) {
                    nR = warp_merge(rd, ri, rx, nR, ad, ai, m, nd, ni, nx, g.ef, lane);
                    float *tf = rd; rd = nd; nd = tf;
                    int *ti = ri; ri = ni; ni = ti;
                    ti = rx; rx = nx; nx = ti;
                } else {
                    n1 = warp_merge(kd, ki, nullptr, n1, ad1, ai1, m, kd2, ki2, nullptr, g.K, lane);
                    float *tf = kd; kd = kd2; kd2 = tf;
                    int *ti = ki; ki = ki2; ki2 = ti;
                }
            }
            if (fresh) dims += (unsigned long long)dstep;
            if (g.pp) {
                // HNSW++: R and S keep every fresh vertex's observed distance
                // (exact at d = D, else (D/d) S_d); R keeps its ef smallest,
                // which a merge of all of them at once gives as well
                const int d = dstep;
                const float key_r = dec != 0 ? sdec : sdec * ((float)g.D / (float)d);
                const bool take_r = fresh && (!full0 || pless(key_r, v, rmax0, rid0));
                const int na = stage_sorted(take_r, key_r, v, ad, ai, lane);
                if (na) {
                    nR = warp_merge(rd, ri, rx, nR, ad, ai, na, nd, ni, nx, g.ef, lane);
                    float *tf = rd; rd = nd; nd = tf;
                    int *ti = ri; ri = ni; ni = ti;
                    ti = rx; rx = nx; nx = ti;
                }
            }
            __syncwarp();
        };
        // Start vertices: the n_ce entries of each of the query's n_entry
        // nearest clusters, 32 list positions per batch, tested like the
        // neighbours of one expansion (distinct; -1 skipped); vertex 0 when
        // no cluster has an entry.
        const int ns = g.n_entry * g.n_ce;
        for (int c0 = 0; c0 < ns + 32; c0 += 32) {
            const bool tail = c0 >= ns;         // the pass after the entries
            if (tail && nR > 0) break;
            int64_t e = -1;
            if (!tail) {
                const int k = c0 + lane;
                if (k < ns) e = g.entry[(int64_t)g.probes[q * g.n_entry + k / g.n_ce] * g.n_ce + k % g.n_ce];
            } else if (lane == 0) {
                e = 0;
            }
            bool fresh = false;
            if (e >= 0) {
                const unsigned bit = 1u << (e & 31);
                fresh = !(atomicOr(bm + (e >> 5), bit) & bit);
            }
            const unsigned fb = __ballot_sync(FULL, fresh);
            if (!fb) continue;
            if (fresh) vl[vcount + __popc(fb & below)] = (int32_t)e;
            vcount += __popc(fb);
            dco_batch((int)e, fresh);
        }
        for (int it = 0; it < g.max_iter; ++it) {
            int u = -1;
            for (int b0 = 0; b0 < nR; b0 += 32) {
                const int k = b0 + lane;
                const unsigned bb = __ballot_sync(FULL, k < nR && rx[k] == 0);
                if (bb) {
                    u = b0 + __ffs(bb) - 1;
                    break;
                }
            }
            if (u < 0) break;
            const int node = ri[u];
            __syncwarp();
            if (lane == 0) rx[u] = 1;
            // neighbours, one per lane, exact visited test
            int v = -1;
            if (lane < g.degree) v = g.nbr[(int64_t)node * g.degree + lane];
            bool fresh = false;
            if (v >= 0) {
                const unsigned bit = 1u << (v & 31);
                fresh = !(atomicOr(bm + (v >> 5), bit) & bit);
            }
            const unsigned fb = __ballot_sync(FULL, fresh);
            if (fresh) vl[vcount + __popc(fb & below)] = v;
            vcount += __popc(fb);
            dco_batch(v, fresh);
        }
        const float *od = g.pp ? kd : rd;
        const int *oi = g.pp ? ki : ri;
        const int no = g.pp ? n1 : nR;
        const bool cosine = g.metric == ADSX_COSINE;
        for (int k = lane; k < g.K; k += 32) {
            const bool has = k < no;
            g.out_ids[q * g.K + k] = has ? (int64_t)oi[k] : (int64_t)-1;
            // cosine similarity of unit vectors: 1 - d^2/2, largest first
            g.out_d2[q * g.K + k] = has ? (cosine ? fmaf(-0.5f, od[k], 1.f) : od[k])
                                        : (cosine ? -INFINITY : INFINITY);
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) dims += __shfl_xor_sync(FULL, dims, s);
        if (lane == 0 && g.out_dims) g.out_dims[q] = (int64_t)dims;
        // leave the bitmap all-zero for the next query
        __syncwarp();
        for (int k = lane; k < vcount; k += 32) bm[vl[k] >> 5] = 0u;
        __syncwarp();
    }
}

}  // namespace

size_t graph_search_smem(int Dp, int ef, int K, int nst)
{
    return graph_warp_bytes(Dp, ef, K, nst) * GW;
}

int graph_search_resident_warps(int Dp, int ef, int K, int nst, int nsm)
{
    const size_t smem = graph_search_smem(Dp, ef, K, nst);
    if (cudaFuncSetAttribute(graph_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, graph_search_kernel, GW * 32, smem) !=
        cudaSuccess)
        return 0;
    return nb * GW * nsm;
}

cudaError_t launch_knn_to_graph(const int64_t *knn, int64_t N, int64_t row0, int Kk, int degree,
                                int32_t *nbr, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    const int64_t blocks = (N + 255) / 256;
    knn_to_graph_kernel<<<(unsigned)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, s>>>(
        knn, N, row0, Kk, degree, nbr);
    return cudaGetLastError();
}

cudaError_t launch_vertex_map(const int64_t *off, int nlist, const int32_t *ids, int Dp,
                              int64_t *vbase, int32_t *vstride, cudaStream_t s)
{
    vertex_map_kernel<<<nlist < 152 * 16 ? nlist : 152 * 16, 256, 0, s>>>(off, nlist, ids, Dp, vbase,
                                                                          vstride);
    return cudaGetLastError();
}

cudaError_t launch_cluster_entries(const float *data, const int64_t *off, const int32_t *ids,
                                   const float *cents, int nlist, int Dp, int E, float *mind,
                                   int64_t *entry, cudaStream_t s)
{
    const int blocks = (nlist + 7) / 8;
    cluster_entry_kernel<<<blocks < 152 * 16 ? blocks : 152 * 16, 256, 0, s>>>(data, off, ids, cents,
                                                                               nlist, Dp, E, mind, entry);
    return cudaGetLastError();
}

cudaError_t launch_graph_search(const GraphArgs &g, cudaStream_t s)
{
    if (g.nq <= 0) return cudaSuccess;
    const size_t smem = graph_search_smem(g.Dp, g.ef, g.K, g.nst);
    cudaError_t e = cudaFuncSetAttribute(graph_search_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(g.qnext, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int blocks = (g.warps + GW - 1) / GW;
    graph_search_kernel<<<blocks, GW * 32, smem, s>>>(g);
    return cudaGetLastError();
}

}  // namespace adsx
