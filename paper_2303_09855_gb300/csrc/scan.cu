// scan.cu -- the IVF+ candidate scan: Algorithm 1 (ADSampling) as the DCO of
// every member of a query's probed clusters (Sec. 4), against the query's
// current K-th distance (Sec. 2.2.2), plus the fixed-threshold linear scan of
// the verification protocol (Sec. 6.2.5).
//
// ads_scan_kernel -- persistent: each 256-thread block repeatedly claims the
// next query from a global counter.  Per query, shared memory holds q', the
// probed clusters' CSR spans, a tile prefix (32 members per tile) and the
// query's top-K.  Each warp:
//   1. claims the next tile of 32 members (shared-memory counter), one member
//      per lane, and reads the first delta_d dims of all 32 members: 2 KB
//      coalesced runs per 16-dim block;
//   2. tests S_d > r^2 f(d) (squared Sec. 3.2 test, r^2 read live from shared
//      memory); a ballot compacts the survivors into the warp's ring of
//      pending candidates (member, cluster slot, blocks done, S);
//   3. whenever 32 candidates are pending, advances all 32 by one delta_d step
//      each (each lane its own candidate, whole 64-byte pieces), tests again
//      and re-queues survivors, so lanes stay busy after compaction;
//   4. candidates that reach d = D with S_D <= r^2 are inserted into the
//      block's top-K under a shared-memory lock (bounded spin); the K-th
//      distance becomes the new r^2 for every warp of the block.
// When tiles run out, each warp drains its ring.  The top-K is then
// bitonic-sorted by (distance, id) and written out.
#include <float.h>

#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr int RING = 64;                       // per-warp pending ring (power of 2)
constexpr unsigned LOCK_SPIN_LIMIT = 1u << 24;  // bounded spin on the top-K lock
constexpr unsigned FULL = 0xffffffffu;

struct Ctl {
    int q;
    int next_tile;
    int total_tiles;
    int lock;
    int count;
    int maxpos;
    int maxi;
    float maxd;
    float r2;
    unsigned long long dims;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemCarve {
    size_t qv, ftab, soff, sn, tpref, tkd, tki, pm, psb, pS, total;
    __host__ __device__ SmemCarve(int Dp, int nblk, int nprobe, int Kp)
    {
        size_t o = 0;
        qv = o;    o = align16(o + sizeof(float) * Dp);
        ftab = o;  o = align16(o + sizeof(float) * (nblk + 1));
        soff = o;  o = align16(o + sizeof(long long) * nprobe);
        sn = o;    o = align16(o + sizeof(int) * nprobe);
        tpref = o; o = align16(o + sizeof(int) * (nprobe + 1));
        tkd = o;   o = align16(o + sizeof(float) * Kp);
        tki = o;   o = align16(o + sizeof(int) * Kp);
        pm = o;    o = align16(o + sizeof(int) * WARPS * RING);
        psb = o;   o = align16(o + sizeof(int) * WARPS * RING);
        pS = o;    o = align16(o + sizeof(float) * WARPS * RING);
        total = o;
    }
};

__device__ __forceinline__ bool pair_less(float d1, int i1, float d2, int i2)
{
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

// Maximum (by (distance, id)) of the K entries of the top-K, warp-wide.
__device__ __forceinline__ void warp_max(const float *tkd, const int *tki, int K, int lane,
                                         float &md, int &mi, int &mp)
{
    float bd = -1.f;
    int bi = -1, bp = -1;
    for (int k = lane; k < K; k += 32) {
        float d = tkd[k];
        int i = tki[k];
        if (bp < 0 || pair_less(bd, bi, d, i)) {
            bd = d;
            bi = i;
            bp = k;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float od = __shfl_xor_sync(FULL, bd, o);
        int oi = __shfl_xor_sync(FULL, bi, o);
        int op = __shfl_xor_sync(FULL, bp, o);
        bool take = (bp < 0) || (op >= 0 && pair_less(bd, bi, od, oi));
        if (take) {
            bd = od;
            bi = oi;
            bp = op;
        }
    }
    md = bd;
    mi = bi;
    mp = bp;
}

struct WarpCtx {
    const ScanArgs *a;
    Ctl *ctl;
    const float *qv;
    const float *ftab;
    const long long *soff;
    const int *sn;
    float *tkd;
    int *tki;
    int *pm;
    int *psb;
    float *pS;
    int lane;
    int head, cnt;                // ring state (warp-uniform)
    unsigned long long dims;      // per-lane dims sampled
};

// Inserts the lanes whose candidate reached d = D with S_D <= r^2 into the
// block's top-K (Sec. 2.2.2: the KNN set keeps the K smallest (dist, id)).
__device__ __forceinline__ void try_insert(WarpCtx &w, bool fin, float S, int slot, int m)
{
    volatile Ctl *vc = w.ctl;
    const float r2 = vc->r2;
    const bool want = fin && (S <= r2);
    unsigned mask = __ballot_sync(FULL, want);
    if (!mask) return;
    int id = 0;
    if (want) id = w.a->ids[w.soff[slot] + m];
    bool ok = true;
    if (w.lane == 0) {
        unsigned spins = 0;
        while (atomicCAS(&w.ctl->lock, 0, 1) != 0) {
            if (++spins > LOCK_SPIN_LIMIT) {
                ok = false;
                break;
            }
            __nanosleep(32);
        }
    }
    ok = __shfl_sync(FULL, ok, 0);
    if (!ok) {
        if (w.lane == 0) atomicOr(w.a->err, ERR_LOCK_TIMEOUT);
        return;
    }
    __threadfence_block();
    const int K = w.a->K;
    int count = vc->count, maxpos = vc->maxpos, maxi = vc->maxi;
    float maxd = vc->maxd;
    volatile float *tkd = w.tkd;
    volatile int *tki = w.tki;
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const float s = __shfl_sync(FULL, S, src);
        const int i = __shfl_sync(FULL, id, src);
        if (count < K) {
            if (w.lane == 0) {
                tkd[count] = s;
                tki[count] = i;
            }
            ++count;
            if (count == K) {
                __syncwarp();
                warp_max(w.tkd, w.tki, K, w.lane, maxd, maxi, maxpos);
            }
        } else if (pair_less(s, i, maxd, maxi)) {
            if (w.lane == 0) {
                tkd[maxpos] = s;
                tki[maxpos] = i;
            }
            __syncwarp();
            warp_max(w.tkd, w.tki, K, w.lane, maxd, maxi, maxpos);
        }
    }
    if (w.lane == 0) {
        vc->count = count;
        vc->maxpos = maxpos;
        vc->maxi = maxi;
        vc->maxd = maxd;
        vc->r2 = (count == K) ? maxd : INFINITY;
        __threadfence_block();
        atomicExch(&w.ctl->lock, 0);
    }
    __syncwarp();
}

// After a candidate has `blk` blocks accumulated in S: exact compare at d = D
// (Case 3), else the hypothesis test (Case 1 reject / Case 2 re-queue).
__device__ __forceinline__ void after_step(WarpCtx &w, bool valid, float S, int blk, int slot,
                                           int m)
{
    const ScanArgs &a = *w.a;
    const bool fin = valid && blk >= a.nblk;
    bool surv = false;
    if (valid && !fin) {
        const float r2 = ((volatile Ctl *)w.ctl)->r2;
        const bool rej = a.test_on && (S > r2 * w.ftab[blk]);
        if (rej) {
            int d = blk * BLK;
            w.dims += (unsigned long long)(d < a.D ? d : a.D);
        } else {
            surv = true;
        }
    }
    if (fin) w.dims += (unsigned long long)a.D;
    const unsigned sm = __ballot_sync(FULL, surv);
    if (surv) {
        const int pos = __popc(sm & ((1u << w.lane) - 1u));
        const int idx = (w.head + w.cnt + pos) & (RING - 1);
        w.pm[idx] = m;
        w.psb[idx] = (slot << 8) | blk;
        w.pS[idx] = S;
    }
    w.cnt += __popc(sm);
    __syncwarp();
    try_insert(w, fin, S, slot, m);
}

// Advances up to 32 pending candidates by one delta_d step each.
__device__ __forceinline__ void process_pending(WarpCtx &w, int nb)
{
    const ScanArgs &a = *w.a;
    const bool valid = w.lane < nb;
    int m = 0, sb = 0;
    float S = 0.f;
    if (valid) {
        const int idx = (w.head + w.lane) & (RING - 1);
        m = w.pm[idx];
        sb = w.psb[idx];
        S = w.pS[idx];
    }
    __syncwarp();
    w.head = (w.head + nb) & (RING - 1);
    w.cnt -= nb;
    const int slot = sb >> 8;
    int blk = sb & 255;
    if (valid) {
        const int64_t n = w.sn[slot];
        const float *base = a.data + w.soff[slot] * (int64_t)a.Dp;
        int e = blk + a.db;
        if (e > a.nblk) e = a.nblk;
        S = accum_range_f32(base, n, m, blk, e, w.qv, S);
        blk = e;
    }
    after_step(w, valid, S, blk, slot, m);
}

__global__ void __launch_bounds__(THREADS) ads_scan_kernel(ScanArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ Ctl ctl;
    const SmemCarve sc(a.Dp, a.nblk, a.nprobe, a.Kp);
    float *qv = reinterpret_cast<float *>(smraw + sc.qv);
    float *ftab = reinterpret_cast<float *>(smraw + sc.ftab);
    long long *soff = reinterpret_cast<long long *>(smraw + sc.soff);
    int *sn = reinterpret_cast<int *>(smraw + sc.sn);
    int *tpref = reinterpret_cast<int *>(smraw + sc.tpref);
    float *tkd = reinterpret_cast<float *>(smraw + sc.tkd);
    int *tki = reinterpret_cast<int *>(smraw + sc.tki);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int b = tid; b <= a.nblk; b += THREADS)
        ftab[b] = (b == 0) ? 0.f : test_factor(b, a.D, a.eps0);

    for (;;) {
        if (tid == 0) ctl.q = (int)atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const int64_t q = ctl.q;
        if (q >= a.nq) break;

        for (int i = tid; i < a.Dp; i += THREADS) qv[i] = a.qrot[q * a.Dp + i];
        for (int i = tid; i < a.nprobe; i += THREADS) {
            const int c = a.probes[q * a.nprobe + i];
            const int64_t o = a.off[c];
            soff[i] = o;
            sn[i] = (int)(a.off[c + 1] - o);
        }
        if (tid == 0) {
            ctl.next_tile = 0;
            ctl.lock = 0;
            ctl.count = 0;
            ctl.maxpos = 0;
            ctl.maxi = 0;
            ctl.maxd = INFINITY;
            ctl.r2 = INFINITY;
            ctl.dims = 0ull;
        }
        __syncthreads();
        if (warp == 0) {
            int run = 0;
            for (int i0 = 0; i0 < a.nprobe; i0 += 32) {
                const int i = i0 + lane;
                const int t = (i < a.nprobe) ? (sn[i] + 31) / 32 : 0;
                int incl = t;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                if (i < a.nprobe) tpref[i] = run + incl - t;
                run += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) {
                tpref[a.nprobe] = run;
                ctl.total_tiles = run;
            }
        }
        __syncthreads();

        WarpCtx w;
        w.a = &a;
        w.ctl = &ctl;
        w.qv = qv;
        w.ftab = ftab;
        w.soff = soff;
        w.sn = sn;
        w.tkd = tkd;
        w.tki = tki;
        w.pm = reinterpret_cast<int *>(smraw + sc.pm) + warp * RING;
        w.psb = reinterpret_cast<int *>(smraw + sc.psb) + warp * RING;
        w.pS = reinterpret_cast<float *>(smraw + sc.pS) + warp * RING;
        w.lane = lane;
        w.head = 0;
        w.cnt = 0;
        w.dims = 0ull;
        const int total = ctl.total_tiles;
        const int nb0 = a.db < a.nblk ? a.db : a.nblk;

        for (;;) {
            int t = 0;
            if (lane == 0) t = atomicAdd(&ctl.next_tile, 1);
            t = __shfl_sync(FULL, t, 0);
            if (t >= total) break;
            int lo = 0, hi = a.nprobe - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tpref[mid] <= t) lo = mid; else hi = mid - 1;
            }
            const int slot = lo;
            const int n = sn[slot];
            const int m = (t - tpref[slot]) * 32 + lane;
            const bool valid = m < n;
            float S = 0.f;
            if (valid)
                S = accum_range_f32(a.data + soff[slot] * (int64_t)a.Dp, n, m, 0, nb0, qv, 0.f);
            after_step(w, valid, S, nb0, slot, m);
            while (w.cnt >= 32) process_pending(w, 32);
        }
        while (w.cnt > 0) process_pending(w, w.cnt < 32 ? w.cnt : 32);

        unsigned long long wd = w.dims;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wd += __shfl_xor_sync(FULL, wd, o);
        if (lane == 0) atomicAdd(&ctl.dims, wd);
        __syncthreads();

        // (distance, id)-sort of the top-K, padded with (+inf, INT_MAX).
        const int count = ctl.count;
        for (int k = count + tid; k < a.Kp; k += THREADS) {
            tkd[k] = INFINITY;
            tki[k] = 0x7fffffff;
        }
        __syncthreads();
        for (int size = 2; size <= a.Kp; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < a.Kp; i += THREADS) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const float di = tkd[i], dj = tkd[j];
                        const int ii = tki[i], ij = tki[j];
                        const bool up = (i & size) == 0;
                        if (pair_less(dj, ij, di, ii) == up) {
                            tkd[i] = dj;
                            tki[i] = ij;
                            tkd[j] = di;
                            tki[j] = ii;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int k = tid; k < a.K; k += THREADS) {
            const bool has = k < count;
            a.out_ids[q * a.K + k] = has ? (int64_t)tki[k] : (int64_t)-1;
            a.out_d2[q * a.K + k] = has ? tkd[k] : INFINITY;
        }
        if (tid == 0 && a.out_dims) a.out_dims[q] = (int64_t)ctl.dims;
        __syncthreads();
    }
}

// Verification protocol (Sec. 6.2.5): every (query, indexed vector) pair,
// fixed threshold r2[q].  One warp per 32-member tile of one cluster, one
// lane per member; the same block accumulation and test as the search scan.
__global__ void __launch_bounds__(THREADS) dco_fixed_r_kernel(FixedRArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    float *qv = reinterpret_cast<float *>(smraw);
    float *ftab = qv + a.Dp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.y;
    for (int i = tid; i < a.Dp; i += THREADS) qv[i] = a.qrot[q * a.Dp + i];
    for (int b = tid; b <= a.nblk; b += THREADS)
        ftab[b] = (b == 0) ? 0.f : test_factor(b, a.D, a.eps0);
    __syncthreads();
    const int t = blockIdx.x * WARPS + warp;
    if (t >= a.total_tiles) return;
    int lo = 0, hi = a.nlist - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int c = lo;
    const int64_t o = a.off[c];
    const int64_t n = a.off[c + 1] - o;
    const int64_t m = (int64_t)(t - a.tile_off[c]) * 32 + lane;
    if (m >= n) return;
    const float r2 = a.r2[q];
    const float *base = a.data + o * a.Dp;
    float S = 0.f;
    int blk = 0;
    uint8_t dec = 0;
    int dims = 0;
    for (;;) {
        int e = blk + a.db;
        if (e > a.nblk) e = a.nblk;
        S = accum_range_f32(base, n, m, blk, e, qv, S);
        blk = e;
        if (blk >= a.nblk) {
            dec = (S <= r2) ? 1 : 2;
            dims = a.D;
            break;
        }
        if (a.test_on && S > r2 * ftab[blk]) {
            dec = 0;
            dims = blk * BLK < a.D ? blk * BLK : a.D;
            break;
        }
    }
    const int64_t id = a.ids[o + m];
    a.decisions[q * a.N + id] = dec;
    if (a.dims) a.dims[q * a.N + id] = dims;
}

}  // namespace

size_t scan_smem_bytes(const ScanArgs &a)
{
    return SmemCarve(a.Dp, a.nblk, a.nprobe, a.Kp).total;
}

int ads_scan_grid(const ScanArgs &a, int device)
{
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    size_t smem = scan_smem_bytes(a);
    cudaFuncSetAttribute(ads_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ads_scan_kernel, THREADS, smem);
    if (per < 1) per = 1;
    int64_t g = (int64_t)nsm * per;
    if (g > a.nq) g = a.nq;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_ads_scan(const ScanArgs &a, int grid, cudaStream_t s)
{
    if (a.nq <= 0) return cudaSuccess;
    size_t smem = scan_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(ads_scan_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ads_scan_kernel<<<grid, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dco_fixed_r(const FixedRArgs &a, cudaStream_t s)
{
    if (a.nq <= 0 || a.total_tiles <= 0) return cudaSuccess;
    size_t smem = sizeof(float) * (a.Dp + a.nblk + 1);
    dim3 grid((unsigned)((a.total_tiles + WARPS - 1) / WARPS), (unsigned)a.nq);
    if (a.nq > 65535) return cudaErrorInvalidValue;
    dco_fixed_r_kernel<<<grid, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace adsx
