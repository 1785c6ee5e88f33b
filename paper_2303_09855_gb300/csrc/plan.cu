// plan.cu -- work plan of the batched form: queries with their own K and
// nprobe in one persistent scan launch.
//
// One block of 1024 threads:
//   1. validates every K_q in [1, maxK] and nprobe_q in [1, maxP] (out-of-range
//      values set ERR_BATCH_ARGS in the index's error word and are clamped);
//   2. picks the splits S_q of each query: enough items to fill the GPU
//      (target_items / nq), at least one item per 64 probe slots for long
//      queries, capped by nprobe_q * (N / nlist) / (2 K_q) (each split should
//      expect 2K candidates: it prunes only once it holds K exact
//      distances), 16 and 16384 / next_pow2(K_q) (the finalize merge buffer);
//   3. orders the queries longest-first (counting sort on nprobe_q) so the
//      longest items start first and short ones fill the tail;
//   4. lays out the items of each query contiguously in that order
//      (x = query, y = split << 16 | S_q) and records each query's first item;
//   5. if the caller gave no output offsets, writes the prefix sums of K_q.
#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int PT = 1024;

__device__ __forceinline__ int splits_of(int K, int np, int64_t nq, int target,
                                         int64_t members_per_list)
{
    int Kp = 1;
    while (Kp < K) Kp <<= 1;
    int64_t S = (target + nq - 1) / nq;
    const int by_len = (np + 63) / 64;
    if (S < by_len) S = by_len;
    const int64_t by_cand = (int64_t)np * members_per_list / (2 * (int64_t)K);
    if (S > by_cand) S = by_cand;
    if (S > 16) S = 16;
    const int cap = 16384 / Kp;
    if (S > cap) S = cap;
    return S < 1 ? 1 : (int)S;
}

// Exclusive block-wide prefix sum of v over the block (1024 threads); returns
// this thread's prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *warp_tot, int64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;          // inclusive over warps
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? warp_tot[warp - 1] : 0) + x - v;
    *total = warp_tot[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(PT) plan_batched_kernel(
    const int32_t *__restrict__ Kq, const int32_t *__restrict__ npq, int64_t nq, int maxK, int maxP,
    int target, int64_t members_per_list, int2 *__restrict__ items,
    int32_t *__restrict__ item_first,
    int32_t *__restrict__ n_items, int32_t *__restrict__ qperm,
    const int64_t *__restrict__ out_off_in, int64_t *__restrict__ out_off, unsigned *err)
{
    extern __shared__ int hist[];            // maxP + 2 bins
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t s_run;
    const int tid = threadIdx.x;
    bool bad = false;
    // 1. histogram of nprobe_q (validated, clamped)
    for (int b = tid; b < maxP + 2; b += PT) hist[b] = 0;
    __syncthreads();
    for (int64_t q = tid; q < nq; q += PT) {
        int np = npq[q], K = Kq[q];
        if (np < 1 || np > maxP || K < 1 || K > maxK) bad = true;
        np = np < 1 ? 1 : (np > maxP ? maxP : np);
        atomicAdd(&hist[np], 1);
    }
    __syncthreads();
    // 2. exclusive start of each bin, largest nprobe first (one thread: <= 1025 bins)
    if (tid == 0) {
        int run = 0;
        for (int b = maxP; b >= 1; --b) {
            const int h = hist[b];
            hist[b] = run;
            run += h;
        }
    }
    __syncthreads();
    // 3. placement by bin (order inside a bin is arbitrary: a query's result
    //    does not depend on when its items run)
    for (int64_t q = tid; q < nq; q += PT) {
        int np = npq[q];
        np = np < 1 ? 1 : (np > maxP ? maxP : np);
        qperm[atomicAdd(&hist[np], 1)] = (int32_t)q;
    }
    __syncthreads();
    // 4. items in qperm order
    if (tid == 0) s_run = 0;
    __syncthreads();
    for (int64_t i0 = 0; i0 < nq; i0 += PT) {
        const int64_t i = i0 + tid;
        int S = 0, q = 0;
        if (i < nq) {
            q = qperm[i];
            int np = npq[q], K = Kq[q];
            np = np < 1 ? 1 : (np > maxP ? maxP : np);
            K = K < 1 ? 1 : (K > maxK ? maxK : K);
            S = splits_of(K, np, nq, target, members_per_list);
        }
        int64_t total;
        const int64_t before = block_excl_scan(S, warp_tot, &total);
        const int64_t first = s_run + before;
        if (i < nq) {
            item_first[q] = (int32_t)first;
            for (int s = 0; s < S; ++s) items[first + s] = make_int2(q, (s << 16) | S);
        }
        __syncthreads();
        if (tid == 0) s_run += total;
        __syncthreads();
    }
    if (tid == 0) *n_items = (int32_t)s_run;
    // 5. output offsets
    if (out_off) {
        if (tid == 0) s_run = 0;
        __syncthreads();
        for (int64_t q0 = 0; q0 < nq; q0 += PT) {
            const int64_t q = q0 + tid;
            int K = 0;
            if (q < nq) {
                K = Kq[q];
                K = K < 1 ? 1 : (K > maxK ? maxK : K);
            }
            int64_t total;
            const int64_t before = block_excl_scan(K, warp_tot, &total);
            if (q < nq) out_off[q] = out_off_in ? out_off_in[q] : s_run + before;
            __syncthreads();
            if (tid == 0) s_run += total;
            __syncthreads();
        }
    }
    if (bad) atomicOr(err, ERR_BATCH_ARGS);
}

}  // namespace

cudaError_t launch_plan_batched(const int32_t *Kq, const int32_t *nprobe_q, int64_t nq,
                                int maxK, int maxP, int target_items, int64_t members_per_list,
                                int2 *items, int32_t *item_first, int32_t *n_items,
                                int32_t *qperm, const int64_t *out_off_in, int64_t *out_off,
                                unsigned *err, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    size_t smem = sizeof(int) * (size_t)(maxP + 2);
    plan_batched_kernel<<<1, PT, smem, s>>>(Kq, nprobe_q, nq, maxK, maxP, target_items,
                                            members_per_list, items,
                                            item_first, n_items, qperm, out_off_in, out_off, err);
    return cudaGetLastError();
}

}  // namespace adsx
