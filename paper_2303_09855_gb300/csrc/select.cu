// select.cu -- top-nprobe cluster selection per query (Sec. 2.2.2: probe the
// N_probe clusters whose centroids are nearest to the query), ordered by
// (squared centroid distance, cluster id).
//
// One 256-thread block per query row.  The row's distances are turned into
// order-preserving 32-bit keys (bit patterns of non-negative floats) in shared
// memory; a 4-pass, 8-bit radix select finds the exact key T of the
// nprobe-th smallest distance and how many keys equal to T are still needed;
// keys below T are gathered, keys equal to T are taken in ascending cluster id
// by one warp (ballot order), and the nprobe winners are bitonic-sorted as
// 64-bit (key, id) words.
#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int ST = 256;

__device__ __forceinline__ unsigned dist_key(float v)
{
    // non-negative floats order like their bit patterns; -0, tiny negative
    // rounding residue and NaN are mapped to 0 / +inf.
    if (!(v > 0.f)) return (v != v) ? 0x7f800000u : 0u;
    return __float_as_uint(v);
}

__global__ void __launch_bounds__(ST) select_nprobe_kernel(const float *__restrict__ dist,
                                                           int64_t nq, int nlist, int pstride,
                                                           int P2, int32_t *__restrict__ probes,
                                                           float *__restrict__ pd2,
                                                           const int32_t *__restrict__ nprobe_q)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *sel = reinterpret_cast<unsigned long long *>(smraw);   // P2
    unsigned *key = reinterpret_cast<unsigned *>(sel + P2);                    // nlist
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_remaining, s_nsel;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
        int nprobe = pstride;
        if (nprobe_q) {                     // per-query count, clamped to [1, pstride]
            nprobe = nprobe_q[q];
            nprobe = nprobe < 1 ? 1 : (nprobe > pstride ? pstride : nprobe);
        }
        const float *row = dist + q * nlist;
        for (int i = tid; i < nlist; i += ST) key[i] = dist_key(row[i]);
        if (tid == 0) {
            s_prefix = 0;
            s_remaining = (unsigned)nprobe;
        }
        __syncthreads();
        unsigned mask = 0;
        for (int shift = 24; shift >= 0; shift -= 8) {
            hist[tid] = 0;
            __syncthreads();
            const unsigned prefix = s_prefix;
            // Keys that still match the prefix vote for their digit; lanes of a
            // warp with the same digit are merged (match.any) into one atomic,
            // since most keys share the high digits of the float's exponent.
            for (int i0 = warp * 32; i0 < nlist; i0 += ST) {
                const int i = i0 + lane;
                unsigned bin = 256u;                    // no vote
                if (i < nlist) {
                    const unsigned u = key[i];
                    if ((u & mask) == prefix) bin = (u >> shift) & 255u;
                }
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                if (bin < 256u && lane == __ffs(peers) - 1)
                    atomicAdd(&hist[bin], (unsigned)__popc(peers));
            }
            __syncthreads();
            if (warp == 0) {
                // warp-wide search of the bin holding the rem-th key: each lane
                // owns 8 consecutive bins, a shuffle scan gives the counts before
                // them, and the one lane whose range crosses rem finds the bin.
                const unsigned rem = s_remaining;
                unsigned h[8], own = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    h[j] = hist[lane * 8 + j];
                    own += h[j];
                }
                unsigned incl = own;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                unsigned cum = incl - own;
                if (cum < rem && incl >= rem) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (cum + h[j] >= rem) {
                            s_prefix = prefix | ((unsigned)(lane * 8 + j) << shift);
                            s_remaining = rem - cum;
                            break;
                        }
                        cum += h[j];
                    }
                }
            }
            mask |= 255u << shift;
            __syncthreads();
        }
        const unsigned T = s_prefix;
        const unsigned need_eq = s_remaining;
        if (tid == 0) s_nsel = 0;
        __syncthreads();
        for (int i = tid; i < nlist; i += ST) {
            unsigned u = key[i];
            if (u < T) {
                unsigned p = atomicAdd(&s_nsel, 1u);
                sel[p] = ((unsigned long long)u << 32) | (unsigned)i;
            }
        }
        __syncthreads();
        if (warp == 0) {
            const unsigned base = s_nsel;
            unsigned taken = 0;
            for (int i0 = 0; i0 < nlist && taken < need_eq; i0 += 32) {
                int i = i0 + lane;
                bool eq = (i < nlist) && key[i] == T;
                unsigned b = __ballot_sync(0xffffffffu, eq);
                unsigned r = __popc(b & ((1u << lane) - 1u));
                if (eq && taken + r < need_eq)
                    sel[base + taken + r] = ((unsigned long long)T << 32) | (unsigned)i;
                taken += __popc(b);
            }
        }
        __syncthreads();
        for (int i = nprobe + tid; i < P2; i += ST) sel[i] = ~0ull;
        __syncthreads();
        for (int size = 2; size <= P2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < P2; i += ST) {
                    int j = i ^ stride;
                    if (j > i) {
                        unsigned long long a = sel[i], b = sel[j];
                        bool up = (i & size) == 0;
                        if ((a > b) == up) {
                            sel[i] = b;
                            sel[j] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int p = tid; p < nprobe; p += ST) {
            unsigned long long v = sel[p];
            probes[q * pstride + p] = (int32_t)(v & 0xffffffffu);
            if (pd2) pd2[q * pstride + p] = __uint_as_float((unsigned)(v >> 32));
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_select_nprobe(const float *dist, int64_t nq, int nlist, int nprobe,
                                 int32_t *probes, float *probe_d2, cudaStream_t s,
                                 const int32_t *nprobe_q)
{
    if (nq <= 0) return cudaSuccess;
    int P2 = 1;
    while (P2 < nprobe) P2 <<= 1;
    size_t smem = (size_t)P2 * 8 + (size_t)nlist * 4;
    cudaError_t e = cudaFuncSetAttribute(select_nprobe_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = nq < 152 * 8 ? nq : 152 * 8;
    select_nprobe_kernel<<<(unsigned)grid, ST, smem, s>>>(dist, nq, nlist, nprobe, P2, probes,
                                                          probe_d2, nprobe_q);
    return cudaGetLastError();
}

}  // namespace adsx
