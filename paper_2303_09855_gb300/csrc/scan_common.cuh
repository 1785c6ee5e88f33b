// scan_common.cuh -- the per-candidate arithmetic shared by the two scan
// schedules of libadsx.so (internal): ads_scan_kernel (query-major, scan.cu)
// and cm_scan_kernel (cluster-major, cmscan.cu).  Both accumulate a
// candidate's partial distance S_d (Algorithm 1) with exactly these
// functions, in the same order, so both give the same FP32 value for every
// (query, candidate, step) and hence the same decisions at a given r.
#pragma once

#include "adsx_internal.cuh"

namespace adsx {
namespace scan {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ bool pair_less(float d1, int i1, float d2, int i2)
{
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

// Order-preserving map of a float key to unsigned (inner-product keys are
// negative), for the atomicMin that shares r between the splits of a query;
// 0xffffffff (the cleared value) means "no bound yet".
__device__ __forceinline__ unsigned key_to_ord(float k)
{
    const unsigned u = __float_as_uint(k);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_to_key(unsigned m)
{
    return __uint_as_float((m & 0x80000000u) ? (m & 0x7fffffffu) : ~m);
}

// The value returned for a key: L2 the squared distance; cosine the
// similarity 1 - ||x^ - q^||^2 / 2; inner product <o,q> (key = -<o,q>).
// Empty slots: +inf for L2, -inf for similarities.
__device__ __forceinline__ float out_value(int metric, float key, bool has)
{
    if (metric == ADSX_L2) return has ? key : INFINITY;
    if (!has) return -INFINITY;
    return metric == ADSX_COSINE ? fmaf(-0.5f, key, 1.f) : -key;
}

// ---- several lanes per candidate.  One 16-dim block of a candidate is 64
// bytes (FP32) or 32 bytes (16-bit); NL = 4 or 2 lanes split it into 16-byte
// pieces.  The warp is 32/NL groups of NL lanes, and lane l (group g = l / NL,
// piece j = l % NL) works on the NL candidates g + (32/NL) k, k < NL, of a set
// of 32.  One load instruction of the warp thus reads whole blocks of 32/NL
// candidates -- a single contiguous 512-byte run when they are consecutive
// members -- instead of 16-byte slices of 32 candidates spread over 16 or more
// cache lines.  Each lane keeps a partial sum per candidate (its piece, two
// FP32 chains: even and odd dims); group_sum then combines the NL pieces so
// that lane l holds the complete sum of candidate own_slot(l).
template <typename T> struct Split {           // 16-bit: 2 lanes x 8 values
    static constexpr int NL = 2;
    typedef uint4 V;
};
template <> struct Split<float> {              // FP32: 4 lanes x 4 values
    static constexpr int NL = 4;
    typedef float4 V;
};

__device__ __forceinline__ float4 ld_piece(const float *p)
{
    return __ldg(reinterpret_cast<const float4 *>(p));
}
template <typename H>
__device__ __forceinline__ uint4 ld_piece(const H *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ void zero_piece(float4 &v) { v = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void zero_piece(uint4 &v) { v = make_uint4(0u, 0u, 0u, 0u); }

// The query values matching a lane's piece (4 or 8 floats, shared memory).
template <int NL> struct QPiece;
template <> struct QPiece<4> { float4 a; };
template <> struct QPiece<2> { float4 a, b; };
template <int NL>
__device__ __forceinline__ QPiece<NL> ld_qpiece(const float *q)
{
    QPiece<NL> r;
    r.a = *reinterpret_cast<const float4 *>(q);
    if constexpr (NL == 2) r.b = *reinterpret_cast<const float4 *>(q + 4);
    return r;
}

// S + (x - q)^2 over two consecutive dims (x0, x1) of a piece: the even dim
// into S.x, the odd one into S.y, each rounded as the scalar
// t = x - q; S = fma(t, t, S) would be.  With ADSX_F32X2 (the default) one
// packed f32x2 subtract and one packed f32x2 FMA (sm_100+) do both lanes of
// the pair: the same IEEE round-to-nearest operation per element, so the
// same values, in half the instructions.
#ifndef ADSX_F32X2
#define ADSX_F32X2 1
#endif
__device__ __forceinline__ float2 add_pair(float x0, float x1, float q0, float q1, float2 S)
{
#if ADSX_F32X2
    asm("{\n .reg .b64 xv, qv, tv, sv;\n"
        " mov.b64 xv, {%2, %3};\n mov.b64 qv, {%4, %5};\n mov.b64 sv, {%0, %1};\n"
        " sub.rn.f32x2 tv, xv, qv;\n fma.rn.f32x2 sv, tv, tv, sv;\n"
        " mov.b64 {%0, %1}, sv;\n}"
        : "+f"(S.x), "+f"(S.y)
        : "f"(x0), "f"(x1), "f"(q0), "f"(q1));
#else
    float t;
    t = x0 - q0; S.x = fmaf(t, t, S.x);
    t = x1 - q1; S.y = fmaf(t, t, S.y);
#endif
    return S;
}

// S + (x - q)^2 over the piece, even dims into S.x and odd dims into S.y
// (dims in ascending order within each chain).
__device__ __forceinline__ float2 add_piece(float4 x, const QPiece<4> &q, float2 S, float)
{
    S = add_pair(x.x, x.y, q.a.x, q.a.y, S);
    S = add_pair(x.z, x.w, q.a.z, q.a.w, S);
    return S;
}
template <typename H>
__device__ __forceinline__ float2 add_piece(uint4 x, const QPiece<2> &q, float2 S, H h)
{
    float v0, v1;
    unpack2(x.x, v0, v1, h);
    S = add_pair(v0, v1, q.a.x, q.a.y, S);
    unpack2(x.y, v0, v1, h);
    S = add_pair(v0, v1, q.a.z, q.a.w, S);
    unpack2(x.z, v0, v1, h);
    S = add_pair(v0, v1, q.b.x, q.b.y, S);
    unpack2(x.w, v0, v1, h);
    S = add_pair(v0, v1, q.b.z, q.b.w, S);
    return S;
}

// A piece held unpacked in FP32 registers (16-bit storage: its 8 values;
// FP32: the piece itself), for a piece used against many queries: the
// conversion is exact, and add_piece_u adds in add_piece's order, so the
// sums are the same.
template <typename T> struct Unpacked {
    struct U { float4 a, b; };
};
template <> struct Unpacked<float> {
    typedef float4 U;
};
__device__ __forceinline__ float4 unpack_piece(float4 x, float) { return x; }
template <typename H>
__device__ __forceinline__ typename Unpacked<H>::U unpack_piece(uint4 x, H h)
{
    typename Unpacked<H>::U u;
    unpack2(x.x, u.a.x, u.a.y, h);
    unpack2(x.y, u.a.z, u.a.w, h);
    unpack2(x.z, u.b.x, u.b.y, h);
    unpack2(x.w, u.b.z, u.b.w, h);
    return u;
}
__device__ __forceinline__ float2 add_piece_u(float4 x, const QPiece<4> &q, float2 S)
{
    return add_piece(x, q, S, 0.f);
}
template <typename U>
__device__ __forceinline__ float2 add_piece_u(const U &x, const QPiece<2> &q, float2 S)
{
    S = add_pair(x.a.x, x.a.y, q.a.x, q.a.y, S);
    S = add_pair(x.a.z, x.a.w, q.a.z, q.a.w, S);
    S = add_pair(x.b.x, x.b.y, q.b.x, q.b.y, S);
    S = add_pair(x.b.z, x.b.w, q.b.z, q.b.w, S);
    return S;
}

// The candidate (of the set of 32) whose complete sum lane l receives from
// group_sum, and the lane that receives candidate g + (32/NL) k.
template <int NL>
__device__ __forceinline__ int own_slot(int lane)
{
    if constexpr (NL == 4) return (lane >> 2) + 8 * (2 * (lane & 1) + ((lane >> 1) & 1));
    else return (lane >> 1) + 16 * (lane & 1);
}
template <int NL>
__device__ __forceinline__ int owner_lane(int g, int k)
{
    if constexpr (NL == 4) return 4 * g + (k >> 1) + 2 * (k & 1);
    else return 2 * g + k;
}

// Transpose-and-add over the NL lanes of a group: lane l enters with the
// partial sums p[k] of its piece for candidates g + (32/NL) k and leaves with
// the sum over all pieces of candidate own_slot(l).  With NL = 4, lanes l, l^1
// split the four candidates into {0, 1} and {2, 3}, then lanes l, l^2 split
// each pair; with NL = 2, lanes l, l^1 split {0, 1}.
template <int NL>
__device__ __forceinline__ float group_sum(const float2 (&pp)[NL], int lane)
{
    float p[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) p[k] = pp[k].x + pp[k].y;
    const bool hi1 = lane & 1;
    if constexpr (NL == 4) {
        const bool hi2 = lane & 2;
        const float u0 = (hi1 ? p[2] : p[0]) + __shfl_xor_sync(FULL, hi1 ? p[0] : p[2], 1);
        const float u1 = (hi1 ? p[3] : p[1]) + __shfl_xor_sync(FULL, hi1 ? p[1] : p[3], 1);
        return (hi2 ? u1 : u0) + __shfl_xor_sync(FULL, hi2 ? u0 : u1, 2);
    } else {
        return (hi1 ? p[1] : p[0]) + __shfl_xor_sync(FULL, hi1 ? p[0] : p[1], 1);
    }
}

// 16-bit storage: the exact FP32 distance of the candidate at CSR row `pos`
// for every lane with `need`, recomputed from the FP32 row copy one candidate
// at a time by the whole warp (each lane a 4-dim slice, then a butterfly sum
// whose result is the same on all lanes).  qv: each lane's query (Dp floats,
// shared or global memory; lanes may hold different queries).
__device__ __forceinline__ float recheck_rows(const float *__restrict__ rows32, int Dp,
                                              const float *qv, bool need, int pos, float S,
                                              int lane)
{
    unsigned mask = __ballot_sync(FULL, need);
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const int p = __shfl_sync(FULL, pos, src);
        const float *qs = reinterpret_cast<const float *>(__shfl_sync(
            FULL, (unsigned long long)reinterpret_cast<uintptr_t>(qv), src));
        const float *row = rows32 + (int64_t)p * Dp;
        float part = 0.f;
        for (int j = lane * 4; j < Dp; j += 128) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(row + j));
            const float4 q = *reinterpret_cast<const float4 *>(qs + j);
            float t;
            t = x.x - q.x; part = fmaf(t, t, part);
            t = x.y - q.y; part = fmaf(t, t, part);
            t = x.z - q.z; part = fmaf(t, t, part);
            t = x.w - q.w; part = fmaf(t, t, part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
        if (lane == src) S = part;
    }
    return S;
}

}  // namespace scan
}  // namespace adsx
