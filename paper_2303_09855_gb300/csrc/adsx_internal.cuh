// adsx_internal.cuh -- internal declarations of libadsx.so (not installed).
//
// Device data layout of an index (Sec. 5.2 IVF++ generalised):
//   rotated vectors y = P x are stored per cluster (CSR order, members of a
//   cluster in ascending id), and inside a cluster "dimension-block major":
//   the 16 dims [16b, 16b+16) of all n_c members are contiguous, member after
//   member.  Element (cluster c, member m, dim j) sits at
//       data[off[c]*Dp + (j/16)*n_c*16 + m*16 + (j%16)]
//   so one delta_d step of 32 consecutive members is a few fully coalesced
//   2 KB runs (FP32), and a single member's step is whole 64-byte pieces.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/adsx.h"

namespace adsx {

constexpr int BLK = 16;                 // dims per layout block
constexpr unsigned ERR_LOCK_TIMEOUT = 1u;  // device error word bits

struct Index {
    int64_t N = 0;
    int32_t D = 0, Dp = 0, nlist = 0, storage = ADSX_F32;
    int device = 0;
    float *P = nullptr;        // Dp x Dp, zero padded, row-major (y = P x)
    float *cents = nullptr;    // nlist x Dp rotated centroids
    float *data = nullptr;     // N x Dp, dim-blocked per cluster
    int32_t *ids = nullptr;    // N: CSR position -> original id
    int64_t *off = nullptr;    // nlist + 1 CSR offsets
    int32_t *tile_off = nullptr;  // nlist + 1 prefix of ceil(n_c/32)
    unsigned int *err = nullptr;  // device error word
    std::vector<int64_t> h_off;
    int32_t total_tiles = 0;
    int64_t bytes = 0;
    // stage timing (adsx_set_stage_timing): events between search stages
    bool timing = false;
    bool timed_once = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

// ----------------------------------------------------------------- device
// One 16-dim block of a candidate against the matching 16 query dims,
// accumulated in dimension order: S += (y_j - q_j)^2 (Algorithm 1, the
// update of the approximate distance).  `x` is 64-byte aligned.
__device__ __forceinline__ float accum_block_f32(const float *__restrict__ x,
                                                 const float *__restrict__ q,
                                                 float S)
{
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float4 a = __ldg(x4 + i);
        float4 b = q4[i];
        float t;
        t = a.x - b.x; S = fmaf(t, t, S);
        t = a.y - b.y; S = fmaf(t, t, S);
        t = a.z - b.z; S = fmaf(t, t, S);
        t = a.w - b.w; S = fmaf(t, t, S);
    }
    return S;
}

// Two blocks with all eight loads issued before the arithmetic.
__device__ __forceinline__ float accum_2blocks_f32(const float *__restrict__ x0,
                                                   const float *__restrict__ x1,
                                                   const float *__restrict__ q,
                                                   float S)
{
    const float4 *a4 = reinterpret_cast<const float4 *>(x0);
    const float4 *b4 = reinterpret_cast<const float4 *>(x1);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    float4 v[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __ldg(a4 + i);
#pragma unroll
    for (int i = 0; i < 4; ++i) v[4 + i] = __ldg(b4 + i);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float4 b = q4[i];
        float t;
        t = v[i].x - b.x; S = fmaf(t, t, S);
        t = v[i].y - b.y; S = fmaf(t, t, S);
        t = v[i].z - b.z; S = fmaf(t, t, S);
        t = v[i].w - b.w; S = fmaf(t, t, S);
    }
    return S;
}

// Blocks [b0, b1) of member m of a cluster with n members whose layout
// starts at `base` (dims in ascending order, two blocks per load batch).
__device__ __forceinline__ float accum_range_f32(const float *__restrict__ base,
                                                 int64_t n, int64_t m, int b0,
                                                 int b1, const float *__restrict__ qv,
                                                 float S)
{
    const int64_t stride = n * BLK;
    const float *x = base + (int64_t)b0 * stride + m * BLK;
    int b = b0;
    for (; b + 2 <= b1; b += 2, x += 2 * stride)
        S = accum_2blocks_f32(x, x + stride, qv + b * BLK, S);
    if (b < b1) S = accum_block_f32(x, qv + b * BLK, S);
    return S;
}

// Threshold factor of the squared test after `blk` blocks (Sec. 3.2):
//   reject  iff  D*S_d > r^2 * d * (1+eps0/sqrt(d))^2
//          iff  S_d > r^2 * f(d),   f(d) = (d/D) (1 + eps0/sqrt(d))^2,
// with d = min(16*blk, D) true (unpadded) dimensions.
__device__ __forceinline__ float test_factor(int blk, int D, float eps0)
{
    int d = blk * BLK;
    if (d > D) d = D;
    float g = 1.0f + eps0 / sqrtf((float)d);
    return ((float)d / (float)D) * g * g;
}

// Sets the message returned by adsx_last_error() on the calling thread.
void set_last_error(const std::string &msg);

// ----------------------------------------------------------------- launches
cudaError_t launch_nt_gemm(const float *A, int64_t M, int lda, const float *B, int Nb,
                           int ldb, int Kd, float *C, int ldc, int Nout, bool dist,
                           cudaStream_t s);

cudaError_t launch_scatter_layout(const float *Y, int64_t N, int Dp, const int32_t *assign,
                                  const int64_t *pos_of_id, const int64_t *off, float *data,
                                  cudaStream_t s);

cudaError_t launch_select_nprobe(const float *dist, int64_t nq, int nlist, int nprobe,
                                 int32_t *probes, float *probe_d2, cudaStream_t s);

struct ScanArgs {
    const float *data;
    const int32_t *ids;
    const int64_t *off;
    const float *qrot;
    const int32_t *probes;
    const float *ftab;         // nblk + 1 test factors f(d) (Sec. 3.2)
    int64_t nq;
    int32_t D, Dp, nblk, nprobe, K, C, db;
    int32_t S, n_items;        // splits per query, work items = nq * S
    int32_t test_on;
    int64_t *out_ids;
    float *out_d2;
    int64_t *out_dims;         // zeroed by the caller when S > 1
    float *part_d;             // n_items x K partial lists (S > 1)
    int32_t *part_i;
    unsigned int *r2g;         // nq shared r^2 bounds, 0xffffffff = none (S > 1)
    unsigned int *work_counter;
    unsigned int *err;
};

size_t scan_smem_bytes(const ScanArgs &a);
int scan_items_target(int device);
cudaError_t launch_test_factors(float *ftab, int nblk, int D, float eps0, cudaStream_t s);
cudaError_t launch_ads_scan(const ScanArgs &a, int grid, cudaStream_t s);
cudaError_t launch_finalize_topk(const ScanArgs &a, cudaStream_t s);
int ads_scan_grid(const ScanArgs &a, int device);

struct FixedRArgs {
    const float *data;
    const int32_t *ids;
    const int64_t *off;
    const int32_t *tile_off;
    int32_t nlist, total_tiles;
    int64_t N;
    const float *qrot;
    const float *r2;
    int64_t nq;
    int32_t D, Dp, nblk, db;
    float eps0;
    int32_t test_on;
    uint8_t *decisions;
    int32_t *dims;
};
cudaError_t launch_dco_fixed_r(const FixedRArgs &a, cudaStream_t s);

}  // namespace adsx
