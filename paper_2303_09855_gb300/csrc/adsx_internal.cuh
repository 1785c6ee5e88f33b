// adsx_internal.cuh -- internal declarations of libadsx.so (not installed).
//
// Device data layout of an index (Sec. 5.2 IVF++ generalised):
//   rotated vectors y = P x are stored per cluster (CSR order, members of a
//   cluster in ascending id), and inside a cluster "dimension-block major":
//   the 16 dims [16b, 16b+16) of all n_c members are contiguous, member after
//   member.  Element (cluster c, member m, dim j) sits at
//       data[off[c]*Dp + (j/16)*n_c*16 + m*16 + (j%16)]
//   so one block of 8 (FP32) or 16 (16-bit) consecutive members is a single
//   contiguous 512-byte run, and a single member's block is one 64- or
//   32-byte piece.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/adsx.h"

namespace adsx {

constexpr int BLK = 16;                 // dims per layout block
// With the test off (eps0 = +inf, delta_d >= D: FDScanning) partial sums are
// still accumulated in steps of this many blocks (32 dims), so that every
// scan schedule and every way of turning the test off sums a candidate's
// distance in the same order.
constexpr int FD_STEP_BLOCKS = 2;
constexpr unsigned ERR_LOCK_TIMEOUT = 1u;  // device error word bits

struct Index {
    int64_t N = 0;
    int32_t D = 0, Dp = 0, nlist = 0, storage = ADSX_F32;
    int device = 0;
    float *P = nullptr;        // Dp x Dp, zero padded, row-major (y = P x)
    float *cents = nullptr;    // nlist x Dp rotated centroids
    float *cnorm = nullptr;    // nlist ||c'||^2
    uint32_t *cents_split = nullptr;  // TF32 halves of cents for the centroid GEMM (tf32_split)
    void *data = nullptr;      // N x Dp of the storage type, dim-blocked per cluster
    float *rows32 = nullptr;   // N x Dp FP32 rotated rows in CSR order (16-bit storage only)
    float *norms = nullptr;    // N FP32 norms ||y|| in CSR order (16-bit storage only)
    float *onorm = nullptr;    // N raw norms ||o|| in CSR order (inner-product indexes)
    int32_t *kac_pairs = nullptr;  // Kac-walk rotation (instead of P): L x 2(D/2) pairs
    float *kac_cs = nullptr;       //   and their (cos, sin)
    int32_t kac_L = 0;
    int32_t metric = ADSX_L2;  // ADSX_L2 / ADSX_IP / ADSX_COSINE
    int32_t *ids = nullptr;    // N: CSR position -> original id
    int64_t *off = nullptr;    // nlist + 1 CSR offsets
    int32_t *tile_off = nullptr;  // nlist + 1 prefix of ceil(n_c/32)
    unsigned int *err = nullptr;  // device error word
    std::vector<int64_t> h_off;
    int32_t total_tiles = 0;
    int64_t bytes = 0;
    int32_t tuned_delta_d = 32;   // used when a search passes delta_d = 0
    int32_t items_per_sm = 48;    // work items per SM targeted when splitting queries
    // scan schedule (adsx_set_scan_schedule / adsx_autotune): ADSX_SCHED_AUTO,
    // _QUERY or _CLUSTER; queries per cluster-major work item (0: chosen per
    // batch); probe ranks of round 0 and the growth factor of later rounds'
    // ranges
    int32_t sched = ADSX_SCHED_AUTO;
    int32_t cm_G = 0;
    int32_t cm_tpi = 2;           // 32-member tiles per cluster-major work item
    int32_t max_tiles = 0;        // tiles of the largest cluster
    int32_t cm_r0 = 1;
    int32_t cm_growth = 4;
    // query rotation on the tensor cores (rot_tc, adsx_set_query_rotation):
    // P's rows split into rot_T integer slices of rot_b bits (rot_F: each
    // row's exponent), laid out per level L = 2..T+1 at rot_B + rot_boff[L]
    // as Dp x (L - 1) Dp matrices; rot_ok when they exist
    bool rot_ok = false, rot_tc = false;
    int32_t rot_b = 0, rot_T = 0, rot_Lmax = 0;
    float *rot_B = nullptr;
    int32_t *rot_F = nullptr;
    int64_t rot_boff[16] = {};
    // stage timing (adsx_set_stage_timing): events between search stages
    bool timing = false;
    bool timed_once = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // and around each scan-kernel launch of the search (rounds of the
    // cluster-major schedule, the query-major scan): start/end pairs
    static constexpr int MAX_KEV = 16;
    cudaEvent_t kev[2 * MAX_KEV] = {};
    int nkev = 0;
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

// 16-bit storage: a 16-dim block is 32 bytes (one sector), converted to FP32
// and accumulated in FP32 in dimension order.
__device__ __forceinline__ void unpack2(unsigned x, float &lo, float &hi, __nv_bfloat16)
{
    lo = __uint_as_float(x << 16);
    hi = __uint_as_float(x & 0xffff0000u);
}

__device__ __forceinline__ void unpack2(unsigned x, float &lo, float &hi, __half)
{
    lo = __half2float(__ushort_as_half((unsigned short)(x & 0xffffu)));
    hi = __half2float(__ushort_as_half((unsigned short)(x >> 16)));
}

__device__ __forceinline__ void unpack8(uint4 w, float *v, __nv_bfloat16 t)
{
    unpack2(w.x, v[0], v[1], t);
    unpack2(w.y, v[2], v[3], t);
    unpack2(w.z, v[4], v[5], t);
    unpack2(w.w, v[6], v[7], t);
}

__device__ __forceinline__ void unpack8(uint4 w, float *v, __half t)
{
    unpack2(w.x, v[0], v[1], t);
    unpack2(w.y, v[2], v[3], t);
    unpack2(w.z, v[4], v[5], t);
    unpack2(w.w, v[6], v[7], t);
}

template <typename H>
__device__ __forceinline__ float accum_8h(uint4 w, const float *__restrict__ q, float S)
{
    float v[8];
    unpack8(w, v, H());
    const float4 q0 = reinterpret_cast<const float4 *>(q)[0];
    const float4 q1 = reinterpret_cast<const float4 *>(q)[1];
    float t;
    t = v[0] - q0.x; S = fmaf(t, t, S);
    t = v[1] - q0.y; S = fmaf(t, t, S);
    t = v[2] - q0.z; S = fmaf(t, t, S);
    t = v[3] - q0.w; S = fmaf(t, t, S);
    t = v[4] - q1.x; S = fmaf(t, t, S);
    t = v[5] - q1.y; S = fmaf(t, t, S);
    t = v[6] - q1.z; S = fmaf(t, t, S);
    t = v[7] - q1.w; S = fmaf(t, t, S);
    return S;
}

// Blocks [b0, b1) of member m, 16-bit storage, two blocks per load batch.
template <typename H>
__device__ __forceinline__ float accum_range_h(const H *__restrict__ base, int64_t n, int64_t m,
                                               int b0, int b1, const float *__restrict__ qv,
                                               float S)
{
    const int64_t stride = n * BLK;
    const H *x = base + (int64_t)b0 * stride + m * BLK;
    int b = b0;
    for (; b + 2 <= b1; b += 2, x += 2 * stride) {
        const uint4 *p0 = reinterpret_cast<const uint4 *>(x);
        const uint4 *p1 = reinterpret_cast<const uint4 *>(x + stride);
        uint4 w0 = __ldg(p0), w1 = __ldg(p0 + 1), w2 = __ldg(p1), w3 = __ldg(p1 + 1);
        const float *q = qv + b * BLK;
        S = accum_8h<H>(w0, q, S);
        S = accum_8h<H>(w1, q + 8, S);
        S = accum_8h<H>(w2, q + 16, S);
        S = accum_8h<H>(w3, q + 24, S);
    }
    if (b < b1) {
        const uint4 *p0 = reinterpret_cast<const uint4 *>(x);
        uint4 w0 = __ldg(p0), w1 = __ldg(p0 + 1);
        const float *q = qv + b * BLK;
        S = accum_8h<H>(w0, q, S);
        S = accum_8h<H>(w1, q + 8, S);
    }
    return S;
}

__device__ __forceinline__ float accum_range(const float *base, int64_t n, int64_t m, int b0,
                                             int b1, const float *qv, float S)
{
    return accum_range_f32(base, n, m, b0, b1, qv, S);
}
__device__ __forceinline__ float accum_range(const __nv_bfloat16 *base, int64_t n, int64_t m,
                                             int b0, int b1, const float *qv, float S)
{
    return accum_range_h(base, n, m, b0, b1, qv, S);
}
__device__ __forceinline__ float accum_range(const __half *base, int64_t n, int64_t m, int b0,
                                             int b1, const float *qv, float S)
{
    return accum_range_h(base, n, m, b0, b1, qv, S);
}

// Unit roundoff of the storage type (round to nearest): |x~ - x| <= u |x|.
template <typename T> struct Roundoff;
template <> struct Roundoff<float> { static constexpr float u = 0.f; };
template <> struct Roundoff<__nv_bfloat16> { static constexpr float u = 1.0f / 256.0f; };
template <> struct Roundoff<__half> { static constexpr float u = 1.0f / 2048.0f; };

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

// ---- probe selection (gemm_tc.cu epilogue, select.cu)
// Ordering key of a query-centroid distance: the bit pattern of a positive
// float orders like the float; zero, negative rounding residue and NaN map
// to 0 / +inf.
__device__ __forceinline__ unsigned dist_key(float v)
{
    if (!(v > 0.f)) return (v != v) ? 0x7f800000u : 0u;
    return __float_as_uint(v);
}

// Keeps t0 <= t1 <= t2 <= t3, the four smallest words seen so far.
__device__ __forceinline__ void keep4(unsigned x, unsigned &t0, unsigned &t1, unsigned &t2,
                                      unsigned &t3)
{
    unsigned m;
    m = min(t0, x); x = max(t0, x); t0 = m;
    m = min(t1, x); x = max(t1, x); t1 = m;
    m = min(t2, x); x = max(t2, x); t2 = m;
    t3 = min(t3, x);
}

// The tile summary of the distance matrix: for every query row and every
// 128-column tile, the tile's four smallest entries, ascending, each as
// (dist_key & ~127) | column within the tile; a tile narrower than four
// columns pads with ~0u.  Row q's tiles are SUMMARY_TILE-wide and stored at
// summary + (q * ntiles + tile) * 4.
constexpr int SUMMARY_TILE = 128;
constexpr unsigned SUMMARY_LOW = SUMMARY_TILE - 1;

// ----------------------------------------------------------------- launches
// C[i][j] = max(an[i] + bn[j] - 2 (A B^T)[i][j], 0) on tcgen05 tensor cores
// (3-term TF32 split, FP32 accumulation in TMEM): A M x Kd (row stride lda),
// B Nb x Kd (row stride ldb; rows >= Nb read as 0), C M x Nout (row stride
// ldc), an / bn the squared row norms of A / B.
// TF32 hi/lo halves of the rows of X (R x K, K a multiple of 16) in the
// layout launch_tc_gemm streams; `out` holds tf32_split_words(R, K) words.
int64_t tf32_split_words(int64_t rows, int K);
cudaError_t launch_tf32_split(const float *X, int64_t R, int ld, int K, uint32_t *out, cudaStream_t s);
// C = max(an + bn - 2 A B^T, 0) (M x Nout, row stride ldc) from split A and B
// (K = Kd), and the probe select's tile summary when `summary` is not NULL.
cudaError_t launch_tc_gemm(const uint32_t *As, int64_t M, const uint32_t *Bs, int Kd, float *C,
                           int ldc, int Nout, const float *an, const float *bn, unsigned *err,
                           cudaStream_t s, unsigned *summary = nullptr);
cudaError_t launch_row_sqnorm(const float *X, int64_t M, int ld, int K, float *out, cudaStream_t s);

// Query rotation Y = X P^T on the tensor cores, FP32-accurate (gemm_tc.cu):
// digit width b, digits T and kept levels for a padded dimension Dp (T = 0:
// not available, Dp > 1024); the partial-sum scratch (floats) that lets a
// batch of nq rows run in one pass of up to 1024 rows; and the rotation
// itself (part: part_floats of scratch, at least one row's worth; xexp: nq
// ints).
void tc_rot_params(int Dp, int *b, int *T, int *Lmax);
int64_t tc_rot_scratch_floats(const Index *ix, int64_t nq);
cudaError_t rotate_queries_tc(const Index *ix, const float *X, int64_t nq, float *Y, float *part,
                              int64_t part_floats, int32_t *xexp, cudaStream_t s);

// Rotation Y = X P^T (N x D times D x D, P row stride ldp) with compensated
// (Dot2) FP32 dot products, written as N x Dp FP32 (columns >= D are 0).
cudaError_t launch_rotate(const float *X, int64_t N, int D, const float *P, int ldp, float *Y,
                          int Dp, cudaStream_t s);

// Layered Kac walk (Sec. 6.2.3): Y = W X for N rows of D values (row stride
// ldx), written as N x Dp FP32 (columns >= D are 0); pairs / cs are L x 2(D/2).
cudaError_t launch_kac_rotate(const float *X, int64_t N, int D, int ldx, const int32_t *pairs,
                              const float *cs, int L, float *Y, int Dp, cudaStream_t s);

// The index's rotation of N raw rows (D values each, contiguous) into an
// N x Dp buffer: the dense P (compensated FP32) or the Kac walk.
inline cudaError_t rotate_rows(const Index *ix, const float *X, int64_t N, float *Y,
                               cudaStream_t s)
{
    if (ix->kac_L > 0)
        return launch_kac_rotate(X, N, ix->D, ix->D, ix->kac_pairs, ix->kac_cs, ix->kac_L, Y,
                                 ix->Dp, s);
    return launch_rotate(X, N, ix->D, ix->P, ix->Dp, Y, ix->Dp, s);
}

// Rotated rows Y (N x Dp, FP32) into the dim-blocked layout of `storage`
// (ADSX_F32 / ADSX_BF16 / ADSX_F16); for 16-bit storage also the FP32 row copy
// and the norms, both in CSR order.
// Scales each of the N rows (D values, row stride ld) to unit norm in place
// (norm accumulated in FP64; a zero row stays zero and, with zero_err, sets
// ERR_ZERO_ROW in *zero_err); norms (may be NULL) receives the original norms.
cudaError_t launch_normalize_rows(float *X, int64_t N, int ld, int D, float *norms,
                                  unsigned *zero_err, cudaStream_t s);
// v[0..n) := max(v): the inner-product index's constant centroid term.
cudaError_t launch_fill_max(float *v, int n, cudaStream_t s);
// dst[pos[i]] = src[i] for i < N (row order -> CSR order).
cudaError_t launch_scatter_f32(const float *src, const int64_t *pos, int64_t N, float *dst,
                               cudaStream_t s);

cudaError_t launch_scatter_layout(const float *Y, int64_t N, int Dp, const int32_t *assign,
                                  const int64_t *pos_of_id, const int64_t *off, void *data,
                                  int storage, float *rows32, float *norms, cudaStream_t s);

cudaError_t launch_select_nprobe(const float *dist, int64_t nq, int nlist, int nprobe,
                                 int32_t *probes, float *probe_d2, cudaStream_t s,
                                 const int32_t *nprobe_q = nullptr,
                                 const unsigned *summary = nullptr);

struct ScanArgs {
    const void *data;          // storage type per `storage`
    const float *rows32;       // FP32 rows (16-bit storage: exact recheck at d = D)
    const float *norms;
    int32_t storage;
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
    // batched form (all NULL for a uniform search): per-query K and nprobe,
    // output offsets, the planned items (x = query, y = split << 16 | splits),
    // each query's first item, and the item count (device)
    const int32_t *Kq = nullptr;
    const int32_t *nprobe_q = nullptr;
    const int64_t *out_off = nullptr;
    const int2 *items = nullptr;
    const int32_t *item_first = nullptr;
    const int32_t *n_items_dev = nullptr;
    int64_t out_total = 0;       // length of out_ids/out_d2 when out_off is set
    int32_t Kmax = 0;            // stride of partial lists (>= every K)
    int32_t probe_stride = 0;    // row stride of `probes` (>= every nprobe)
    int32_t finalize_T = 0;
    // similarity (Sec. 8, extension (1)): ADSX_L2 keys are squared distances;
    // ADSX_COSINE keys are squared distances of normalised vectors; ADSX_IP
    // keys are -<o,q> with per-object thresholds 2 - 2 r / (||o|| ||q||) on
    // the normalised vectors (onorm: ||o|| per CSR row, qnorm: ||q|| per query)
    int32_t metric = ADSX_L2;
    const float *onorm = nullptr;
    const float *qnorm = nullptr;
    // fixed-threshold mode (the verification protocol of Sec. 6.2.5,
    // adsx_dco_fixed_r): decisions != NULL makes every item test all members
    // of every cluster (probe slot p is cluster p; probes unused) against the
    // fixed r2fixed[q], with the same accumulation, test and recheck code as
    // a search but no KNN set; each candidate's decision (0 rejected at
    // d < D, 1 positive, 2 negative at d = D) and dims go to
    // decisions / dec_dims[q * N + original id]
    const float *r2fixed = nullptr;
    uint8_t *decisions = nullptr;
    int32_t *dec_dims = nullptr;
    int64_t N = 0;
};

// Graph search with ADSampling DCOs (HNSW+, graph.cu).
struct GraphArgs {
    const float *data;          // the index's FP32 dim-blocked vectors
    const int64_t *vbase;       // per vertex: element offset of its block 0
    const int32_t *vstride;     // per vertex: block stride (16 * cluster size)
    const int32_t *nbr;         // N x degree neighbour ids (-1 = none)
    int32_t degree;
    const int64_t *entry;       // nlist x n_ce start vertices (-1 = none)
    int32_t n_ce;               // entries per cluster
    const float *qrot;          // nq x Dp rotated queries
    const int32_t *probes;      // nq x n_entry nearest clusters
    int32_t n_entry;
    const float *ftab;          // nblk + 1 test factors
    int64_t nq;
    int32_t D, Dp, nblk, db, test_on, K, ef, max_iter;
    int32_t nst;                // Algorithm 1 steps of one DCO at most
    int32_t pp;                 // 0: HNSW+, 1: HNSW++ (Sec. 5.1)
    int32_t metric;             // ADSX_L2, or ADSX_COSINE (output 1 - d^2/2)
    int64_t *out_ids;
    float *out_d2;
    int64_t *out_dims;          // may be NULL
    unsigned *bitmap;           // warps x bm_words visited bits (all zero between queries)
    int64_t bm_words;
    int32_t *vlist;             // warps x vcap visited ids of the current query
    int64_t vcap;               // >= min(n_entry n_ce + 1 + max_iter * degree, N)
    int32_t warps;              // resident warps launched
    unsigned long long *qnext;  // next query to take (zeroed by the launcher)
};
// nst: Algorithm 1 steps of one DCO at most (ceil(nblk / db))
size_t graph_search_smem(int Dp, int ef, int K, int nst);
// warps of graph_search_kernel resident at once on nsm SMs (0: does not fit)
int graph_search_resident_warps(int Dp, int ef, int K, int nst, int nsm);
cudaError_t launch_knn_to_graph(const int64_t *knn, int64_t N, int64_t row0, int Kk, int degree,
                                int32_t *nbr, cudaStream_t s);
cudaError_t launch_vertex_map(const int64_t *off, int nlist, const int32_t *ids, int Dp,
                              int64_t *vbase, int32_t *vstride, cudaStream_t s);
cudaError_t launch_cluster_entries(const float *data, const int64_t *off, const int32_t *ids,
                                   const float *cents, int nlist, int Dp, int E, float *mind,
                                   int64_t *entry,
                                   cudaStream_t s);
cudaError_t launch_graph_search(const GraphArgs &g, cudaStream_t s);

size_t scan_smem_bytes(const ScanArgs &a);
int scan_items_target(int device, int items_per_sm = 48);
cudaError_t launch_test_factors(float *ftab, int nblk, int D, float eps0, cudaStream_t s,
                                int pd = 0);
cudaError_t launch_ads_scan(const ScanArgs &a, int grid, cudaStream_t s);
cudaError_t launch_finalize_topk(const ScanArgs &a, cudaStream_t s);

// Splits per query of the uniform search: enough work items to fill the GPU
// (`target`), but each split should expect at least 2K candidates (a split
// prunes only once it holds K exact distances), and at most 64 and the
// finalize kernel's merge buffer (S * next_pow2(K) <= 16384).
// members_per_list = N / nlist.
inline int32_t uniform_splits(int64_t nq, int nprobe, int K, int64_t target,
                              int64_t members_per_list)
{
    int Kp = 1;
    while (Kp < K) Kp <<= 1;
    int64_t S = (target + nq - 1) / (nq > 0 ? nq : 1);
    const int64_t by_cand = (int64_t)nprobe * members_per_list / (2 * (int64_t)K);
    if (S > by_cand) S = by_cand;
    if (S > 64) S = 64;
    const int64_t cap = 16384 / Kp > 1 ? 16384 / Kp : 1;
    if (S > cap) S = cap;
    return (int32_t)(S > 1 ? S : 1);
}


// Candidate-buffer capacity of a warp's KNN set for K: a power of two
// >= max(2 next_pow2(K), K + 32).
inline int32_t knn_buffer_capacity(int K)
{
    int Kp = 1;
    while (Kp < K) Kp <<= 1;
    const int need = 2 * Kp > K + 32 ? 2 * Kp : K + 32;
    int C = 1;
    while (C < need) C <<= 1;
    return C;
}

// The fields of a uniform search's scan (one K and one nprobe for every
// query) that every entry point sets the same way: the index's arrays and
// shapes, the buffer capacity, the splits per query, the step and whether the
// test runs (eps0 = +inf, delta_d >= D: FDScanning, one full-width step; pd:
// PDScanning's f(d) = 1).  The caller sets the per-call buffers (queries,
// probes, test factors, outputs, counters and split scratch).  Returns
// false when nq * S does not fit the item counter.
inline bool fill_uniform_scan(ScanArgs &a, const Index *ix, int64_t nq, int K, int nprobe,
                              float eps0, int delta_d, int pd)
{
    a.metric = ix->metric;
    a.onorm = ix->onorm;
    a.data = ix->data;
    a.rows32 = ix->rows32;
    a.norms = ix->norms;
    a.storage = ix->storage;
    a.ids = ix->ids;
    a.off = ix->off;
    a.nq = nq;
    a.D = ix->D;
    a.Dp = ix->Dp;
    a.nblk = ix->Dp / BLK;
    a.nprobe = nprobe;
    a.K = K;
    a.C = knn_buffer_capacity(K);
    a.S = uniform_splits(nq, nprobe, K, scan_items_target(ix->device, ix->items_per_sm),
                         ix->N / ix->nlist);
    if (nq * (int64_t)a.S >= ((int64_t)1 << 31)) return false;
    a.n_items = (int32_t)(nq * a.S);
    a.db = delta_d / BLK;
    a.test_on = (isinf(eps0) && !pd) ? 0 : 1;
    if (a.db >= a.nblk) a.test_on = 0;
    if (!a.test_on) a.db = FD_STEP_BLOCKS < a.nblk ? FD_STEP_BLOCKS : a.nblk;   // FDScanning
    a.out_dims = nullptr;
    a.part_d = nullptr;
    a.part_i = nullptr;
    a.r2g = nullptr;
    a.err = ix->err;
    return true;
}

// Batched form: validates per-query K / nprobe, chooses splits, orders the
// queries longest-first and writes the item list (capacity nq * 64 items).
cudaError_t launch_plan_batched(const int32_t *Kq, const int32_t *nprobe_q, int64_t nq,
                                int maxK, int maxP, int target_items, int64_t members_per_list,
                                int2 *items, int32_t *item_first, int32_t *n_items,
                                int32_t *qperm, const int64_t *out_off_in, int64_t *out_off,
                                unsigned *err, cudaStream_t s);
constexpr unsigned ERR_BATCH_ARGS = 2u;   // a per-query K or nprobe was out of range
constexpr unsigned ERR_OUT_RANGE = 4u;    // an output offset + K exceeded the output length
constexpr unsigned ERR_ZERO_ROW = 16u;    // a zero-norm row where a unit row is required
constexpr int BATCH_MAX_SPLITS = 16;
int ads_scan_grid(const ScanArgs &a, int device);

// ---- cluster-major schedule (cmscan.cu)
constexpr int CM_MAX_DB = 4;     // blocks per step (delta_d <= 64)
constexpr int CM_MAX_G = 64;     // queries per work item
struct CmArgs {
    const void *data;
    const float *rows32;
    const float *norms;
    int32_t storage;
    const int32_t *ids;
    const int64_t *off;
    const float *qrot;
    int32_t D, Dp, nblk, db, test_on;
    const float *ftab;
    const float *r2;            // per query: the round's r^2 (+inf: none yet)
    const int32_t *coff;        // nlist + 1 offsets into qlist
    const int32_t *qlist;       // queries of each cluster in this round
    const int2 *items;          // (cluster, first query slot of the item)
    const int32_t *n_items;     // device count of items
    int32_t items_cap;          // upper bound of *n_items (grid sizing)
    int32_t G;                  // queries per item
    int32_t tpi;                // 32-member tiles per item (a chunk of the cluster)
    unsigned *work_counter;
    float *app_d;               // nq x cap appended (distance, id)
    int32_t *app_i;
    unsigned *app_n;            // nq appended counts
    int32_t cap;
    int64_t *out_dims;          // may be NULL: dims sampled, added per query
    // 16-bit storage, round 0 (no r yet): append the approximate S_D and the
    // CSR row of every member instead of rechecking each one; the exact
    // distances of the few that can reach the top-K follow (cm_recheck0)
    int32_t defer_recheck = 0;
    // fixed-threshold mode (decisions != NULL), as ScanArgs
    const float *r2fixed = nullptr;
    uint8_t *decisions = nullptr;
    int32_t *dec_dims = nullptr;
    int64_t N = 0;
};
struct CmMergeArgs {
    int64_t nq;
    int32_t K, cap, T;
    int64_t *ids;               // nq x K running top-K ids (-1 padded)
    float *d2;                  // nq x K keys (values after the final pass)
    const float *app_d;
    const int32_t *app_i;
    unsigned *app_n;            // may be NULL (nothing appended)
    float *r2;
    int32_t *ovf;
    int32_t metric;
    int32_t final_pass;
};
// Round 0 of a 16-bit cluster-major search, per query: the appended
// (approximate S_D, CSR row) pairs become the exact (S_D, id) pairs of every
// member that can be among the K nearest (the others are dropped).
struct CmRecheck0Args {
    int64_t nq;
    int32_t K, cap, Dp;
    float u;                    // unit roundoff of the storage type
    const float *rows32, *norms, *qrot;
    const int32_t *ids;
    float *app_d;
    int32_t *app_i;
    unsigned *app_n;
};
cudaError_t launch_cm_recheck0(const CmRecheck0Args &r, cudaStream_t s);
// The rounds of a cluster-major search: probe ranks [lo[r], lo[r + 1]) form
// round r; its work items start at ibase[r] of the plan's item array.
constexpr int CM_MAX_ROUNDS = 8;
struct CmRounds {
    int32_t n;
    int32_t lo[CM_MAX_ROUNDS + 1];
    int64_t ibase[CM_MAX_ROUNDS];
};
// Plans of all rounds: cnt, ioff and cur are n x nlist, coff n x (nlist + 1),
// n_items n; round r's query lists start at qlist + nq * (lo[r] - lo[0]).
struct CmPlan {
    int32_t *cnt, *coff, *ioff, *cur, *qlist, *n_items;
    int2 *items;
};
size_t cm_smem_bytes(int G, int db, int storage);
cudaError_t launch_cm_plan(const int32_t *probes, int64_t nq, int pstride, const CmRounds &R,
                           int nlist, int G, int tpi, const int64_t *off, CmPlan &pl,
                           cudaStream_t s);
cudaError_t launch_cm_scan(const CmArgs &a, int device, cudaStream_t s);
cudaError_t launch_cm_merge(const CmMergeArgs &m, cudaStream_t s);
cudaError_t launch_cm_overflow_items(const int32_t *ovf, int64_t nq, int2 *items, int32_t *n_items,
                                     cudaStream_t s);
cudaError_t launch_cm_all_clusters(int32_t *probes, int64_t nq, int nlist, cudaStream_t s);



}  // namespace adsx
