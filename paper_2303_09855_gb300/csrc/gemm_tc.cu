// gemm_tc.cu -- the dense contractions of the path on the 5th-generation
// tensor cores (tcgen05, sm_103a), FP32-accurate by a 3-term TF32 split:
//   x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi), and
//   A B^T ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T   (the lo*lo term, of
//   relative size 2^-22, is dropped), all accumulated in FP32 in TMEM.
// Use: the query-centroid distances of the probe step (Sec. 2.2.2),
//   D2[q][c] = ||q'||^2 + ||c'||^2 - 2 q'.c'  (clamped at 0),
// a dense nq x nlist x Dp contraction.
//
// One 128-thread CTA computes a 128 x 128 output tile.  Per 32-wide k-step
// every thread converts one row of A and one row of B (fp32 from global) into
// hi/lo TF32 halves in shared memory, in the canonical K-major no-swizzle
// layout of the tensor core (8-row x 16-byte core matrices); one thread then
// issues 4 x 3 tcgen05.mma (M = 128, N = 128, K = 8 each) into a 128-column
// FP32 accumulator in tensor memory and commits them to an mbarrier; after
// the last step each warp reads its 32 accumulator rows with tcgen05.ld and
// writes the epilogue.  The mbarrier wait is bounded: on time-out the kernel
// sets the error word, waits (bounded by 1 s of device time) for the batch
// already committed to arrive, frees its tensor memory and returns.
#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int TM = 128, TN = 128, BK = 32;
constexpr int SLAB = 4096;                     // bytes of one K = 8 slab of 128 rows
constexpr int OPER = (BK / 8) * SLAB;          // bytes of one operand (hi or lo) per k-step
constexpr int OPER_BYTES = 4 * OPER;           // A_hi, A_lo, B_hi, B_lo
constexpr int STAGE_BYTES = 4 * 32 * (TN + 4) * 4;  // epilogue: 4 warps x 32 rows x 132 floats
constexpr int SMEM_BYTES = OPER_BYTES > STAGE_BYTES ? OPER_BYTES : STAGE_BYTES;
constexpr uint32_t TMEM_COLS = 128;
constexpr unsigned WAIT_LIMIT = 1u << 22;
constexpr unsigned ERR_MMA_TIMEOUT = 8u;
constexpr unsigned ERR_MMA_DRAIN = 32u;
constexpr uint64_t DRAIN_NS = 1000000000ull;   // 1 s

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9 = bits 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// (K-direction) core-matrix offset >> 4 (bits 16-29), stride (M/N-direction)
// core-matrix offset >> 4 (bits 32-45), the fixed 0b001 at bits 46-48, no
// swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    const uint32_t LBO = 128, SBO = 256;
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (row r, k) inside a 128-row K = 8 slab: core matrix
// (r / 8, k / 4) is 128 contiguous bytes (8 rows x 16 bytes), K-adjacent core
// matrices 128 bytes apart, row groups 256 bytes apart.
__device__ __forceinline__ uint32_t slab_off(int r, int k)
{
    return (uint32_t)((r >> 3) * 256 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase)
{
    for (unsigned i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// The same wait bounded by time (%globaltimer nanoseconds) instead of a
// count: used to drain MMAs already committed after a timed-out wait.
__device__ __forceinline__ bool mbar_wait_ns(uint32_t bar, uint32_t phase, uint64_t limit_ns)
{
    uint64_t t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        :
        : "r"(tmem), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
        : "memory");
}

// Loads row `r` of a 128-row tile (rows >= rows_valid or k >= Kd read as 0)
// for the 32-wide k-step k0, splits it and stores hi/lo into their slabs.
__device__ __forceinline__ void stage_row(const float *__restrict__ src, bool valid,
                                          int k0, int Kd, int r, uint8_t *hi, uint8_t *lo)
{
    const bool vec = valid && (k0 + BK <= Kd) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
    float x[BK];
    if (vec) {
#pragma unroll
        for (int i = 0; i < BK / 4; ++i) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(src) + i);
            x[4 * i] = t.x;
            x[4 * i + 1] = t.y;
            x[4 * i + 2] = t.z;
            x[4 * i + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < BK; ++k) x[k] = (valid && k0 + k < Kd) ? src[k] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
        const uint32_t h = to_tf32(x[k]);
        const uint32_t l = to_tf32(x[k] - __uint_as_float(h));
        const uint32_t o = (uint32_t)(k >> 3) * SLAB + slab_off(r, k & 7);
        *reinterpret_cast<uint32_t *>(hi + o) = h;
        *reinterpret_cast<uint32_t *>(lo + o) = l;
    }
}

// C[i][j] = max(an[i] + bn[j] - 2 (A B^T)[i][j], 0).
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const float *__restrict__ A, int64_t M, int lda, const float *__restrict__ B,
                   int Nb, int ldb, int Kd, float *__restrict__ C, int ldc, int Nout,
                   const float *__restrict__ an, const float *__restrict__ bn, unsigned *err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;
    uint8_t *Ah = sm, *Al = sm + OPER, *Bh = sm + 2 * OPER, *Bl = sm + 3 * OPER;
    const uint32_t bar = smem_addr(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(&tmem_slot)), "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    uint32_t phase = 0;
    bool ok = true;
    const int64_t arow = m0 + tid;
    const int brow = n0 + tid;
    for (int k0 = 0; k0 < Kd && ok; k0 += BK) {
        stage_row(A + arow * lda + k0, arow < M, k0, Kd, tid, Ah, Al);
        stage_row(B + (int64_t)brow * ldb + k0, brow < Nb, k0, Kd, tid, Bh, Bl);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < BK / 8; ++s) {
                const uint64_t ah = make_desc(smem_addr(Ah + s * SLAB));
                const uint64_t al = make_desc(smem_addr(Al + s * SLAB));
                const uint64_t bh = make_desc(smem_addr(Bh + s * SLAB));
                const uint64_t bl = make_desc(smem_addr(Bl + s * SLAB));
                mma_tf32(tmem, al, bh, (k0 > 0 || s > 0) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, 1u);
                mma_tf32(tmem, ah, bh, 1u);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                :
                : "r"(bar)
                : "memory");
        }
        ok = mbar_wait(bar, phase);
        phase ^= 1u;
        ok = __syncthreads_and(ok);
    }
    if (!ok) {
        // The MMAs of the last batch were committed to the barrier and will
        // arrive on it: wait for that arrival (up to DRAIN_NS, far beyond the
        // duration of one batch) so that tensor memory is not released under
        // them.  Should even that wait give up (the device is not making
        // progress), ERR_MMA_DRAIN records it; the allocation is released
        // regardless, as a CTA must not exit holding tensor memory.
        if (tid == 0) atomicOr(err, ERR_MMA_TIMEOUT);
        const bool drained = mbar_wait_ns(bar, phase ^ 1u, DRAIN_NS);
        if (!__syncthreads_and(drained) && tid == 0) atomicOr(err, ERR_MMA_DRAIN);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // Each warp reads its 32 accumulator rows (lane = row) and stages the
        // finished 32 x 128 distances in the (now idle) operand shared memory,
        // rows 132 floats apart (float4 writes of 8 lanes hit distinct banks),
        // then writes every row as one coalesced 512-byte run.
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        const float rn = (row < M) ? an[row] : 0.f;
        float *stage = reinterpret_cast<float *>(sm) + warp * 32 * (TN + 4);
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                "%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(trow + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float o[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c0 + j;
                const float cn = (col < Nout) ? bn[col] : 0.f;
                o[j] = fmaxf(rn + cn - 2.f * __uint_as_float(v[j]), 0.f);
            }
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(stage + lane * (TN + 4) + c0 + j) =
                    make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
        }
        __syncwarp();
        const int col = n0 + lane * 4;
        const bool vec_ok = (ldc % 4 == 0) && (col + 4 <= Nout);
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
            const int64_t grow = m0 + warp * 32 + r;
            if (grow >= M) break;
            const float4 x = *reinterpret_cast<const float4 *>(stage + r * (TN + 4) + lane * 4);
            float *dst = C + grow * ldc + col;
            if (vec_ok) {
                *reinterpret_cast<float4 *>(dst) = x;
            } else {
                if (col < Nout) dst[0] = x.x;
                if (col + 1 < Nout) dst[1] = x.y;
                if (col + 2 < Nout) dst[2] = x.z;
                if (col + 3 < Nout) dst[3] = x.w;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :
                     : "r"(tmem), "r"(TMEM_COLS)
                     : "memory");
}

// Squared norms of the rows of a row-major matrix (one warp per row).
__global__ void row_sqnorm_kernel(const float *__restrict__ X, int64_t M, int ld, int K,
                                  float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < M;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        for (int k = lane; k < K; k += 32) {
            const float x = X[r * ld + k];
            s = fmaf(x, x, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[r] = s;
    }
}

}  // namespace

cudaError_t launch_tc_gemm(const float *A, int64_t M, int lda, const float *B, int Nb, int ldb,
                           int Kd, float *C, int ldc, int Nout, const float *an, const float *bn,
                           unsigned *err, cudaStream_t s)
{
    if (M <= 0 || Nout <= 0) return cudaSuccess;
    if ((M + TM - 1) / TM > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (!an || !bn) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)((Nout + TN - 1) / TN));
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<<<grid, 128, SMEM_BYTES, s>>>(A, M, lda, B, Nb, ldb, Kd, C, ldc, Nout, an, bn, err);
    return cudaGetLastError();
}

cudaError_t launch_row_sqnorm(const float *X, int64_t M, int ld, int K, float *out, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    int64_t blocks = (M * 32 + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    row_sqnorm_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, M, ld, K, out);
    return cudaGetLastError();
}

}  // namespace adsx
