// gemm_tc.cu -- the dense contractions of the path on the 5th-generation
// tensor cores (tcgen05, sm_103a), FP32-accurate by a 3-term TF32 split:
//   x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi), and
//   A B^T ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T   (the lo*lo term, of
//   relative size 2^-22, is dropped), all accumulated in FP32 in TMEM.
// Use: the query-centroid distances of the probe step (Sec. 2.2.2),
//   D2[q][c] = ||q'||^2 + ||c'||^2 - 2 q'.c'  (clamped at 0),
// a dense nq x nlist x Dp contraction.
//
// The operands are split once into hi/lo TF32 halves (tf32_split_kernel:
// the queries per search, the centroids at index build), already in the
// canonical K-major no-swizzle layout of the tensor core (8-row x 16-byte
// core matrices), so that a 128-row block's K = 16 step is one contiguous
// 16 KB run per operand.  One 128-thread CTA computes a 128 x 128 output
// tile: one thread streams the steps into a 2-deep shared-memory ring with
// bulk copies (the TMA engine) and issues 2 x 3 tcgen05.mma (M = 128,
// N = 128, K = 8 each) per step into a 128-column FP32 accumulator in tensor
// memory; three CTAs share an SM, so that while one waits for its copies or
// writes its epilogue the others keep the tensor pipe busy.  After the last step each warp reads its 32 accumulator rows with
// tcgen05.ld and writes the epilogue: the distances, and for the probe
// select the tile's four smallest entries per row (one thread owns a row, so
// this costs a compare-exchange chain per value and no communication).
#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int TM = 128, TN = 128, BK = 32;
constexpr int SLAB = 4096;                     // bytes of one K = 8 slab of 128 rows
constexpr int OPER = (BK / 8) * SLAB;          // bytes of one operand (hi or lo) per k-step
constexpr int STAGE_BYTES = 4 * 32 * (TN + 4) * 4;  // epilogue: 4 warps x 32 rows x 132 floats
// the centroid GEMM's ring: stages of K = 16 (two slabs), A and B halves
constexpr int GEMM_KS = 2;                              // slabs per stage
constexpr int GEMM_OPND_BYTES = GEMM_KS * 2 * SLAB;      // one operand's hi + lo per stage
constexpr int GEMM_STAGE_BYTES = 2 * GEMM_OPND_BYTES;    // A and B: 32 KB
// two stages: the block's shared memory (67.6 KB with the epilogue staging,
// which reuses the ring) lets three CTAs share an SM; measured faster than
// three stages with two CTAs (0.121 vs 0.135 ms for 10k x 4096 x 128)
constexpr int GEMM_STAGES = 2;
constexpr int GEMM_RING = GEMM_STAGES * GEMM_STAGE_BYTES;
constexpr int SMEM_BYTES = GEMM_RING > STAGE_BYTES ? GEMM_RING : STAGE_BYTES;
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

// Bulk copy (the TMA engine's linear form) of `bytes` from global to shared
// memory, completing as transaction bytes on the mbarrier `bar`; both
// addresses 16-byte aligned, `bytes` a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :
        : "r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(bar)
                 : "memory");
}

// Rows of X (R x K, row stride ld floats, K a multiple of 16, rows 16-byte
// aligned) split into TF32 halves in the order tc_gemm_kernel streams them:
// per 128-row block and K = 8 slab, the block's 4 KB of hi words, then its
// 4 KB of lo words, each in the canonical core-matrix order of slab_off.
// Rows R .. Rpad - 1 (Rpad a multiple of 128) are written as zeros.
__global__ void tf32_split_kernel(const float *__restrict__ X, int64_t R, int ld, int K,
                                  int64_t Rpad, uint32_t *__restrict__ out)
{
    const int kq = K / 4;
    const int nslab = K / 8;
    uint8_t *ob = reinterpret_cast<uint8_t *>(out);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Rpad * kq;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / kq;
        const int k = (int)(i - r * kq) * 4;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < R) x = __ldg(reinterpret_cast<const float4 *>(X + r * ld + k));
        const float v[4] = {x.x, x.y, x.z, x.w};
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h[j] = to_tf32(v[j]);
            l[j] = to_tf32(v[j] - __uint_as_float(h[j]));
        }
        uint8_t *o = ob + ((r >> 7) * nslab + (k >> 3)) * 2 * SLAB + slab_off((int)(r & 127), k & 7);
        *reinterpret_cast<uint4 *>(o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(o + SLAB) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// C[i][j] = max(an[i] + bn[j] - 2 (A B^T)[i][j], 0) from the TF32 halves of
// A (M rows) and B laid out by tf32_split_kernel, and (summary != NULL) the
// tile summary of C used by the top-nprobe select: per row of the 128 x 128
// output tile its four smallest entries, packed as dist_key with the column
// within the tile in the low 7 bits (SUMMARY_TILE = TN).
//
// Thread 0 drives a ring of GEMM_STAGES stages of K = 16: it bulk-copies a
// stage's A and B halves (16 KB each, contiguous in the split layout) onto
// the stage's `full` barrier, waits for them, issues the stage's 2 x 3 MMAs
// (per K = 8 slab: lo*hi, hi*lo, hi*hi, the order of the FP32 accumulation)
// and commits them to the stage's `empty` barrier; the stage the previous
// step used is refilled as soon as its MMAs have completed, so that the
// tensor pipe always has the next step's operands.  A final commit to `done`
// releases the epilogue.  Every wait is bounded; on time-out the kernel sets
// the error word, waits (bounded by 1 s of device time) for the copies and
// MMAs already issued, frees its tensor memory and returns.
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const uint32_t *__restrict__ As, int64_t M, const uint32_t *__restrict__ Bs,
                   int Kd, float *__restrict__ C, int ldc, int Nout, const float *__restrict__ an,
                   const float *__restrict__ bn, unsigned *err, unsigned *__restrict__ summary)
{
    static_assert(TN == SUMMARY_TILE, "one summary tile per output tile");
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t full[GEMM_STAGES], empty[GEMM_STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;
    const int nslab = Kd / 8, nsteps = nslab / GEMM_KS;
    const uint8_t *ga = reinterpret_cast<const uint8_t *>(As) + (size_t)blockIdx.x * nslab * 2 * SLAB;
    const uint8_t *gb = reinterpret_cast<const uint8_t *>(Bs) + (size_t)blockIdx.y * nslab * 2 * SLAB;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(&tmem_slot)), "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < GEMM_STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(smem_addr(&full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(smem_addr(&empty[i])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(smem_addr(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (tid == 0) {
        auto produce = [&](int step) {
            const int st = step % GEMM_STAGES;
            const uint32_t fb = smem_addr(&full[st]);
            const uint32_t dst = smem_addr(sm + st * GEMM_STAGE_BYTES);
            mbar_expect(fb, GEMM_STAGE_BYTES);
            bulk_g2s(dst, ga + (size_t)step * GEMM_OPND_BYTES, GEMM_OPND_BYTES, fb);
            bulk_g2s(dst + GEMM_OPND_BYTES, gb + (size_t)step * GEMM_OPND_BYTES, GEMM_OPND_BYTES, fb);
        };
        int produced = nsteps < GEMM_STAGES ? nsteps : GEMM_STAGES;
        for (int p = 0; p < produced; ++p) produce(p);
        int consumed = 0;            // steps whose copies have been waited for
        bool ok = true;
        for (int step = 0; step < nsteps && ok; ++step) {
            const int st = step % GEMM_STAGES;
            if (!mbar_wait(smem_addr(&full[st]), (uint32_t)(step / GEMM_STAGES) & 1u)) {
                ok = false;
                break;
            }
            consumed = step + 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint8_t *Ab = sm + st * GEMM_STAGE_BYTES, *Bb = Ab + GEMM_OPND_BYTES;
#pragma unroll
            for (int j = 0; j < GEMM_KS; ++j) {
                const uint64_t ah = make_desc(smem_addr(Ab + j * 2 * SLAB));
                const uint64_t al = make_desc(smem_addr(Ab + j * 2 * SLAB + SLAB));
                const uint64_t bh = make_desc(smem_addr(Bb + j * 2 * SLAB));
                const uint64_t bl = make_desc(smem_addr(Bb + j * 2 * SLAB + SLAB));
                mma_tf32(tmem, al, bh, (step > 0 || j > 0) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, 1u);
                mma_tf32(tmem, ah, bh, 1u);
            }
            mma_commit(smem_addr(&empty[st]));
            // refill the stage of the previous step once its MMAs are done
            if (step >= 1 && produced < nsteps) {
                const int prev = step - 1;
                if (!mbar_wait(smem_addr(&empty[prev % GEMM_STAGES]),
                               (uint32_t)(prev / GEMM_STAGES) & 1u)) {
                    ok = false;
                    break;
                }
                produce(produced);
                ++produced;
            }
        }
        mma_commit(smem_addr(&done));        // every MMA issued above
        if (!ok) {
            s_ok = 0;
            atomicOr(err, ERR_MMA_TIMEOUT);
            // copies still in flight write into this block's shared memory:
            // wait for them before anyone leaves
            for (int step = consumed; step < produced; ++step)
                if (!mbar_wait_ns(smem_addr(&full[step % GEMM_STAGES]),
                                  (uint32_t)(step / GEMM_STAGES) & 1u, DRAIN_NS))
                    atomicOr(err, ERR_MMA_DRAIN);
        }
    }
    // every thread: the accumulator is final once `done` completes
    bool ok = mbar_wait_ns(smem_addr(&done), 0u, DRAIN_NS);
    __syncthreads();
    if (!ok && tid == 0) atomicOr(err, ERR_MMA_DRAIN);
    ok = __syncthreads_and(ok && s_ok);
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // Each warp reads its 32 accumulator rows (lane = row) and stages the
        // finished 32 x 128 distances in the (now idle) operand ring, rows
        // 132 floats apart (float4 writes of 8 lanes hit distinct banks),
        // then writes every row as one coalesced 512-byte run.
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        const float rn = (row < M) ? an[row] : 0.f;
        float *stage = reinterpret_cast<float *>(sm) + warp * 32 * (TN + 4);
        unsigned t0 = ~0u, t1 = ~0u, t2 = ~0u, t3 = ~0u;   // the row's four smallest
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
            if (summary) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int cl = c0 + j;
                    keep4(n0 + cl < Nout ? (dist_key(o[j]) & ~SUMMARY_LOW) | (unsigned)cl : ~0u,
                          t0, t1, t2, t3);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(stage + lane * (TN + 4) + c0 + j) =
                    make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
        }
        if (summary && row < M)
            *reinterpret_cast<uint4 *>(summary + ((size_t)row * gridDim.y + blockIdx.y) * 4) =
                make_uint4(t0, t1, t2, t3);
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

int64_t tf32_split_words(int64_t rows, int K)
{
    return (rows + TM - 1) / TM * TM * (int64_t)K * 2;
}

cudaError_t launch_tf32_split(const float *X, int64_t R, int ld, int K, uint32_t *out, cudaStream_t s)
{
    if (R <= 0) return cudaSuccess;
    if (K % 16 != 0 || ld % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(out) & 15) != 0)
        return cudaErrorInvalidValue;
    const int64_t Rpad = (R + TM - 1) / TM * TM;
    int64_t blocks = (Rpad * (K / 4) + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    tf32_split_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, R, ld, K, Rpad, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const uint32_t *As, int64_t M, const uint32_t *Bs, int Kd, float *C,
                           int ldc, int Nout, const float *an, const float *bn, unsigned *err,
                           cudaStream_t s, unsigned *summary)
{
    if (M <= 0 || Nout <= 0) return cudaSuccess;
    if ((M + TM - 1) / TM > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (!an || !bn || Kd <= 0 || Kd % (8 * GEMM_KS) != 0) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(As) & 15) != 0 || (reinterpret_cast<uintptr_t>(Bs) & 15) != 0)
        return cudaErrorInvalidValue;
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)((Nout + TN - 1) / TN));
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<<<grid, 128, SMEM_BYTES, s>>>(As, M, Bs, Kd, C, ldc, Nout, an, bn, err, summary);
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

namespace {

// ---- query rotation Y = X P^T on the tensor cores, FP32-accurate.
//
// Each value x of a row becomes the integer V = trunc(x 2^(bT - E)), E the
// exponent of the row's largest |x| (so |V| < 2^(bT)), and V is written as T
// signed digits of b bits, s_1 (most significant) .. s_T:
// x = sum_t s_t 2^(E - bt) up to the truncated remainder (below 2^(E - bT)).
// P's rows are split the same way once, at index build (digits p_u,
// exponents F).  Then
//   (X P^T)[r][c] = 2^(E_r + F_c) sum_L 2^(-bL) sum_{t + u = L} sum_k s_t[r][k] p_u[c][k],
// and each inner sum adds products of integers below 2^b in magnitude: with
// T Dp (2^b - 1)^2 < 2^24 every partial sum of a level is an integer an FP32
// accumulator holds exactly, in whatever order the tensor core adds.  The
// digit pairs of one level L are laid side by side along K (digits t of X
// against digits L - t of P), so one exact accumulation serves a level.
// Levels 2..Lmax are kept, Lmax chosen so that the others weigh below
// 2^(-bT) of the row and column scales (bT >= 28); each level is split along
// K into work units for parallelism.  The units' exact sums, each times its
// level's power of two (still exact in FP32), are added by compensated
// summation and the total is scaled by 2^(E_r + F_c).  The
// approach is the error-free splitting of matrix products of Ozaki, Ogita,
// Oishi and Rump (Numer. Algorithms, 2012), with one digit width.
constexpr int ROT_MAX_UNITS = 64;
constexpr int ROT_MAX_LEVEL = 16;

struct TcRot {
    const float *dig;          // M x T x Dp digits of X (rot_digits_kernel)
    int64_t M;
    int D, Dp;
    const int32_t *xexp;
    int b, T;
    const float *B;
    int64_t boff[ROT_MAX_LEVEL];
    int nz;
    int zL[ROT_MAX_UNITS], zk0[ROT_MAX_UNITS], zk1[ROT_MAX_UNITS];
    float *part;
    unsigned *err;
};

// Work units of the levels 2..Lmax (K' of level L: its digit pairs times Dp);
// returns their number (at most 24 units, by the K' per unit).
int rot_plan(int Dp, int T, int Lmax, TcRot &r)
{
    for (int kc = 512;; kc *= 2) {
        int n = 0;
        bool over = false;
        for (int L = 2; L <= Lmax && !over; ++L) {
            const int lo = L - T > 1 ? L - T : 1, hi = L - 1 < T ? L - 1 : T;
            const int kl = (hi - lo + 1) * Dp;
            for (int k0 = 0; k0 < kl; k0 += kc) {
                if (n >= ROT_MAX_UNITS) {
                    over = true;
                    break;
                }
                r.zL[n] = L;
                r.zk0[n] = k0;
                r.zk1[n] = k0 + kc < kl ? k0 + kc : kl;
                ++n;
            }
        }
        if (!over && n <= 24) {
            r.nz = n;
            return n;
        }
        if (kc > (1 << 20)) return -1;
    }
}

// Per row (one warp): E, the exponent of its largest |x| (x = m 2^E, m in
// [0.5, 1); 0 for a zero row), and its T digits, dig[r][(t - 1) Dp + k]
// (FP32 values of small integers; 0 for k >= D).
__global__ void rot_digits_kernel(const float *__restrict__ X, int64_t M, int D, int Dp, int b,
                                  int T, int32_t *__restrict__ xexp, float *__restrict__ dig)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long mask = (1ull << b) - 1ull;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < M;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float m = 0.f;
        for (int k = lane; k < D; k += 32) m = fmaxf(m, fabsf(X[r * D + k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        int E = 0;
        if (m > 0.f) frexpf(m, &E);
        if (lane == 0) xexp[r] = E;
        const int sh = b * T - E;
        // 2^sh as two exact factors (sh may exceed the FP32 exponent range)
        const float s1 = ldexpf(1.f, sh < 127 ? sh : 127), s2 = ldexpf(1.f, sh > 127 ? sh - 127 : 0);
        float *dr = dig + r * (int64_t)T * Dp;
        for (int k = lane; k < Dp; k += 32) {
            // |V| < 2^(bT) <= 2^32: 64-bit
            const long long V = k < D ? __float2ll_rz((X[r * D + k] * s1) * s2) : 0ll;
            const unsigned long long av = (unsigned long long)(V < 0 ? -V : V);
            for (int t = 1; t <= T; ++t) {
                const int d = (int)((av >> (b * (T - t))) & mask);
                dr[(int64_t)(t - 1) * Dp + k] = (float)(V < 0 ? -d : d);
            }
        }
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool full)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(full ? 16 : 0)
                 : "memory");
}

// One work unit (blockIdx.z: a level L and a K' range) of a 128 x 128 output
// tile: the digits t of X (K' block j holds digit max(1, L - T) + j, read
// from the precomputed digits) against digits L - t of P, one tcgen05.mma
// (kind::tf32; the digits are small integers, exact in TF32) per 8-wide K
// slab, with the exact partial sums written to part[z].  Operands reach
// shared memory by cp.async in a ROT_STAGES-deep ring, so the copies of the
// next k-steps overlap the MMAs of the current one.
constexpr int ROT_STAGES = 3;
constexpr int ROT_STAGE_BYTES = 2 * OPER;                 // A and B of one 32-wide k-step
constexpr int ROT_SMEM = ROT_STAGES * ROT_STAGE_BYTES > STAGE_BYTES ? ROT_STAGES * ROT_STAGE_BYTES
                                                                    : STAGE_BYTES;

__global__ void __launch_bounds__(128, 1) tc_rot_kernel(TcRot r)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t mbar[ROT_STAGES];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;
    const int z = blockIdx.z;
    const int L = r.zL[z], kb = r.zk0[z], ke = r.zk1[z];
    const int tlo = L - r.T > 1 ? L - r.T : 1, thi = L - 1 < r.T ? L - 1 : r.T;
    const int ldb = (thi - tlo + 1) * r.Dp;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(&tmem_slot)), "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < ROT_STAGES; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(smem_addr(&mbar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // A k-step moves 128 rows x 32 values of A (digits of queries m0..) and
    // of B (the level's digits of P rows n0..) as 16-byte chunks: chunk
    // c = tid + 128 j is row c / 8, values 4 (c % 8) .. +3, so the lanes of a
    // warp read 4 rows x 128 contiguous bytes per instruction.
    const int rsub = tid >> 3, csub = tid & 7;
    const float *asrc = r.dig + (int64_t)(tlo - 1) * r.Dp;
    const float *bsrc = r.B + r.boff[L];
    const int64_t astride = (int64_t)r.T * r.Dp;
    const int nsteps = (ke - kb + BK - 1) / BK;
    auto issue = [&](int step) {
        if (step < nsteps) {
            const int k = kb + step * BK + 4 * csub;      // K' ends on a multiple of 16
            const bool in = k < ke;
            uint8_t *Ab = sm + (step % ROT_STAGES) * ROT_STAGE_BYTES, *Bb = Ab + OPER;
            const uint32_t co = (uint32_t)(csub >> 1) * SLAB;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int row = rsub + 16 * j;
                const uint32_t o = co + slab_off(row, (4 * csub) & 7);
                const int64_t ar = m0 + row;
                const bool av = in && ar < r.M, bv = in && n0 + row < r.Dp;
                cp_async16(smem_addr(Ab + o), asrc + (av ? ar * astride + k : 0), av);
                cp_async16(smem_addr(Bb + o), bsrc + (bv ? (int64_t)(n0 + row) * ldb + k : 0), bv);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int i = 0; i < ROT_STAGES - 1; ++i) issue(i);

    uint32_t phases = 0;                                  // bit b: phase of mbar[b]
    int last = 0;                                         // buffer of the last commit
    bool ok = true;
    for (int i = 0; i < nsteps && ok; ++i) {
        asm volatile("cp.async.wait_group %0;" ::"n"(ROT_STAGES - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const int buf = i % ROT_STAGES;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint8_t *Ab = sm + buf * ROT_STAGE_BYTES, *Bb = Ab + OPER;
#pragma unroll
            for (int s = 0; s < BK / 8; ++s)
                mma_tf32(tmem, make_desc(smem_addr(Ab + s * SLAB)), make_desc(smem_addr(Bb + s * SLAB)),
                         (i > 0 || s > 0) ? 1u : 0u);
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                :
                : "r"(smem_addr(&mbar[buf]))
                : "memory");
        }
        last = buf;
        // the buffer of step i - 1 is refilled with step i + ROT_STAGES - 1
        // once its MMAs are done
        if (i > 0) {
            const int pb = (i - 1) % ROT_STAGES;
            ok = __syncthreads_and(mbar_wait(smem_addr(&mbar[pb]), (phases >> pb) & 1u));
            if (ok) phases ^= 1u << pb;
        }
        if (ok) issue(i + ROT_STAGES - 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (ok) {
        // the last step's MMAs
        ok = __syncthreads_and(mbar_wait(smem_addr(&mbar[last]), (phases >> last) & 1u));
        if (ok) phases ^= 1u << last;
    }
    if (!ok) {
        // as in tc_gemm_kernel: flag, then wait (bounded by time) for the
        // last committed batch -- MMAs complete in order, so every earlier
        // one is done when it is -- before tensor memory is released
        if (tid == 0) atomicOr(r.err, ERR_MMA_TIMEOUT);
        const bool drained = mbar_wait_ns(smem_addr(&mbar[last]), (phases >> last) & 1u, DRAIN_NS);
        if (!__syncthreads_and(drained) && tid == 0) atomicOr(r.err, ERR_MMA_DRAIN);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // each warp stages its 32 accumulator rows, then writes them row by
        // row as coalesced runs
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
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
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(stage + lane * (TN + 4) + c0 + j) =
                    make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        }
        __syncwarp();
        float *pz = r.part + (int64_t)z * r.M * r.Dp;
        for (int rr = 0; rr < 32; ++rr) {
            const int64_t grow = m0 + warp * 32 + rr;
            if (grow >= r.M) break;
            for (int c = lane; c < TN; c += 32)
                if (n0 + c < r.Dp) pz[grow * r.Dp + n0 + c] = stage[rr * (TN + 4) + c];
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

// Y[r][c] = 2^(E_r + F_c) sum_z part[z][r][c] 2^(-b L_z).  Each term is an
// integer below 2^24 times a power of two, so exact in FP32; the terms are
// added by Sum2 (TwoSum on the running sum, the errors added apart: as
// accurate as twice the working precision, Ogita, Rump and Oishi 2005), the
// two parts added and the total scaled by 2^(E_r + F_c) (0 for c >= D).
__global__ void rot_combine_kernel(TcRot r, const int32_t *__restrict__ fexp, float *__restrict__ Y)
{
    const int64_t total = r.M * r.Dp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / r.Dp;
        const int c = (int)(i - row * r.Dp);
        float hi = 0.f, lo = 0.f;
        for (int z = 0; z < r.nz; ++z) {
            const float v = ldexpf(r.part[(int64_t)z * total + i], -r.b * r.zL[z]);
            const float sum = hi + v, zz = sum - hi;
            lo += (hi - (sum - zz)) + (v - zz);
            hi = sum;
        }
        Y[i] = c < r.D ? ldexpf(hi + lo, r.xexp[row] + fexp[c]) : 0.f;
    }
}

}  // namespace

void tc_rot_params(int Dp, int *b, int *T, int *Lmax)
{
    *b = 0;
    *T = 0;
    *Lmax = 0;
    if (Dp > 1024) return;
    for (int bb = 8; bb >= 3; --bb) {
        const int tt = (28 + bb - 1) / bb;
        const int64_t lim = (int64_t)tt * Dp * ((1ll << bb) - 1) * ((1ll << bb) - 1);
        if (lim < (1ll << 24)) {
            // dropped levels weigh at most T Dp 2^(2b - b(Lmax + 1)) <= 2^(-bT)
            int lg = 0;
            while ((1ll << lg) < (int64_t)tt * Dp) ++lg;
            int lm = tt + 1 + (lg + bb - 1) / bb;
            if (lm > 2 * tt) lm = 2 * tt;
            *b = bb;
            *T = tt;
            *Lmax = lm;
            return;
        }
    }
}

int64_t tc_rot_scratch_floats(const Index *ix, int64_t rows)
{
    if (!ix->rot_ok) return 0;
    TcRot r;
    const int nz = rot_plan(ix->Dp, ix->rot_T, ix->rot_Lmax, r);
    return nz > 0 ? (int64_t)(nz + ix->rot_T) * rows * ix->Dp : 0;
}

cudaError_t rotate_queries_tc(const Index *ix, const float *X, int64_t nq, float *Y, float *part,
                              int64_t part_floats, int32_t *xexp, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    if (!ix->rot_ok || (nq + TM - 1) / TM > 0x7fffffffLL) return cudaErrorInvalidValue;
    TcRot r;
    r.D = ix->D;
    r.Dp = ix->Dp;
    r.b = ix->rot_b;
    r.T = ix->rot_T;
    r.B = ix->rot_B;
    for (int i = 0; i < ROT_MAX_LEVEL; ++i) r.boff[i] = ix->rot_boff[i];
    r.err = ix->err;
    const int nz = rot_plan(ix->Dp, ix->rot_T, ix->rot_Lmax, r);
    if (nz <= 0) return cudaErrorInvalidValue;
    // rows per pass: as many as the scratch holds (digits and partial sums)
    const int64_t per_row = (int64_t)(nz + ix->rot_T) * ix->Dp;
    int64_t chunk = part_floats / per_row;
    if (chunk < 1) return cudaErrorInvalidValue;
    if (chunk > TM && chunk < nq) chunk -= chunk % TM;
    cudaError_t e = cudaFuncSetAttribute(tc_rot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         ROT_SMEM);
    if (e != cudaSuccess) return e;
    for (int64_t r0 = 0; r0 < nq; r0 += chunk) {
        const int64_t m = nq - r0 < chunk ? nq - r0 : chunk;
        float *dig = part + (int64_t)nz * m * ix->Dp;
        int64_t blocks = (m * 32 + 255) / 256;
        if (blocks > 152 * 32) blocks = 152 * 32;
        rot_digits_kernel<<<(unsigned)blocks, 256, 0, s>>>(X + r0 * ix->D, m, ix->D, ix->Dp, r.b, r.T,
                                                            xexp + r0, dig);
        r.dig = dig;
        r.M = m;
        r.xexp = xexp + r0;
        r.part = part;
        dim3 grid((unsigned)((m + TM - 1) / TM), (unsigned)((ix->Dp + TN - 1) / TN), (unsigned)nz);
        tc_rot_kernel<<<grid, 128, ROT_SMEM, s>>>(r);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        int64_t cb = (m * ix->Dp + 255) / 256;
        if (cb > 152 * 32) cb = 152 * 32;
        rot_combine_kernel<<<(unsigned)cb, 256, 0, s>>>(r, ix->rot_F, Y + r0 * ix->Dp);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace adsx
