// layout.cu -- index-phase scatter of rotated vectors into the
// dimension-blocked per-cluster layout (Sec. 5.2 IVF++: the first dims of all
// candidates stored together; here every 16-dim block of a cluster is stored
// together, so any delta_d that is a multiple of 16 reads contiguous runs).
// 16-bit storage types also get an FP32 copy of each rotated row and its
// norm, in CSR order, for the exact recheck of candidates reaching d = D.
#include "adsx_internal.cuh"

namespace adsx {
namespace {

__device__ __forceinline__ void store16(float *dst, const float *v)
{
    float4 *d = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

__device__ __forceinline__ void store16(__nv_bfloat16 *dst, const float *v)
{
    __nv_bfloat162 h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = *reinterpret_cast<uint4 *>(&h[0]);
    d[1] = *reinterpret_cast<uint4 *>(&h[4]);
}

__device__ __forceinline__ void store16(__half *dst, const float *v)
{
    __half2 h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = *reinterpret_cast<uint4 *>(&h[0]);
    d[1] = *reinterpret_cast<uint4 *>(&h[4]);
}

// One thread per (vector, 16-dim block): a 64-byte piece of the row-major
// rotated matrix Y (coalesced along the row) written to its block of its
// cluster (converted to the storage type).
template <typename T>
__global__ void scatter_layout_kernel(const float *__restrict__ Y, int64_t N, int Dp,
                                      const int32_t *__restrict__ assign,
                                      const int64_t *__restrict__ pos_of_id,
                                      const int64_t *__restrict__ off, T *__restrict__ data,
                                      float *__restrict__ rows32)
{
    const int nblk = Dp / BLK;
    const int64_t total = N * nblk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t id = e / nblk;
        const int b = (int)(e - id * nblk);
        const int c = assign[id];
        const int64_t o = off[c];
        const int64_t n = off[c + 1] - o;
        const int64_t p = pos_of_id[id];
        const int64_t m = p - o;
        float v[16];
        const float4 *src = reinterpret_cast<const float4 *>(Y + id * Dp + b * BLK);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float4 t = src[i];
            v[4 * i] = t.x;
            v[4 * i + 1] = t.y;
            v[4 * i + 2] = t.z;
            v[4 * i + 3] = t.w;
        }
        store16(data + o * Dp + (int64_t)b * n * BLK + m * BLK, v);
        if (rows32) store16(rows32 + p * Dp + b * BLK, v);
    }
}

// ||y|| of each FP32 row (CSR order), one warp per row.
__global__ void row_norms_kernel(const float *__restrict__ rows32, int64_t N, int Dp,
                                 float *__restrict__ norms)
{
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        for (int j = lane; j < Dp; j += 32) {
            float x = rows32[r * Dp + j];
            s = fmaf(x, x, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) norms[r] = sqrtf(s);
    }
}

}  // namespace

cudaError_t launch_scatter_layout(const float *Y, int64_t N, int Dp, const int32_t *assign,
                                  const int64_t *pos_of_id, const int64_t *off, void *data,
                                  int storage, float *rows32, float *norms, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    int64_t total = N * (Dp / BLK);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (storage == ADSX_F32)
        scatter_layout_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(
            Y, N, Dp, assign, pos_of_id, off, static_cast<float *>(data), nullptr);
    else if (storage == ADSX_BF16)
        scatter_layout_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(
            Y, N, Dp, assign, pos_of_id, off, static_cast<__nv_bfloat16 *>(data), rows32);
    else
        scatter_layout_kernel<__half><<<(unsigned)blocks, 256, 0, s>>>(
            Y, N, Dp, assign, pos_of_id, off, static_cast<__half *>(data), rows32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || storage == ADSX_F32) return e;
    int64_t nb = (N * 32 + 255) / 256;
    if (nb > 152 * 64) nb = 152 * 64;
    row_norms_kernel<<<(unsigned)nb, 256, 0, s>>>(rows32, N, Dp, norms);
    return cudaGetLastError();
}

}  // namespace adsx

namespace adsx {
namespace {

// Rotation Y = X P^T (y = P x, Sec. 3.1) with compensated FP32 dot products:
// Dot2 of Ogita, Rump & Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 2005).  Each product is split exactly by TwoProduct (h = a*b,
// r = fma(a, b, -h)), the running sum by TwoSum (Knuth), and the errors are
// summed separately, so y is as accurate as if computed in twice the working
// precision and then rounded once to FP32.
// 64 x 64 (or 32 x 32) output tile per 256-thread block, 4 x 4 (2 x 2) per
// thread, k-steps of 16; neighbouring outputs of a thread go through the
// same operations as packed FP32 pairs.

// Packed FP32 pair arithmetic (sm_100+ f32x2: each element rounded as the
// scalar instruction would be, two elements per instruction).
__device__ __forceinline__ float2 f2_op_add(float2 a, float2 b)
{
    float2 r;
    asm("{\n .reg .b64 av, bv, rv;\n mov.b64 av, {%2, %3};\n mov.b64 bv, {%4, %5};\n"
        " add.rn.f32x2 rv, av, bv;\n mov.b64 {%0, %1}, rv;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_op_sub(float2 a, float2 b)
{
    float2 r;
    asm("{\n .reg .b64 av, bv, rv;\n mov.b64 av, {%2, %3};\n mov.b64 bv, {%4, %5};\n"
        " sub.rn.f32x2 rv, av, bv;\n mov.b64 {%0, %1}, rv;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_op_mul(float2 a, float2 b)
{
    float2 r;
    asm("{\n .reg .b64 av, bv, rv;\n mov.b64 av, {%2, %3};\n mov.b64 bv, {%4, %5};\n"
        " mul.rn.f32x2 rv, av, bv;\n mov.b64 {%0, %1}, rv;\n}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_op_fma(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{\n .reg .b64 av, bv, cv, rv;\n mov.b64 av, {%2, %3};\n mov.b64 bv, {%4, %5};\n"
        " mov.b64 cv, {%6, %7};\n fma.rn.f32x2 rv, av, bv, cv;\n mov.b64 {%0, %1}, rv;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// One Dot2 step for two outputs sharing the factor a: the products a*b.x and
// a*b.y split exactly (TwoProduct: h = a*b, r = fma(a, b, -h), taken here as
// r = -fma(-a, b, h), the same value), h added to hi by TwoSum, the errors
// q + r into lo -- element by element the scalar sequence.
__device__ __forceinline__ void dot2_pair(float a, float2 b, float2 &hi, float2 &lo)
{
    const float2 aa = make_float2(a, a), na = make_float2(-a, -a);
    const float2 h = f2_op_mul(aa, b);
    const float2 t = f2_op_fma(na, b, h);          // -r
    const float2 s = f2_op_add(hi, h);
    const float2 z = f2_op_sub(s, hi);
    const float2 e = f2_op_add(f2_op_sub(hi, f2_op_sub(s, z)), f2_op_sub(h, z));
    hi = s;
    lo = f2_op_add(lo, f2_op_sub(e, t));           // lo + (q + r)
}

template <int T>
__global__ void __launch_bounds__(256) rotate_dot2_kernel(const float *__restrict__ X, int64_t N,
                                                          int D, const float *__restrict__ P,
                                                          int ldp, float *__restrict__ Y, int Dp)
{
    constexpr int TM = T / 16;          // outputs per thread along each side
    __shared__ float Xs[16][T + 4];
    __shared__ float Ps[16][T + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * T;
    const int c0 = blockIdx.y * T;
    float2 hi[TM][TM / 2], lo[TM][TM / 2];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM / 2; ++j) hi[i][j] = lo[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < D; k0 += 16) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int e = tid + i * 256, r = e >> 4, kk = e & 15;
            const int64_t gr = r0 + r;
            const int gk = k0 + kk, gc = c0 + r;
            Xs[kk][r] = (gr < N && gk < D) ? X[gr * D + gk] : 0.f;
            Ps[kk][r] = (gc < D && gk < D) ? P[(int64_t)gc * ldp + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            float a[TM], b[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = Xs[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TM; ++j) b[j] = Ps[kk][tx * TM + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM / 2; ++j)
                    dot2_pair(a[i], make_float2(b[2 * j], b[2 * j + 1]), hi[i][j], lo[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gr = r0 + ty * TM + i;
        if (gr >= N) continue;
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            const int gc = c0 + tx * TM + j;
            const float2 h = hi[i][j / 2], l = lo[i][j / 2];
            if (gc < Dp) Y[gr * Dp + gc] = (j & 1) ? h.y + l.y : h.x + l.x;
        }
    }
}

}  // namespace

cudaError_t launch_rotate(const float *X, int64_t N, int D, const float *P, int ldp, float *Y,
                          int Dp, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    if ((N + 63) / 64 > 0x7fffffffLL) return cudaErrorInvalidValue;
    // 64 x 64 output tiles, or 32 x 32 ones when the former would give fewer
    // than about 8 blocks per SM (a query batch; each output is summed in the
    // same order either way)
    const int64_t b64 = ((N + 63) / 64) * ((Dp + 63) / 64);
    if (b64 >= 8 * 152) {
        dim3 grid((unsigned)((N + 63) / 64), (unsigned)((Dp + 63) / 64));
        rotate_dot2_kernel<64><<<grid, 256, 0, s>>>(X, N, D, P, ldp, Y, Dp);
    } else {
        dim3 grid((unsigned)((N + 31) / 32), (unsigned)((Dp + 31) / 32));
        rotate_dot2_kernel<32><<<grid, 256, 0, s>>>(X, N, D, P, ldp, Y, Dp);
    }
    return cudaGetLastError();
}

}  // namespace adsx

// ---- cosine / inner-product support (Sec. 8, extension (1)): rows scaled
// to unit norm, the constant centroid term of inner-product probing, and a
// row-order -> CSR-order scatter of per-row values.
namespace adsx {
namespace {

// One warp per row: the squared norm is accumulated in FP64, the row is
// scaled by the FP32 value of 1/||x||.
__global__ void __launch_bounds__(256) normalize_rows_kernel(float *X, int64_t N, int ld, int D,
                                                             float *norms, unsigned *zero_err)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N; r += nw) {
        float *x = X + r * ld;
        double s = 0.0;
        for (int j = lane; j < D; j += 32) s += (double)x[j] * (double)x[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double n = sqrt(s);
        if (lane == 0 && norms) norms[r] = (float)n;
        if (n > 0.0) {
            const float inv = (float)(1.0 / n);
            for (int j = lane; j < D; j += 32) x[j] *= inv;
        } else if (lane == 0 && zero_err) {
            atomicOr(zero_err, ERR_ZERO_ROW);
        }
    }
}

__global__ void __launch_bounds__(1024) fill_max_kernel(float *v, int n)
{
    __shared__ float wmax[32];
    float m = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, v[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) wmax[0] = m;
    }
    __syncthreads();
    m = wmax[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = m;
}

__global__ void scatter_f32_kernel(const float *__restrict__ src, const int64_t *__restrict__ pos,
                                   int64_t N, float *__restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[pos[i]] = src[i];
}

}  // namespace

cudaError_t launch_normalize_rows(float *X, int64_t N, int ld, int D, float *norms,
                                  unsigned *zero_err, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    const int64_t blocks = (N + 7) / 8;
    normalize_rows_kernel<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, s>>>(
        X, N, ld, D, norms, zero_err);
    return cudaGetLastError();
}

cudaError_t launch_fill_max(float *v, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_max_kernel<<<1, 1024, 0, s>>>(v, n);
    return cudaGetLastError();
}

cudaError_t launch_scatter_f32(const float *src, const int64_t *pos, int64_t N, float *dst,
                               cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    const int64_t blocks = (N + 255) / 256;
    scatter_f32_kernel<<<(unsigned)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, s>>>(src, pos,
                                                                                       N, dst);
    return cudaGetLastError();
}

}  // namespace adsx

// ---- Kac-walk rotation (Sec. 6.2.3: the random rotation in O(D log D)).
namespace adsx {
namespace {

// R rows per block live in shared memory; for each layer the block stages the
// layer's pairs and (c, s) and applies its disjoint Givens rotations to every
// row: (x_i, x_j) <- (c x_i - s x_j, s x_i + c x_j).
__global__ void __launch_bounds__(256) kac_rotate_kernel(const float *__restrict__ X, int64_t N,
                                                         int D, int ldx,
                                                         const int32_t *__restrict__ pairs,
                                                         const float *__restrict__ cs, int L,
                                                         float *__restrict__ Y, int ldy, int R)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int m = D / 2;
    float *xs = reinterpret_cast<float *>(smraw);               // R x D
    int *pr = reinterpret_cast<int *>(xs + (size_t)R * D);      // 2m
    float *cv = reinterpret_cast<float *>(pr + 2 * m);          // 2m
    for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < N; r0 += (int64_t)gridDim.x * R) {
        const int nr = (int)(N - r0 < R ? N - r0 : R);
        for (int idx = threadIdx.x; idx < nr * D; idx += blockDim.x) {
            const int r = idx / D, j = idx - r * D;
            xs[idx] = X[(r0 + r) * ldx + j];
        }
        for (int l = 0; l < L; ++l) {
            __syncthreads();            // rows loaded / previous layer applied
            for (int t = threadIdx.x; t < 2 * m; t += blockDim.x) {
                pr[t] = pairs[(size_t)l * 2 * m + t];
                cv[t] = cs[(size_t)l * 2 * m + t];
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < nr * m; idx += blockDim.x) {
                const int r = idx / m, t = idx - r * m;
                const int i = pr[2 * t], j = pr[2 * t + 1];
                const float c = cv[2 * t], s = cv[2 * t + 1];
                float *x = xs + (size_t)r * D;
                const float xi = x[i], xj = x[j];
                x[i] = fmaf(c, xi, -s * xj);
                x[j] = fmaf(s, xi, c * xj);
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nr * ldy; idx += blockDim.x) {
            const int r = idx / ldy, j = idx - r * ldy;
            Y[(r0 + r) * ldy + j] = j < D ? xs[(size_t)r * D + j] : 0.f;
        }
        __syncthreads();                // before the next rows overwrite xs
    }
}

}  // namespace

cudaError_t launch_kac_rotate(const float *X, int64_t N, int D, int ldx, const int32_t *pairs,
                              const float *cs, int L, float *Y, int Dp, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    const int m = D / 2;
    const size_t params = (size_t)2 * m * 8;
    int R = (int)(((size_t)64 << 10) > params ? (((size_t)64 << 10) - params) / ((size_t)D * 4) : 1);
    R = R < 1 ? 1 : (R > 64 ? 64 : R);
    const size_t smem = (size_t)R * D * 4 + params;
    cudaError_t e = cudaFuncSetAttribute(kac_rotate_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (N + R - 1) / R;
    if (grid > 152 * 8) grid = 152 * 8;
    kac_rotate_kernel<<<(unsigned)grid, 256, smem, s>>>(X, N, D, ldx, pairs, cs, L, Y, Dp, R);
    return cudaGetLastError();
}

}  // namespace adsx
