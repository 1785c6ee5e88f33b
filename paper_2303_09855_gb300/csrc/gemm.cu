// gemm.cu -- the two dense contractions of the path on CUDA cores (FP32):
//   rotation   Y = X P^T        (Sec. 3.1, y = P x; index vectors, centroids, queries)
//   distances  D2[q][c] = sum_j (q'_j - c'_j)^2   (Sec. 2.2.2, centroid ranking)
// Both operands are row-major with the contraction dimension contiguous.
// A 64 x 64 output tile per 256-thread block, 4 x 4 per thread, k-steps of 16
// staged through shared memory.  Out-of-range rows/columns/k read as zero.
#include "adsx_internal.cuh"

namespace adsx {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <bool DIST>
__global__ void __launch_bounds__(256) nt_gemm_kernel(const float *__restrict__ A, int64_t M,
                                                      int lda, const float *__restrict__ B,
                                                      int Nb, int ldb, int Kd,
                                                      float *__restrict__ C, int ldc, int Nout)
{
    __shared__ __align__(16) float As[TK][TM + 4];
    __shared__ __align__(16) float Bs[TK][TN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < Kd; k0 += TK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int e = tid + i * 256;
            int r = e >> 4, kk = e & 15;
            int64_t gm = m0 + r;
            int gk = k0 + kk;
            As[kk][r] = (gm < M && gk < Kd) ? A[gm * lda + gk] : 0.f;
            int gn = n0 + r;
            Bs[kk][r] = (gn < Nb && gk < Kd) ? B[(int64_t)gn * ldb + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float4 a4 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            float4 b4 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            float a[4] = {a4.x, a4.y, a4.z, a4.w};
            float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (DIST) {
                        float t = a[i] - b[j];
                        acc[i][j] = fmaf(t, t, acc[i][j]);
                    } else {
                        acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                    }
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx * 4 + j;
            if (gn < Nout) C[gm * ldc + gn] = acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_nt_gemm(const float *A, int64_t M, int lda, const float *B, int Nb,
                           int ldb, int Kd, float *C, int ldc, int Nout, bool dist,
                           cudaStream_t s)
{
    if (M <= 0 || Nout <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)((Nout + TN - 1) / TN));
    if (dist)
        nt_gemm_kernel<true><<<grid, 256, 0, s>>>(A, M, lda, B, Nb, ldb, Kd, C, ldc, Nout);
    else
        nt_gemm_kernel<false><<<grid, 256, 0, s>>>(A, M, lda, B, Nb, ldb, Kd, C, ldc, Nout);
    return cudaGetLastError();
}

}  // namespace adsx
