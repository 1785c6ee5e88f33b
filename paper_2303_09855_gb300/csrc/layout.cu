// layout.cu -- index-phase scatter of rotated vectors into the
// dimension-blocked per-cluster layout (Sec. 5.2 IVF++: the first dims of all
// candidates stored together; here every 16-dim block of a cluster is stored
// together, so any delta_d that is a multiple of 16 reads contiguous runs).
#include "adsx_internal.cuh"

namespace adsx {
namespace {

// One thread per (vector, 16-dim block): a 64-byte row piece read from the
// row-major rotated matrix Y (coalesced along the row) and written to its
// block of its cluster.
__global__ void scatter_layout_kernel(const float *__restrict__ Y, int64_t N, int Dp,
                                      const int32_t *__restrict__ assign,
                                      const int64_t *__restrict__ pos_of_id,
                                      const int64_t *__restrict__ off, float *__restrict__ data)
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
        const int64_t m = pos_of_id[id] - o;
        const float4 *src = reinterpret_cast<const float4 *>(Y + id * Dp + b * BLK);
        float4 *dst = reinterpret_cast<float4 *>(data + o * Dp + (int64_t)b * n * BLK + m * BLK);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = src[i];
    }
}

}  // namespace

cudaError_t launch_scatter_layout(const float *Y, int64_t N, int Dp, const int32_t *assign,
                                  const int64_t *pos_of_id, const int64_t *off, float *data,
                                  cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    int64_t total = N * (Dp / BLK);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    scatter_layout_kernel<<<(unsigned)blocks, 256, 0, s>>>(Y, N, Dp, assign, pos_of_id, off,
                                                           data);
    return cudaGetLastError();
}

}  // namespace adsx
