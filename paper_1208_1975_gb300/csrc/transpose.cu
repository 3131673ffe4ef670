// Axis permutations of a grid, for y-line and z-line blocks: a y-line (z-line) sweep is an
// x-line sweep of the grid whose fastest axis is y (z), with the coefficients permuted with
// the axes.  Both permutations are batches of 2D transposes:
//   y lines: for every plane k, [j][i] -> [i][j]            (batch k)
//   z lines: for every row j,   [k][i] -> [i][k] at j nx nz (batch j)
// The kernel moves one 32 x 32 tile per CTA through shared memory (one padded column against
// bank conflicts): reads run along the source's contiguous axis, writes along the
// destination's.
#include "brs_internal.cuh"

namespace {

constexpr int kTile = 32;
constexpr int kRows = 8;  // thread rows per CTA; each thread moves kTile / kRows elements

// dst[b * db + c * dc + r] = src[b * sb + r * sr + c] for r < R, c < C
template <typename T>
__global__ void __launch_bounds__(kTile * kRows) transpose_kernel(const T* __restrict__ src,
                                                                   T* __restrict__ dst, int R,
                                                                   int C, long long sr,
                                                                   long long sb, long long dc,
                                                                   long long db)
{
    __shared__ T tile[kTile][kTile + 1];
    const long long bsrc = (long long)blockIdx.z * sb, bdst = (long long)blockIdx.z * db;
    const int c0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int q = 0; q < kTile; q += kRows) {
        const int r = r0 + ty + q, c = c0 + tx;
        if (r < R && c < C)
            tile[ty + q][tx] = src[bsrc + r * sr + c];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kTile; q += kRows) {
        const int c = c0 + ty + q, r = r0 + tx;
        if (r < R && c < C)
            dst[bdst + c * dc + r] = tile[tx][ty + q];
    }
}

}  // namespace

int transpose_launch(int dtype, const void* src, void* dst, int R, int C, int batch,
                     long long sr, long long sb, long long dc, long long db, cudaStream_t s)
{
    if (R <= 0 || C <= 0 || batch <= 0)
        return BRS_OK;
    if (batch > 65535)
        return BRS_ERR_UNSUPPORTED;
    const dim3 grid((C + kTile - 1) / kTile, (R + kTile - 1) / kTile, batch);
    const dim3 block(kTile, kRows);
    if (dtype == BRS_F64)
        transpose_kernel<double><<<grid, block, 0, s>>>(static_cast<const double*>(src),
                                                        static_cast<double*>(dst), R, C, sr,
                                                        sb, dc, db);
    else
        transpose_kernel<float><<<grid, block, 0, s>>>(static_cast<const float*>(src),
                                                       static_cast<float*>(dst), R, C, sr, sb,
                                                       dc, db);
    return brs_cuda_status(cudaGetLastError());
}
