// Mixed-precision defect correction around the block-relaxation sweeps.
//
// The outer loop keeps the iterate u, the residual and its norm in FP64; the inner
// correction equation A c = r is relaxed in FP32 by the context's own sweeps (Sec. 2,
// Eq. blockiteration2, applied to the correction):
//   r = b - A u          FP64 arithmetic, stored as FP32 (fused cast), ||r|| in FP64
//   c = 0; m sweeps of the FP32 context on A c = r
//   u = u + c            FP64 accumulate (and c is re-zeroed in the same pass)
// until ||r||_2 / ||b||_2 <= rtol.  Only the norm crosses to the host (one read per outer
// step).
#include <cmath>

#include "brs_internal.cuh"
#include "plane.cuh"

namespace {

__global__ void correct_kernel(double* __restrict__ u, float* __restrict__ c, long long n)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        u[t] += (double)c[t];
        c[t] = 0.0f;
    }
}

int read_norm(brs_ctx* c, cudaStream_t s, double* out)
{
    double h = 0.0;
    cudaError_t e = cudaMemcpyAsync(&h, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    *out = std::sqrt(h);
    return BRS_OK;
}

}  // namespace

extern "C" int brsmooth_defect_correction(brs_ctx* outer, brs_ctx* inner, double* u,
                                          const double* b, double rtol, int inner_sweeps,
                                          int max_outer, int* outer_done, double* rel_residual,
                                          double* history, void* stream)
{
    cudaGetLastError();  // start from a clean launch-error state
    if (!outer || !inner || !u || !b || inner_sweeps < 1 || max_outer < 0 || !(rtol >= 0.0))
        return BRS_ERR_ARG;
    if (outer->batch || inner->batch || outer->p.dtype != BRS_F64 || inner->p.dtype != BRS_F32)
        return BRS_ERR_ARG;
    const brs_params &po = outer->p, &pi = inner->p;
    if (po.nx != pi.nx || po.ny != pi.ny || po.nz != pi.nz || po.ax != pi.ax || po.ay != pi.ay ||
        po.az != pi.az)
        return BRS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(u) & 15u) || (reinterpret_cast<uintptr_t>(b) & 15u))
        return BRS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = outer->cells;
    cudaError_t e = cudaSuccess;
    if (!inner->dc_r)
        e = cudaMalloc(&inner->dc_r, sizeof(float) * n);
    if (e == cudaSuccess && !inner->dc_c)
        e = cudaMalloc(&inner->dc_c, sizeof(float) * n);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(inner->dc_c, 0, sizeof(float) * n, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    int rc = norm2sq_launch(outer, b, s);
    double nb = 0.0;
    if (rc == BRS_OK)
        rc = read_norm(outer, s, &nb);
    if (rc != BRS_OK)
        return rc;
    if (nb == 0.0)
        nb = 1.0;
    int it = 0;
    double rel = 0.0;
    int blocks = 152 * 8;
    while (true) {
        rc = residual_launch_f32out(outer, u, b, inner->dc_r, s);
        double nr = 0.0;
        if (rc == BRS_OK)
            rc = read_norm(outer, s, &nr);
        if (rc != BRS_OK)
            return rc;
        rel = nr / nb;
        if (history)
            history[it] = rel;
        if (rel <= rtol || it >= max_outer)
            break;
        // c starts from zero: a plane context in the x-sine form skips c's transform
        rc = inner->plane ? plane_modes_sweep(inner, inner->dc_c, inner->dc_r, inner_sweeps, s,
                                              true)
                          : BRS_ERR_UNSUPPORTED;
        if (rc == BRS_ERR_UNSUPPORTED)
            rc = brsmooth_sweep(inner, inner->dc_c, inner->dc_r, inner_sweeps, stream);
        if (rc != BRS_OK)
            return rc;
        correct_kernel<<<blocks, 256, 0, s>>>(u, inner->dc_c, n);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        ++it;
    }
    if (outer_done)
        *outer_done = it;
    if (rel_residual)
        *rel_residual = rel;
    return BRS_OK;
}
