// Measurement helper: a kernel bound by FP64 fused multiply-adds, used to measure the FP64
// rate that the FP64 sweeps are judged against (their roof is FP64 operations, not bytes).
#include "brs_internal.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent FMA chains per thread

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_probe(double* out, int iters,
                                                               double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q)
        x[q] = (double)(threadIdx.x + q);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q)
            x[q] = fma(x[q], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q)
        s += x[q];
    out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int brsmooth_probe_fp64_fma(double* out, int blocks, int iters, void* stream)
{
    cudaGetLastError();
    if (!out || blocks < 1 || iters < 1)
        return BRS_ERR_ARG;
    fp64_fma_probe<<<blocks, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        out, iters, 0.999999, 1e-7);
    return brs_cuda_status(cudaGetLastError());
}
