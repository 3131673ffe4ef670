// Residual r = b - A u (the r^k of Eq. blockiteration2, Sec. 2) and ||r||_2.
//
// One thread per cell in a grid-stride loop over a fixed grid, so every CTA's partial
// sum of squares covers a fixed set of cells; partials are FP64 and summed by one CTA in
// a fixed order, which makes the norm bitwise reproducible run to run.
#include "brs_internal.cuh"

namespace {

constexpr int kResThreads = 256;

template <typename T, typename TR>
__global__ void __launch_bounds__(kResThreads) residual_kernel(const T* __restrict__ u,
                                                               const T* __restrict__ b,
                                                               TR* __restrict__ r, int nx, int ny,
                                                               int nz, double ax, double ay,
                                                               double az, double* partials)
{
    const long long n = (long long)nx * ny * nz;
    const long long plane = (long long)nx * ny;
    const T cx = (T)ax, cy = (T)ay, cz = (T)az, dg = (T)(2.0 * (ax + ay + az));
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx);
        const long long jk = t / nx;
        const int j = (int)(jk % ny);
        const int k = (int)(jk / ny);
        const T sx = (i > 0 ? u[t - 1] : T(0)) + (i + 1 < nx ? u[t + 1] : T(0));
        const T sy = (j > 0 ? u[t - nx] : T(0)) + (j + 1 < ny ? u[t + nx] : T(0));
        const T sz = (k > 0 ? u[t - plane] : T(0)) + (k + 1 < nz ? u[t + plane] : T(0));
        // b - A u = b - d u + ax sx + ay sy + az sz
        const T rv = fma(cz, sz, fma(cy, sy, fma(cx, sx, fma(-dg, u[t], b[t]))));
        if (r)
            r[t] = (TR)rv;
        acc += (double)rv * (double)rv;
    }
    // block reduction in a fixed tree
    __shared__ double red[kResThreads / 32];
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kResThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && partials)
            partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kResThreads) sum_partials_kernel(const double* partials,
                                                                   int n, double* out)
{
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x)
        acc += partials[t];
    __shared__ double red[kResThreads / 32];
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kResThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0)
            *out = v;
    }
}

}  // namespace

int residual_setup(brs_ctx* c)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->npartials = (sms > 0 ? sms : 152) * 8;
    cudaError_t e = cudaMalloc(&c->partials, sizeof(double) * (c->npartials + 1));
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    c->norm_dev = c->partials + c->npartials;
    return BRS_OK;
}

template <typename T, typename TR>
int residual_run(brs_ctx* c, const T* u, const T* b, TR* r, bool want_norm, double ax,
                 double ay, double az, cudaStream_t s)
{
    const brs_params& p = c->p;
    const long long n = c->cells;
    long long need = (n + kResThreads - 1) / kResThreads;
    int blocks = (int)(need < c->npartials ? need : c->npartials);
    if (blocks < 1)
        blocks = 1;
    double* part = want_norm ? c->partials : nullptr;
    residual_kernel<T, TR><<<blocks, kResThreads, 0, s>>>(u, b, r, p.nx, p.ny, p.nz, ax, ay, az,
                                                          part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    if (want_norm) {
        sum_partials_kernel<<<1, kResThreads, 0, s>>>(c->partials, blocks, c->norm_dev);
        e = cudaGetLastError();
    }
    return brs_cuda_status(e);
}

int residual_launch(brs_ctx* c, const void* u, const void* b, void* r, bool want_norm,
                    cudaStream_t s)
{
    const brs_params& p = c->p;
    if (p.dtype == BRS_F64)
        return residual_run<double, double>(c, (const double*)u, (const double*)b, (double*)r,
                                            want_norm, p.ax, p.ay, p.az, s);
    return residual_run<float, float>(c, (const float*)u, (const float*)b, (float*)r, want_norm,
                                      p.ax, p.ay, p.az, s);
}

int residual_launch_f32out(brs_ctx* c, const double* u, const double* b, float* r,
                           cudaStream_t s)
{
    const brs_params& p = c->p;
    return residual_run<double, float>(c, u, b, r, true, p.ax, p.ay, p.az, s);
}

int norm2sq_launch(brs_ctx* c, const void* x, cudaStream_t s)
{
    // with zero coefficients the residual kernel returns b itself: ||x||^2 into norm_dev
    if (c->p.dtype == BRS_F64)
        return residual_run<double, double>(c, (const double*)x, (const double*)x, nullptr, true,
                                            0.0, 0.0, 0.0, s);
    return residual_run<float, float>(c, (const float*)x, (const float*)x, nullptr, true, 0.0,
                                      0.0, 0.0, s);
}
