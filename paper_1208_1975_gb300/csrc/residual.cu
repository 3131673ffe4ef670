// Residual r = b - A u (the r^k of Eq. blockiteration2, Sec. 2) and ||r||_2.
//
// Rows of the grid in a grid-stride loop over a fixed grid, so every CTA's partial sum of
// squares covers a fixed set of cells; partials are FP64 and summed by one CTA in a fixed
// order, which makes the norm bitwise reproducible run to run.
#include "brs_internal.cuh"

namespace {

constexpr int kResThreads = 256;

// Four consecutive cells of a row from p (rem = cells left in the row, may be < 4); VEC:
// 16-byte vectors (rows and arrays 16-byte aligned, nx a multiple of 4).
template <typename T>
__device__ __forceinline__ void ld4(T (&v)[4], const T* p, int rem, bool vec)
{
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(p));
            v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
        } else {
            const double2 f0 = __ldg(reinterpret_cast<const double2*>(p));
            const double2 f1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
            v[0] = f0.x, v[1] = f0.y, v[2] = f1.x, v[3] = f1.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            v[q] = q < rem ? p[q] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4], int rem, bool vec)
{
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
            reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < rem)
                p[q] = v[q];
    }
}

// One warp per grid row (j, k) at a time, in a grid-stride loop over rows with a fixed
// grid, four cells per lane: no per-cell index division, and each CTA's partial sum of
// squares covers a fixed set of cells.  Squares of an FP32 residual are summed in FP32 over
// a lane's cells of one row and then in FP64 (the FP64 pipe is the narrow one on this part).
template <typename T, typename TR>
__global__ void __launch_bounds__(kResThreads) residual_kernel(const T* __restrict__ u,
                                                               const T* __restrict__ b,
                                                               TR* __restrict__ r, int nx, int ny,
                                                               int nz, double ax, double ay,
                                                               double az, double* partials,
                                                               bool vec)
{
    const long long plane = (long long)nx * ny;
    const long long nrows = (long long)ny * nz;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const T cx = (T)ax, cy = (T)ay, cz = (T)az, dg = (T)(2.0 * (ax + ay + az));
    double acc = 0.0;
    for (long long row = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); row < nrows;
         row += (long long)gridDim.x * wpb) {
        const int k = (int)(row / ny), j = (int)(row - (long long)k * ny);
        const long long base = row * nx;
        T sq = T(0);  // FP32: the lane's squares over the row
        for (int i0 = 4 * lane; i0 < nx; i0 += 128) {
            const int rem = nx - i0;
            const T* pu = u + base + i0;
            T uc[4], bv[4], a[4], c[4];
            ld4(uc, pu, rem, vec);
            ld4(bv, b + base + i0, rem, vec);
            T sy[4], sz[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                sy[q] = sz[q] = T(0);
            if (j > 0) {
                ld4(a, pu - nx, rem, vec);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    sy[q] += a[q];
            }
            if (j + 1 < ny) {
                ld4(c, pu + nx, rem, vec);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    sy[q] += c[q];
            }
            if (k > 0) {
                ld4(a, pu - plane, rem, vec);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    sz[q] += a[q];
            }
            if (k + 1 < nz) {
                ld4(c, pu + plane, rem, vec);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    sz[q] += c[q];
            }
            const T left = i0 > 0 ? pu[-1] : T(0);
            const T right = rem > 4 ? pu[4] : T(0);
            T rv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T l = q == 0 ? left : uc[q - 1];
                const T rr = q == 3 ? right : (q + 1 < rem ? uc[q + 1] : T(0));
                // b - A u = b - d u + ax sx + ay sy + az sz
                rv[q] = fma(cz, sz[q], fma(cy, sy[q], fma(cx, l + rr, fma(-dg, uc[q], bv[q]))));
                if (q < rem) {
                    if constexpr (sizeof(T) == 4)
                        sq = fma(rv[q], rv[q], sq);
                    else
                        acc = fma(rv[q], rv[q], acc);
                }
            }
            if (r) {
                TR o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    o[q] = (TR)rv[q];
                st4<TR>(r + base + i0, o, rem, vec && sizeof(TR) == sizeof(T));
            }
        }
        if constexpr (sizeof(T) == 4)
            acc += (double)sq;
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
    const long long rows = (long long)p.ny * p.nz;
    const int wpb = kResThreads / 32;
    long long need = (rows + wpb - 1) / wpb;
    int blocks = (int)(need < c->npartials ? need : c->npartials);
    if (blocks < 1)
        blocks = 1;
    double* part = want_norm ? c->partials : nullptr;
    auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    const bool vec = p.nx % 4 == 0 && a16(u) && a16(b) && (!r || a16(r));
    residual_kernel<T, TR><<<blocks, kResThreads, 0, s>>>(u, b, r, p.nx, p.ny, p.nz, ax, ay, az,
                                                          part, vec);
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
