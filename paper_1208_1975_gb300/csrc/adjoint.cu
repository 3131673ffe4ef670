// Reverse-mode sweep of damped x-line block Jacobi (the transpose of Eq. blockiteration2).
//
// A forward sweep is u_{k+1} = u_k + omega z_k with z_k = M^{-1}(b - A u_k), i.e.
// u_{k+1} = G u_k + omega M^{-1} b with G = I - omega M^{-1} A.  A and the line block
// diagonal M are symmetric, so for a loss L(u_K) with lambda_{k+1} = dL/du_{k+1}:
//   mu_k       = M^{-1} lambda_{k+1}
//   lambda_k   = G^T lambda_{k+1} = lambda_{k+1} - omega A mu_k
//   dL/db     += omega mu_k
//   dL/da_d   += -omega mu_k . ( (dM/da_d) z_k + (dA/da_d) u_k )
// with dA/da_d = T_d (second difference along axis d, zero outside), and for x-line
// blocks dM/dax = Tx, dM/day = dM/daz = 2 I.
// One call performs these updates for one sweep; the caller supplies u_k (checkpointed
// or recomputed) and runs the calls from the last sweep to the first.
#include "brs_internal.cuh"
#include "line_impl.cuh"

namespace {

constexpr int kThreads = 256;

// out = M_line^{-1} in, one line group per (j,k); in-place safe (a group reads its whole
// line before writing it).
template <typename T, int E, int G>
__global__ void __launch_bounds__(kThreads) line_minv_kernel(const T* in, T* out,
                                                             const T* __restrict__ tab, int nx,
                                                             int ny, int nz)
{
    const int groups = blockDim.x / G;
    const long long line = (long long)blockIdx.x * groups + threadIdx.x / G;
    const int lane = threadIdx.x % G;
    const bool active = line < (long long)ny * nz;
    brs::LineTables<T, E, G> tb;
    tb.load(tab, lane);
    constexpr int NP = G * E;
    constexpr int LG = brs::Log2<G>::value;
    const T* ptab = tab + 3 * NP + 2 * LG * G;
    const size_t base = (size_t)(active ? line : 0) * nx;
    T r[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int x = lane * E + q;
        r[q] = (active && x < nx) ? in[base + x] : T(0);
    }
    brs::line_solve<T, E, G>(r, tb, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int x = lane * E + q;
        if (active && x < nx)
            out[base + x] = ptab[lane * E + q] * r[q];
    }
}

// lambda <- lambda - omega A mu; gb += omega mu; per-CTA partial sums of the three
// coefficient-gradient terms.  z = M^{-1}(b - A u_k), u = u_k.
template <typename T>
__global__ void __launch_bounds__(kThreads) adjoint_update_kernel(
    T* __restrict__ lam, const T* __restrict__ mu, const T* __restrict__ z,
    const T* __restrict__ u, T* __restrict__ gb, int nx, int ny, int nz, double ax, double ay,
    double az, double omega, double* partials)
{
    const long long n = (long long)nx * ny * nz;
    const long long plane = (long long)nx * ny;
    const T cx = (T)ax, cy = (T)ay, cz = (T)az, dg = (T)(2.0 * (ax + ay + az)), om = (T)omega;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx);
        const long long jk = t / nx;
        const int j = (int)(jk % ny);
        const int k = (int)(jk / ny);
        const bool xm = i > 0, xp = i + 1 < nx, ym = j > 0, yp = j + 1 < ny, zm = k > 0,
                   zp = k + 1 < nz;
        auto sum_x = [&](const T* a) { return (xm ? a[t - 1] : T(0)) + (xp ? a[t + 1] : T(0)); };
        auto sum_y = [&](const T* a) { return (ym ? a[t - nx] : T(0)) + (yp ? a[t + nx] : T(0)); };
        auto sum_z = [&](const T* a) {
            return (zm ? a[t - plane] : T(0)) + (zp ? a[t + plane] : T(0));
        };
        const T m = mu[t];
        const T Amu = dg * m - cx * sum_x(mu) - cy * sum_y(mu) - cz * sum_z(mu);
        lam[t] = lam[t] - om * Amu;
        gb[t] += om * m;
        const T zt = z[t], ut = u[t];
        const T Txz_u = (T(2) * (zt + ut)) - sum_x(z) - sum_x(u);  // Tx (z + u)
        const T Tyu = T(2) * ut - sum_y(u);
        const T Tzu = T(2) * ut - sum_z(u);
        g0 += (double)m * (double)Txz_u;
        g1 += (double)m * (double)(T(2) * zt + Tyu);
        g2 += (double)m * (double)(T(2) * zt + Tzu);
    }
    __shared__ double red[3][kThreads / 32];
    double v[3] = {g0, g1, g2};
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1)
            v[d] += __shfl_down_sync(0xffffffffu, v[d], o);
        if ((threadIdx.x & 31) == 0)
            red[d][threadIdx.x >> 5] = v[d];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int d = 0; d < 3; ++d) {
            double w = threadIdx.x < kThreads / 32 ? red[d][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                w += __shfl_down_sync(0xffffffffu, w, o);
            if (threadIdx.x == 0)
                partials[3 * blockIdx.x + d] = w;
        }
    }
}

// grad_a[d] += -omega * sum of the partials, in a fixed order.
__global__ void adjoint_reduce_kernel(const double* partials, int nblocks, double omega,
                                      double* grad_a)
{
    __shared__ double red[3][kThreads / 32];
    for (int d = 0; d < 3; ++d) {
        double acc = 0.0;
        for (int t = threadIdx.x; t < nblocks; t += blockDim.x)
            acc += partials[3 * t + d];
        for (int o = 16; o > 0; o >>= 1)
            acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0)
            red[d][threadIdx.x >> 5] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int d = 0; d < 3; ++d) {
            double w = threadIdx.x < kThreads / 32 ? red[d][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                w += __shfl_down_sync(0xffffffffu, w, o);
            if (threadIdx.x == 0)
                grad_a[d] += -omega * w;
        }
    }
}

template <typename T>
cudaError_t launch_minv(const brs_ctx* c, const T* in, T* out, cudaStream_t s)
{
    const LineCfg& L = c->lcfg;
    const int groups = kThreads / L.G;
    const long long nlines = (long long)c->p.ny * c->p.nz;
    const unsigned blocks = (unsigned)((nlines + groups - 1) / groups);
    const T* tab = static_cast<const T*>(c->line_tab);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
#define BRS_MINV_CASE(EE, GG)                                                          \
    if (L.E == EE && L.G == GG) {                                                      \
        line_minv_kernel<T, EE, GG><<<blocks, kThreads, 0, s>>>(in, out, tab, nx, ny, nz); \
        return cudaGetLastError();                                                     \
    }
    BRS_MINV_CASE(4, 4)
    BRS_MINV_CASE(4, 8)
    BRS_MINV_CASE(4, 16)
    BRS_MINV_CASE(4, 32)
    BRS_MINV_CASE(8, 32)
    BRS_MINV_CASE(12, 32)
    BRS_MINV_CASE(16, 32)
#undef BRS_MINV_CASE
    return cudaErrorInvalidConfiguration;
}

struct AdjState {
    void* mu = nullptr;
    double* partials = nullptr;
    int nblocks = 0;
};

template <typename T>
int adjoint_run(brs_ctx* c, T* lam, const T* u, const T* b, T* gb, double* ga, cudaStream_t s)
{
    AdjState* A = static_cast<AdjState*>(c->adjoint);
    T* z = static_cast<T*>(c->scratch);
    T* mu = static_cast<T*>(A->mu);
    // z = M^{-1}(b - A u_k)
    int rc = residual_launch(c, u, b, z, false, s);
    if (rc != BRS_OK)
        return rc;
    cudaError_t e = launch_minv<T>(c, z, z, s);
    if (e == cudaSuccess)
        e = launch_minv<T>(c, lam, mu, s);  // mu = M^{-1} lambda
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    adjoint_update_kernel<T><<<A->nblocks, kThreads, 0, s>>>(lam, mu, z, u, gb, c->p.nx, c->p.ny,
                                                             c->p.nz, c->p.ax, c->p.ay, c->p.az,
                                                             c->omega, A->partials);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    adjoint_reduce_kernel<<<1, kThreads, 0, s>>>(A->partials, A->nblocks, c->omega, ga);
    return brs_cuda_status(cudaGetLastError());
}

}  // namespace

void adjoint_teardown(brs_ctx* c)
{
    AdjState* A = static_cast<AdjState*>(c->adjoint);
    if (!A)
        return;
    if (A->mu)
        cudaFree(A->mu);
    if (A->partials)
        cudaFree(A->partials);
    delete A;
    c->adjoint = nullptr;
}

extern "C" int brsmooth_adjoint_sweep(brs_ctx* c, void* lam, const void* u_k, const void* b,
                                      void* grad_b, double* grad_a, void* stream)
{
    cudaGetLastError();  // start from a clean launch-error state
    if (!c || !lam || !u_k || !b || !grad_b || !grad_a)
        return BRS_ERR_ARG;
    if (c->batch || c->p.block != BRS_XLINE || c->p.method != BRS_JACOBI)
        return BRS_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!c->adjoint) {
        AdjState* A = new AdjState();
        c->adjoint = A;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const long long need = (c->cells + kThreads - 1) / kThreads;
        A->nblocks = (int)(need < (long long)sms * 8 ? need : (long long)sms * 8);
        if (A->nblocks < 1)
            A->nblocks = 1;
        cudaError_t e = cudaMalloc(&A->mu, (size_t)c->cells * c->esize);
        if (e == cudaSuccess)
            e = cudaMalloc(&A->partials, sizeof(double) * 3 * A->nblocks);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
    }
    c->last_stream = s;
    if (c->p.dtype == BRS_F64)
        return adjoint_run<double>(c, (double*)lam, (const double*)u_k, (const double*)b,
                                   (double*)grad_b, grad_a, s);
    return adjoint_run<float>(c, (float*)lam, (const float*)u_k, (const float*)b, (float*)grad_b,
                              grad_a, s);
}
