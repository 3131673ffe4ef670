// Allocation-free x-line block-Jacobi sweeps.
//
// brsmooth_create allocates device memory (factor tables, the Jacobi second vector,
// reduction scratch).  Some callers cannot do that: their device memory is owned entirely
// by another allocator (a framework's caching pool or a fixed memory budget), or they run
// latency-sensitive loops where cudaMalloc/cudaFree and the device-wide synchronisation
// they imply are not acceptable.  This file gives them one entry point that allocates
// nothing: the factor tables and the second vector live in file-scope __device__ arrays
// of fixed size, which every GPU that loads the library holds until the process exits.
//
// In host code the arrays' names are host-side stand-ins, not device addresses, so each
// device's addresses come from cudaGetSymbolAddress (called once per device, with that
// device current) and are passed to the kernel as plain pointers.
#include <cmath>
#include <mutex>

#include "line_impl.cuh"
#include "thomas_tables.h"

// Fixed scratch: the second vector of block Jacobi (sized for FP64, reused for FP32) and
// the line factor tables (at most 4*512 + 2*5*32 entries).
static __device__ __align__(256) double g_noalloc_vec[BRSMOOTH_NOALLOC_MAX_CELLS];
static __device__ __align__(256) double g_noalloc_tab[4096];

namespace {

constexpr int kMaxDevices = 128;

struct DevScratch {
    void* vec = nullptr;
    void* tab = nullptr;
    bool ready = false;
};

DevScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

// Device addresses of the two arrays on the current device (first call per device looks
// them up).
int device_scratch(DevScratch* out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices)
        return BRS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    DevScratch& d = g_scratch[dev];
    if (!d.ready) {
        void* v = nullptr;
        void* t = nullptr;
        e = cudaGetSymbolAddress(&v, g_noalloc_vec);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        e = cudaGetSymbolAddress(&t, g_noalloc_tab);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        d.vec = v;
        d.tab = t;
        d.ready = true;
    }
    *out = d;
    return BRS_OK;
}

// The line factor tables built on the device by one thread, from the coefficients passed
// as kernel arguments: no host buffer and no host-to-device copy, so the call only
// enqueues work.  The routine is the one the context set-up runs on the host.
template <typename T>
__global__ void noalloc_tables_kernel(T* tab, int cap, int nx, double ax, double ay, double az,
                                      double omega, int E, int G)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        scan_thomas_fill<T>(tab, cap, nx, ax, 2.0 * (ax + ay + az), omega, E, G, false);
}

template <typename T>
const void* plain_kernel(int E, int G)
{
#define BRS_NA_CASE(EE, GG)                                             \
    if (E == EE && G == GG)                                             \
        return (const void*)brs::line_plain_kernel<T, EE, GG, false>;
    BRS_NA_CASE(4, 4)
    BRS_NA_CASE(4, 8)
    BRS_NA_CASE(4, 16)
    BRS_NA_CASE(4, 32)
    BRS_NA_CASE(8, 32)
    BRS_NA_CASE(12, 32)
    BRS_NA_CASE(16, 32)
#undef BRS_NA_CASE
    return nullptr;
}

template <typename T>
int run(int nx, int ny, int nz, double ax, double ay, double az, double omega, T* u,
        const T* b, int nsweeps, cudaStream_t s, const DevScratch& scr)
{
    int E = 0, G = 0;
    if (!scan_lanes(nx, &E, &G))
        return BRS_ERR_UNSUPPORTED;
    const int cap = (int)(sizeof(g_noalloc_tab) / sizeof(T));
    if (scan_table_len(E, G, false) > cap)
        return BRS_ERR_UNSUPPORTED;
    // the tables are rewritten on every call (the array keeps the previous call's contents)
    noalloc_tables_kernel<T><<<1, 1, 0, s>>>(static_cast<T*>(scr.tab), cap, nx, ax, ay, az,
                                             omega, E, G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    const void* k = plain_kernel<T>(E, G);
    LineArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.ay = ay;
    a.az = az;
    a.om1 = 1.0 - omega;
    const int groups = 256 / G;
    const long long nlines = (long long)ny * nz;
    const unsigned blocks = (unsigned)((nlines + groups - 1) / groups);
    const T* tab = static_cast<const T*>(scr.tab);
    T* cur = u;
    T* nxt = static_cast<T*>(scr.vec);
    // every sweep writes every cell of its output, so nothing in the second vector needs
    // clearing before use
    for (int q = 0; q < nsweeps; ++q) {
        const T* in = cur;
        T* out = nxt;
        void* args[] = {(void*)&in, &out, (void*)&b, (void*)&tab, &a};
        e = cudaLaunchKernel(k, dim3(blocks), dim3(256), args, 0, s);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != u) {
        e = cudaMemcpyAsync(u, cur, sizeof(T) * (size_t)nx * ny * nz, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
    }
    return BRS_OK;
}

}  // namespace

extern "C" int brsmooth_line_jacobi_noalloc(int nx, int ny, int nz, double ax, double ay,
                                            double az, double omega, int dtype, void* u,
                                            const void* b, int nsweeps, void* stream)
{
    cudaGetLastError();  // start from a clean launch-error state
    if (nx < 1 || ny < 1 || nz < 1 || !u || !b || nsweeps < 0 || u == b)
        return BRS_ERR_ARG;
    if (!(ax > 0.0) || !(ay > 0.0) || !(az > 0.0) || !std::isfinite(ax) || !std::isfinite(ay) ||
        !std::isfinite(az) || !std::isfinite(omega) || omega >= 2.0)
        return BRS_ERR_ARG;
    if (dtype != BRS_F64 && dtype != BRS_F32)
        return BRS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(u) & 15u) || (reinterpret_cast<uintptr_t>(b) & 15u))
        return BRS_ERR_ARG;
    if ((long long)nx * ny * nz > (long long)BRSMOOTH_NOALLOC_MAX_CELLS || nx > 512)
        return BRS_ERR_UNSUPPORTED;
    const double om = omega > 0.0 ? omega : 0.8;
    DevScratch scr;
    int rc = device_scratch(&scr);
    if (rc != BRS_OK)
        return rc;
    if (nsweeps == 0)
        return BRS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == BRS_F64)
        return run<double>(nx, ny, nz, ax, ay, az, om, static_cast<double*>(u),
                           static_cast<const double*>(b), nsweeps, s, scr);
    return run<float>(nx, ny, nz, ax, ay, az, om, static_cast<float*>(u),
                      static_cast<const float*>(b), nsweeps, s, scr);
}
