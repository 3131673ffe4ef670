// C ABI of brsmooth (declared in include/brsmooth.h): context lifetime, argument checks,
// sweep dispatch, residual, host-buffer path and status reporting.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "brs_internal.cuh"
#include "batched.cuh"
#include "box.cuh"
#include "plane.cuh"

namespace {
thread_local const char* g_last_cuda_error = "no error";
}

int brs_cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return BRS_OK;
    g_last_cuda_error = cudaGetErrorString(e);
    cudaGetLastError();  // clear a non-sticky launch error so later calls start clean
    if (e == cudaErrorMemoryAllocation)
        return BRS_ERR_NOMEM;
    return BRS_ERR_CUDA;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode;
}

bool aligned16(const void* p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

bool finite_pos(double v)
{
    return std::isfinite(v) && v > 0.0;
}

// Device status word is host-mapped pinned memory: kernels set it on a device-side
// failure and every later call on the context can read it without synchronising.
int poll_status(brs_ctx* c)
{
    if (c->sticky == BRS_OK && c->dev_status) {
        volatile int* hs = reinterpret_cast<volatile int*>(c->dev_status);
        if (*hs != 0)
            c->sticky = *hs;
    }
    if (c->sticky == BRS_OK && c->perm)  // the permuted grid's kernels report there
        c->sticky = poll_status(c->perm);
    return c->sticky;
}

int validate(const brs_params* p)
{
    if (!p)
        return BRS_ERR_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1)
        return BRS_ERR_ARG;
    if (!finite_pos(p->ax) || !finite_pos(p->ay) || !finite_pos(p->az))
        return BRS_ERR_ARG;
    if (p->block != BRS_XLINE && p->block != BRS_XYPLANE && p->block != BRS_BOX &&
        p->block != BRS_YLINE && p->block != BRS_ZLINE)
        return BRS_ERR_ARG;
    if (p->block == BRS_BOX &&
        (p->bx < 1 || p->by < 1 || p->bz < 1 || p->nx % p->bx || p->ny % p->by || p->nz % p->bz))
        return BRS_ERR_ARG;
    if (p->method != BRS_JACOBI && p->method != BRS_CHAOTIC_GS)
        return BRS_ERR_ARG;
    if (p->dtype != BRS_F64 && p->dtype != BRS_F32)
        return BRS_ERR_ARG;
    if (!std::isfinite(p->omega) || p->omega >= 2.0)
        return BRS_ERR_ARG;
    if (p->plane_math < BRS_PLANE_AUTO || p->plane_math > BRS_PLANE_3XTF32)
        return BRS_ERR_ARG;
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n > (1ll << 40))
        return BRS_ERR_UNSUPPORTED;
    return BRS_OK;
}

// y-line / z-line blocks: permutation of the axes that makes them x-lines.  Axis a of the
// permuted grid is axis ax[a] of the grid (0 = x, 1 = y, 2 = z).
void perm_axes(int block, int ax[3])
{
    if (block == BRS_YLINE) {
        ax[0] = 1, ax[1] = 0, ax[2] = 2;  // (y, x, z)
    } else {
        ax[0] = 2, ax[1] = 0, ax[2] = 1;  // (z, x, y)
    }
}

// Grid -> permuted grid (forward) or back.  y-lines: per plane k, [j][i] <-> [i][j];
// z-lines: per row j, [k][i] (plane stride) <-> [i][k] (rows of nz at j nx nz).
int permute(brs_ctx* c, const void* src, void* dst, bool forward, cudaStream_t s)
{
    const long long nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const int dt = c->p.dtype;
    if (c->p.block == BRS_YLINE) {
        if (forward)  // (r = j, c = i) -> i * ny + j
            return transpose_launch(dt, src, dst, (int)ny, (int)nx, (int)nz, nx, nx * ny, ny,
                                    nx * ny, s);
        return transpose_launch(dt, src, dst, (int)nx, (int)ny, (int)nz, ny, nx * ny, nx,
                                nx * ny, s);
    }
    if (forward)  // batch j: (r = k, c = i) at k nx ny + j nx + i -> j nx nz + i nz + k
        return transpose_launch(dt, src, dst, (int)nz, (int)nx, (int)ny, nx * ny, nx, nz,
                                nx * nz, s);
    // batch j: (r = i, c = k) at j nx nz + i nz + k -> k nx ny + j nx + i
    return transpose_launch(dt, src, dst, (int)nx, (int)nz, (int)ny, nz, nx * nz, nx * ny, nx,
                            s);
}

int perm_setup(brs_ctx* c)
{
    const brs_params& p = c->p;
    int ax[3];
    perm_axes(p.block, ax);
    const int n[3] = {p.nx, p.ny, p.nz};
    const double a[3] = {p.ax, p.ay, p.az};
    if (n[ax[2]] > 65535)
        return BRS_ERR_UNSUPPORTED;  // the permutation's batch count
    brs_params q = p;
    q.block = BRS_XLINE;
    q.nx = n[ax[0]], q.ny = n[ax[1]], q.nz = n[ax[2]];
    q.ax = a[ax[0]], q.ay = a[ax[1]], q.az = a[ax[2]];
    int rc = brsmooth_create(&q, &c->perm);
    if (rc != BRS_OK)
        return rc;
    cudaError_t e = cudaMalloc(&c->perm_u, (size_t)c->cells * c->esize);
    if (e == cudaSuccess)
        e = cudaMalloc(&c->perm_b, (size_t)c->cells * c->esize);
    return brs_cuda_status(e);
}

int perm_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s)
{
    if (nsweeps == 0)
        return BRS_OK;
    int rc = permute(c, u, c->perm_u, true, s);
    if (rc == BRS_OK)
        rc = permute(c, b, c->perm_b, true, s);
    if (rc == BRS_OK)
        rc = brsmooth_sweep(c->perm, c->perm_u, c->perm_b, nsweeps, s);
    if (rc == BRS_OK)
        rc = permute(c, c->perm_u, u, false, s);
    return rc;
}

void free_ctx(brs_ctx* c)
{
    if (!c)
        return;
    line_teardown(c);
    line_seq_teardown(c);
    plane_teardown(c);
    box_teardown(c);
    batched_teardown(c);
    adjoint_teardown(c);
    free_ctx(c->perm);
    if (c->perm_u)
        cudaFree(c->perm_u);
    if (c->perm_b)
        cudaFree(c->perm_b);
    if (c->scratch)
        cudaFree(c->scratch);
    if (c->partials)
        cudaFree(c->partials);
    if (c->host_u_dev)
        cudaFree(c->host_u_dev);
    if (c->host_b_dev)
        cudaFree(c->host_b_dev);
    if (c->dc_r)
        cudaFree(c->dc_r);
    if (c->dc_c)
        cudaFree(c->dc_c);
    if (c->dev_status)
        cudaFreeHost(c->dev_status);
    delete c;
}

}  // namespace

PFN_encode_tiled brs_encoder()
{
    return reinterpret_cast<PFN_encode_tiled>(encoder());
}

const CUtensorMap* brs_tmap(brs_ctx* c, const void* ptr, int rows, int* rc)
{
    for (auto& t : c->tmaps)
        if (t.ptr == ptr && t.rows == rows)
            return &t.map;
    auto enc = encoder();
    if (!enc) {
        *rc = BRS_ERR_CUDA;
        return nullptr;
    }
    const brs_params& p = c->p;
    TmapEntry ent{};
    ent.ptr = ptr;
    ent.rows = rows;
    cuuint64_t gdim[3] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz};
    cuuint64_t gstride[2] = {(cuuint64_t)p.nx * c->esize, (cuuint64_t)p.nx * p.ny * c->esize};
    cuuint32_t box[3] = {(cuuint32_t)c->lcfg.bx, (cuuint32_t)rows, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(&ent.map,
                     p.dtype == BRS_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     3, const_cast<void*>(ptr), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *rc = BRS_ERR_CUDA;
        return nullptr;
    }
    if (c->tmaps.size() >= 16)
        c->tmaps.erase(c->tmaps.begin());
    c->tmaps.push_back(ent);
    return &c->tmaps.back().map;
}

extern "C" {

const char* brsmooth_cuda_error_string(void)
{
    return g_last_cuda_error;
}

const char* brsmooth_strerror(int code)
{
    switch (code) {
    case BRS_OK: return "success";
    case BRS_ERR_ARG: return "invalid argument";
    case BRS_ERR_UNSUPPORTED: return "unsupported configuration";
    case BRS_ERR_CUDA: return "CUDA runtime error";
    case BRS_ERR_NOMEM: return "out of memory";
    case BRS_ERR_TIMEOUT: return "device-side wait timed out";
    case BRS_ERR_BOUNDS: return "device-side bounds check failed";
    default: return "unknown status code";
    }
}

int brsmooth_create(const brs_params* p, brs_ctx** out)
{
    if (!out)
        return BRS_ERR_ARG;
    *out = nullptr;
    int rc = validate(p);
    if (rc != BRS_OK)
        return rc;
    brs_ctx* c = new (std::nothrow) brs_ctx();
    if (!c)
        return BRS_ERR_NOMEM;
    c->p = *p;
    c->omega = p->omega > 0.0 ? p->omega : (p->method == BRS_JACOBI ? 0.8 : 1.0);
    c->esize = p->dtype == BRS_F64 ? 8 : 4;
    c->cells = (long long)p->nx * p->ny * p->nz;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        free_ctx(c);
        return brs_cuda_status(e);
    }
    e = cudaHostAlloc((void**)&c->dev_status, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) {
        free_ctx(c);
        return brs_cuda_status(e);
    }
    *c->dev_status = 0;
    if (p->block == BRS_XLINE) {
        rc = line_setup(c);
        // FP64 lines: the twisted-elimination path (BRSMOOTH_LINE_SEQ=0: the lane-scan kernel)
        const char* ev = std::getenv("BRSMOOTH_LINE_SEQ");
        if (rc == BRS_OK && p->dtype == BRS_F64 && !(ev && ev[0] == '0'))
            rc = line_seq_setup(c);
    } else if (p->block == BRS_XYPLANE)
        rc = plane_setup(c);
    else if (p->block == BRS_BOX)
        rc = box_setup(c);
    else
        rc = perm_setup(c);
    if (rc == BRS_OK)
        rc = residual_setup(c);
    if (rc == BRS_OK && p->method == BRS_JACOBI && !c->perm) {
        e = cudaMalloc(&c->scratch, (size_t)c->cells * c->esize);
        rc = brs_cuda_status(e);
    }
    if (rc != BRS_OK) {
        free_ctx(c);
        return rc;
    }
    // the status word's device alias (same address under unified addressing)
    int* dptr = nullptr;
    e = cudaHostGetDevicePointer((void**)&dptr, c->dev_status, 0);
    if (e != cudaSuccess || dptr != c->dev_status) {
        free_ctx(c);
        return e != cudaSuccess ? brs_cuda_status(e) : BRS_ERR_UNSUPPORTED;
    }
    *out = c;
    return BRS_OK;
}

static int sweep_one(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s)
{
    if (c->p.block == BRS_XLINE)
        return line_sweep_launch(c, uin, uout, b, s);
    if (c->p.block == BRS_XYPLANE)
        return plane_sweep_launch(c, uin, uout, b, s);
    return box_sweep_launch(c, uin, uout, b, s);
}

int brsmooth_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, void* stream)
{
    cudaGetLastError();  // start from a clean launch-error state
    if (!c || !u || !b || nsweeps < 0)
        return BRS_ERR_ARG;
    if (!aligned16(u) || !aligned16(b) || u == b)
        return BRS_ERR_ARG;
    int rc = poll_status(c);
    if (rc != BRS_OK)
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    c->last_stream = s;
    if (c->batch)
        return batched_sweep(c, u, b, nsweeps, s);
    if (c->perm)
        return perm_sweep(c, u, b, nsweeps, s);
    if (c->lseq)
        return line_seq_sweep(c, u, b, nsweeps, s);
    if (c->plane) {
        // several plane sweeps in one call: the x-sine form, where the context has it
        rc = plane_modes_sweep(c, u, b, nsweeps, s);
        if (rc != BRS_ERR_UNSUPPORTED)
            return rc;
        rc = BRS_OK;
    }
    if (c->p.method == BRS_CHAOTIC_GS) {
        for (int k = 0; k < nsweeps && rc == BRS_OK; ++k)
            rc = sweep_one(c, u, u, b, s);
        return rc;
    }
    // block Jacobi: v = u + omega M^{-1}(b - A u) into the second vector, then swap (Alg. 2)
    void* cur = u;
    void* nxt = c->scratch;
    for (int k = 0; k < nsweeps && rc == BRS_OK; ++k) {
        rc = sweep_one(c, cur, nxt, b, s);
        void* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (rc == BRS_OK && cur != u)
        rc = brs_cuda_status(
            cudaMemcpyAsync(u, cur, (size_t)c->cells * c->esize, cudaMemcpyDeviceToDevice, s));
    return rc;
}

int brsmooth_residual(brs_ctx* c, const void* u, const void* b, void* r, double* norm2,
                      void* stream)
{
    cudaGetLastError();  // start from a clean launch-error state
    if (!c || !u || !b)
        return BRS_ERR_ARG;
    if (c->batch)
        return BRS_ERR_UNSUPPORTED;
    int rc = poll_status(c);
    if (rc != BRS_OK)
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    c->last_stream = s;
    rc = residual_launch(c, u, b, r, norm2 != nullptr, s);
    if (rc != BRS_OK || !norm2)
        return rc;
    double h = 0.0;
    cudaError_t e = cudaMemcpyAsync(&h, c->norm_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    *norm2 = std::sqrt(h);
    return BRS_OK;
}

static int sweep_host_enqueue(brs_ctx* c, void* u_host, const void* b_host, int nsweeps,
                              cudaStream_t s)
{
    if (!c || !u_host || !b_host || nsweeps < 0)
        return BRS_ERR_ARG;
    const size_t bytes = (size_t)c->cells * c->esize;
    cudaError_t e = cudaSuccess;
    if (!c->host_u_dev)
        e = cudaMalloc(&c->host_u_dev, bytes);
    if (e == cudaSuccess && !c->host_b_dev)
        e = cudaMalloc(&c->host_b_dev, bytes);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    e = cudaMemcpyAsync(c->host_b_dev, b_host, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->host_u_dev, u_host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    int rc = brsmooth_sweep(c, c->host_u_dev, c->host_b_dev, nsweeps, s);
    if (rc != BRS_OK)
        return rc;
    return brs_cuda_status(
        cudaMemcpyAsync(u_host, c->host_u_dev, bytes, cudaMemcpyDeviceToHost, s));
}

int brsmooth_sweep_host(brs_ctx* c, void* u_host, const void* b_host, int nsweeps, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = sweep_host_enqueue(c, u_host, b_host, nsweeps, s);
    if (rc != BRS_OK)
        return rc;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    return poll_status(c);
}

int brsmooth_sweep_host_async(brs_ctx* c, void* u_host, const void* b_host, int nsweeps,
                              void* stream)
{
    return sweep_host_enqueue(c, u_host, b_host, nsweeps, static_cast<cudaStream_t>(stream));
}

int brsmooth_destroy(brs_ctx* c)
{
    if (!c)
        return BRS_OK;
    cudaDeviceSynchronize();
    free_ctx(c);
    return BRS_OK;
}

int brsmooth_last_error(brs_ctx* c)
{
    if (!c)
        return BRS_ERR_ARG;
    if (c->last_stream)
        cudaStreamSynchronize(c->last_stream);
    else
        cudaDeviceSynchronize();
    int rc = poll_status(c);
    c->sticky = BRS_OK;
    if (c->dev_status)
        *reinterpret_cast<volatile int*>(c->dev_status) = 0;
    return rc;
}

int brsmooth_create_batched(int npatch, const int* dims, const brs_params* common,
                            brs_ctx** out)
{
    if (!out)
        return BRS_ERR_ARG;
    *out = nullptr;
    if (npatch < 1 || !dims || !common)
        return BRS_ERR_ARG;
    brs_params p = *common;
    p.nx = p.ny = p.nz = 1;
    int rc = validate(&p);
    if (rc != BRS_OK)
        return rc;
    if (p.block != BRS_XLINE)
        return BRS_ERR_UNSUPPORTED;
    long long total = 0;
    for (int q = 0; q < npatch; ++q) {
        const int nx = dims[3 * q], ny = dims[3 * q + 1], nz = dims[3 * q + 2];
        if (nx < 1 || ny < 1 || nz < 1)
            return BRS_ERR_ARG;
        if (nx > 128)
            return BRS_ERR_UNSUPPORTED;
        total += (long long)nx * ny * nz;
    }
    if (total > (1ll << 36))
        return BRS_ERR_UNSUPPORTED;
    brs_ctx* c = new (std::nothrow) brs_ctx();
    if (!c)
        return BRS_ERR_NOMEM;
    c->p = p;
    c->omega = p.omega > 0.0 ? p.omega : (p.method == BRS_JACOBI ? 0.8 : 1.0);
    c->esize = p.dtype == BRS_F64 ? 8 : 4;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void**)&c->dev_status, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) {
        free_ctx(c);
        return brs_cuda_status(e);
    }
    *c->dev_status = 0;
    rc = batched_setup(c, npatch, dims);
    if (rc != BRS_OK) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return BRS_OK;
}

int brsmooth_create_level(int npatch, const int* dims, const int* nbr,
                          const brs_params* common, brs_ctx** out)
{
    if (!out)
        return BRS_ERR_ARG;
    *out = nullptr;
    if (npatch < 1 || !dims || !nbr || !common)
        return BRS_ERR_ARG;
    // the neighbour table is checked in full before anything touches the device
    for (int p = 0; p < npatch; ++p) {
        for (int d = 0; d < 3; ++d)
            if (dims[3 * p + d] < 2)
                return BRS_ERR_ARG;
        for (int f = 0; f < 6; ++f) {
            const int q = nbr[6 * p + f];
            if (q < -1 || q >= npatch)
                return BRS_ERR_ARG;
            if (q < 0)
                continue;
            if (nbr[6 * q + (f ^ 1)] != p)
                return BRS_ERR_ARG;
            const int axis = f >> 1;  // the face's normal axis
            for (int d = 0; d < 3; ++d)
                if (d != axis && dims[3 * q + d] != dims[3 * p + d])
                    return BRS_ERR_ARG;
        }
    }
    brs_ctx* c = nullptr;
    int rc = brsmooth_create_batched(npatch, dims, common, &c);
    if (rc != BRS_OK)
        return rc;
    rc = level_setup(c, nbr);
    if (rc != BRS_OK) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return BRS_OK;
}

int brsmooth_sweep_batched(brs_ctx* c, void* u_packed, const void* b_packed, int nsweeps,
                           void* stream)
{
    if (!c || !c->batch)
        return BRS_ERR_ARG;
    return brsmooth_sweep(c, u_packed, b_packed, nsweeps, stream);
}

int brsmooth_batched_config(const brs_ctx* c, int* kchunk, int* warps_per_cta, int* ctas,
                            int* work_items)
{
    if (!c || !c->batch || !kchunk || !warps_per_cta || !ctas || !work_items)
        return BRS_ERR_ARG;
    batched_describe(c, kchunk, warps_per_cta, ctas, work_items);
    return BRS_OK;
}

int brsmooth_level_keep_ghosts(brs_ctx* c, int on)
{
    if (!c || !c->batch)
        return BRS_ERR_ARG;
    return level_keep_ghosts(c, on);
}

long long brsmooth_cells(const brs_ctx* c)
{
    return c ? c->cells : 0;
}

}  // extern "C"
