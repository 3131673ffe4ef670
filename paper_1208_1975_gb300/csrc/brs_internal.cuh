// Internal declarations shared by the brsmooth CUDA translation units.
// Target: sm_103a (GB300).  Nothing here is part of the public C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "brsmooth.h"

// --------------------------------------------------------------------------------------
// Launch configuration of the x-line sweep kernels.
// A "line group" of G lanes owns one x-line; lane l holds the E consecutive cells
// [l*E, l*E+E).  A CTA holds JT groups (lines j0..j0+JT-1 of one k) and marches in +z.
struct LineCfg {
    int E = 0, G = 0;   // elements per lane, lanes per line (G*E >= nx)
    int JT = 0;         // lines per CTA tile (y extent of the tile)
    int NS = 0;         // shared-memory ring stages (TMA path)
    int pieces = 1;     // TMA boxes per row (nx / pieces <= 256 elements)
    int bx = 0;         // TMA box width in elements
    bool tma = false;   // TMA ring path (rows 16-byte aligned) or the plain-load path
    int grid = 0;       // persistent CTAs (TMA path)
    size_t smem = 0;    // dynamic shared memory bytes (TMA path)
    bool pdl = true;    // launch each sweep as a programmatic dependent of the previous one
    bool pair = false;  // TMA path, FP32 lines of 385-512 cells: two warps per line
                        // (64 lanes of 8 cells, tables in line_tab2); E, G stay the
                        // one-warp layout of line_tab, which the other line kernels use
};

// Arguments of the line kernels (passed by value).
struct LineArgs {
    int nx, ny, nz;
    int JT, NS, pieces, bx;
    int nj;               // number of y tiles = ceil(ny / JT)
    long long total;      // nj * nz plane-steps
    double ay, az, om1;   // coefficients and 1 - omega
    int* status;          // device status word (sticky error flag)
};

struct TmapEntry {
    const void* ptr;
    int rows;
    CUtensorMap map;
};

struct brs_ctx {
    brs_params p{};
    double omega = 0.0;
    int device = 0;
    long long cells = 0;
    size_t esize = 8;       // bytes per element
    // block Jacobi second vector (Alg. 2) -- grid sized
    void* scratch = nullptr;
    // line solve tables (device, context dtype)
    void* line_tab = nullptr;
    void* line_tab2 = nullptr;  // two-warp layout (LineCfg::pair), FP32
    LineCfg lcfg;
    // residual reduction
    double* partials = nullptr;
    int npartials = 0;
    double* norm_dev = nullptr;
    // device status word, host-side sticky copy
    int* dev_status = nullptr;
    int sticky = BRS_OK;
    cudaStream_t last_stream = nullptr;
    // host-buffer entry point
    void* host_u_dev = nullptr;
    void* host_b_dev = nullptr;
    // tensor-map cache keyed by (pointer, box rows)
    std::vector<TmapEntry> tmaps;
    // plane path state (owned by plane.cu)
    void* plane = nullptr;
    // box path state (owned by box.cu)
    void* box = nullptr;
    // many-patch state (owned by batched.cu); non-null for batched contexts
    void* batch = nullptr;
    // defect-correction buffers of an FP32 inner context: residual and correction
    float* dc_r = nullptr;
    float* dc_c = nullptr;
    // adjoint-sweep state (owned by adjoint.cu)
    void* adjoint = nullptr;
    // FP64 x-line sweeps on the line-major copy (owned by line_seq.cu); null otherwise
    void* lseq = nullptr;
    // y-line / z-line blocks (api.cu): an x-line context of the permuted grid and the
    // permuted copies of u and b it sweeps
    brs_ctx* perm = nullptr;
    void* perm_u = nullptr;
    void* perm_b = nullptr;
};

// Status helpers -------------------------------------------------------------------------
int brs_cuda_status(cudaError_t e);

// Line path (line.cu) ----------------------------------------------------------------------
// Chooses E/G/JT/NS and uploads the factor tables; returns a BRS_* code.
int line_setup(brs_ctx* c);
void line_teardown(brs_ctx* c);
// One sweep from `uin` into `uout` (Jacobi) or in place (GS: uin == uout).
int line_sweep_launch(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s);

// FP64 x-line path (line_seq.cu): one thread per half line, elimination from both ends,
// on a line-major colour-split copy of u and b made by each call.
int line_seq_setup(brs_ctx* c);
void line_seq_teardown(brs_ctx* c);
int line_seq_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s);

// Residual (residual.cu) -------------------------------------------------------------------
int residual_setup(brs_ctx* c);
int residual_launch(brs_ctx* c, const void* u, const void* b, void* r, bool want_norm,
                    cudaStream_t s);
// FP64 residual of an FP64 context stored as FP32 (fused cast), norm into norm_dev.
int residual_launch_f32out(brs_ctx* c, const double* u, const double* b, float* r,
                           cudaStream_t s);
// ||x||_2^2 of a grid array (context dtype) into norm_dev.
int norm2sq_launch(brs_ctx* c, const void* x, cudaStream_t s);

// Axis permutation (transpose.cu) ------------------------------------------------------------
// dst[b * db + c * dc + r] = src[b * sb + r * sr + c] for r < R, c < C, b < batch.
int transpose_launch(int dtype, const void* src, void* dst, int R, int C, int batch,
                     long long sr, long long sb, long long dc, long long db, cudaStream_t s);

// Adjoint (adjoint.cu) ------------------------------------------------------------------------
void adjoint_teardown(brs_ctx* c);

// Tensor maps (api.cu) ---------------------------------------------------------------------
typedef CUresult (*PFN_encode_tiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                     const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                     const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                     CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// cuTensorMapEncodeTiled from the driver (nullptr if unavailable).
PFN_encode_tiled brs_encoder();
// 3D tiled map over a grid array with box (bx, rows, 1); cached per (pointer, rows).
const CUtensorMap* brs_tmap(brs_ctx* c, const void* ptr, int rows, int* rc);

// --------------------------------------------------------------------------------------
// Device helpers: PTX wrappers for mbarrier + TMA, bounded waits.
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for `parity` on `bar` for at most `limit_ns`; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (globaltimer_ns() - t0 > limit_ns)
            return false;
    }
}

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void set_status(int* status, int code)
{
    if (status)
        atomicCAS(status, 0, code);
}

// Programmatic dependent launch, device side.  pdl_wait: wait until the kernel this one was
// launched after has completed and its writes are visible.  Every kernel launched with
// launch_pdl calls it before it reads or writes data the previous kernel touches; for a
// normal launch it returns at once.  pdl_trigger: let the next kernel in the stream be
// scheduled as this grid's CTAs retire (without it that happens when they exit).  A
// long-running kernel that leaves room on its SMs does not trigger early: the next
// kernel's CTAs would sit beside it, waiting, for its whole run.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_trigger()
{
    pdl_wait();
    pdl_trigger();
}

// Host side: launch with programmatic stream serialisation, so that the kernel's CTAs may
// start (and run up to pdl_wait_trigger) while the previous kernel in the stream finishes.
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, A&&... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// The same for a kernel given as a function pointer with its argument array.
inline cudaError_t launch_pdl_c(const void* kernel, dim3 grid, dim3 block, size_t smem,
                                cudaStream_t s, void** args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

#endif  // __CUDACC__
