// Host side of the x-line sweep: factor tables, launch configuration, dispatch.
#include <cmath>
#include <cstdlib>
#include <vector>

#include "line_impl.cuh"
#include "thomas_tables.h"

namespace {

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

// Factor tables of M_line = tridiag(-ax, 2(ax+ay+az), -ax), computed once in FP64 (the
// constant block is factored once and shared by every line, Sec. 2 / Sec. 4.3), with the
// unscaled pivots appended for the adjoint's plain block solve.
template <typename T>
std::vector<T> line_tables(int nx, double ax, double ay, double az, double omega, int E, int G)
{
    return scan_thomas_tables<T>(nx, ax, 2.0 * (ax + ay + az), omega, E, G, true);
}

template <typename T, int E, int G>
struct LineKernels {
    static const void* tma(bool gs)
    {
        return gs ? (const void*)brs::line_tma_kernel<T, E, G, true>
                  : (const void*)brs::line_tma_kernel<T, E, G, false>;
    }
    static const void* plain(bool gs)
    {
        return gs ? (const void*)brs::line_plain_kernel<T, E, G, true>
                  : (const void*)brs::line_plain_kernel<T, E, G, false>;
    }
};

// The TMA kernel of two-warp lines (8 cells x 64 lanes), FP32.
const void* pair_kernel(bool gs)
{
    return gs ? (const void*)brs::line_tma_kernel<float, 8, 64, true>
              : (const void*)brs::line_tma_kernel<float, 8, 64, false>;
}

template <typename T>
bool kernels_for(int E, int G, bool gs, const void** tma, const void** plain)
{
#define BRS_LINE_CASE(EE, GG)                              \
    if (E == EE && G == GG) {                              \
        *tma = LineKernels<T, EE, GG>::tma(gs);            \
        *plain = LineKernels<T, EE, GG>::plain(gs);        \
        return true;                                       \
    }
    BRS_LINE_CASE(4, 4)
    BRS_LINE_CASE(4, 8)
    BRS_LINE_CASE(4, 16)
    BRS_LINE_CASE(4, 32)
    BRS_LINE_CASE(8, 32)
    BRS_LINE_CASE(12, 32)
    BRS_LINE_CASE(16, 32)
#undef BRS_LINE_CASE
    return false;
}

size_t tma_slot_bytes(const LineCfg& L, size_t es)
{
    const size_t ubox = ((size_t)(L.JT + 2) * L.bx * es + 127) & ~size_t(127);
    const size_t bbox = ((size_t)L.JT * L.bx * es + 127) & ~size_t(127);
    return (size_t)L.pieces * (ubox + bbox);
}

}  // namespace

int line_setup(brs_ctx* c)
{
    const brs_params& p = c->p;
    LineCfg L;
    if (!scan_lanes(p.nx, &L.E, &L.G))
        return BRS_ERR_UNSUPPORTED;
    const size_t es = c->esize;
    // TMA path: rows 16-byte aligned, whole lane chunks, boxes of <= 256 elements
    L.pieces = (p.nx + 255) / 256;
    L.bx = p.nx / L.pieces;
    L.tma = (p.nx * es) % 16 == 0 && p.nx % L.E == 0 && p.nx % L.pieces == 0 &&
            (L.bx * es) % 16 == 0 && L.bx % L.E == 0 && L.bx <= 256 &&
            env_int("BRSMOOTH_LINE_PLAIN", 0) == 0;
    // FP32 lines of 385-512 cells on the TMA path: two warps per line at 8 cells per lane
    // (the one-warp form holds 16 cells per lane at 221 registers, two 128-thread CTAs per
    // SM); BRSMOOTH_LINE_PAIR=0 keeps the one-warp form
    L.pair = L.tma && c->p.dtype == BRS_F32 && L.E == 16 && L.bx % kPairE == 0 &&
             env_int("BRSMOOTH_LINE_PAIR", 1) != 0;
    const int lanes = L.pair ? 64 : L.G;  // threads per line
    const int groups_per_warp = lanes >= 32 ? 1 : 32 / lanes;
    // Wide lines (E >= 12 cells per lane, 168+ registers) fit one 256-thread CTA per SM; at
    // 4 lines per tile and a 4-stage ring three (nx = 384) or two (512) CTAs fit, which
    // measured 409 -> 471 Gcell/s at 384^3 and 321 -> 336 at 512^3 (same box, FP32 Jacobi).
    const bool wide = c->p.dtype == BRS_F32 && L.E >= 12 && !L.pair;
    int jt_default = (c->p.dtype == BRS_F64 && L.E >= 8) ? 4 : wide ? 128 / L.G : 256 / lanes;
    int jt = env_int("BRSMOOTH_LINE_JT", jt_default);
    const int ny_round = ((p.ny + groups_per_warp - 1) / groups_per_warp) * groups_per_warp;
    if (jt > ny_round)
        jt = ny_round;
    jt = ((jt + groups_per_warp - 1) / groups_per_warp) * groups_per_warp;
    if (jt * lanes > 256)
        jt = 256 / lanes;
    L.JT = jt;
    // ring depth: stages s..s+2 are being read, the rest are loads in flight
    L.NS = env_int("BRSMOOTH_LINE_NS", (p.dtype == BRS_F64 || wide || L.pair) ? 4 : 6);
    if (L.NS < 3)
        L.NS = 3;
    while (L.NS > 3 && (size_t)L.NS * (tma_slot_bytes(L, es) + 8) > 227u * 1024u)
        --L.NS;

    const bool gs = p.method == BRS_CHAOTIC_GS;
    const void *ktma = nullptr, *kplain = nullptr;
    bool ok = (p.dtype == BRS_F64) ? kernels_for<double>(L.E, L.G, gs, &ktma, &kplain)
                                   : kernels_for<float>(L.E, L.G, gs, &ktma, &kplain);
    if (!ok)
        return BRS_ERR_UNSUPPORTED;
    if (L.pair)
        ktma = pair_kernel(gs);
    if (L.tma) {
        // ring, its barriers, and (two-warp lines) two exchange slots per line
        L.smem = (size_t)L.NS * tma_slot_bytes(L, es) + (size_t)L.NS * 8 +
                 (L.pair ? (size_t)2 * L.JT * es : 0);
        // the attribute belongs to the kernel, shared by every context: only ever raise it
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, ktma);
        if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < L.smem)
            e = cudaFuncSetAttribute(ktma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)L.smem);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ktma, L.JT * lanes, L.smem);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        if (occ < 1)
            return BRS_ERR_UNSUPPORTED;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const int per_sm = env_int("BRSMOOTH_LINE_CTAS_PER_SM", occ);
        L.grid = sms * (per_sm < occ ? per_sm : occ);
        const long long nj = (p.ny + L.JT - 1) / L.JT;
        const long long total = nj * p.nz;
        if (L.grid > total)
            L.grid = (int)total;
        L.pdl = env_int("BRSMOOTH_LINE_PDL", 1) != 0;
    }
    c->lcfg = L;

    // factor tables
    size_t bytes;
    cudaError_t e;
    if (p.dtype == BRS_F64) {
        auto tab = line_tables<double>(p.nx, p.ax, p.ay, p.az, c->omega, L.E, L.G);
        bytes = tab.size() * sizeof(double);
        e = cudaMalloc(&c->line_tab, bytes);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->line_tab, tab.data(), bytes, cudaMemcpyHostToDevice);
    } else {
        auto tab = line_tables<float>(p.nx, p.ax, p.ay, p.az, c->omega, L.E, L.G);
        bytes = tab.size() * sizeof(float);
        e = cudaMalloc(&c->line_tab, bytes);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->line_tab, tab.data(), bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && L.pair) {
            auto t2 = scan_pair_tables<float>(p.nx, p.ax, 2.0 * (p.ax + p.ay + p.az), c->omega);
            if (t2.empty())
                return BRS_ERR_UNSUPPORTED;
            e = cudaMalloc(&c->line_tab2, t2.size() * sizeof(float));
            if (e == cudaSuccess)
                e = cudaMemcpy(c->line_tab2, t2.data(), t2.size() * sizeof(float),
                               cudaMemcpyHostToDevice);
        }
    }
    return brs_cuda_status(e);
}

void line_teardown(brs_ctx* c)
{
    if (c->line_tab)
        cudaFree(c->line_tab);
    if (c->line_tab2)
        cudaFree(c->line_tab2);
    c->line_tab = nullptr;
    c->line_tab2 = nullptr;
}

int line_sweep_launch(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s)
{
    const brs_params& p = c->p;
    const LineCfg& L = c->lcfg;
    const bool gs = p.method == BRS_CHAOTIC_GS;
    const void *ktma = nullptr, *kplain = nullptr;
    if (p.dtype == BRS_F64)
        kernels_for<double>(L.E, L.G, gs, &ktma, &kplain);
    else
        kernels_for<float>(L.E, L.G, gs, &ktma, &kplain);
    if (L.pair)
        ktma = pair_kernel(gs);
    LineArgs a{};
    a.nx = p.nx;
    a.ny = p.ny;
    a.nz = p.nz;
    a.JT = L.JT;
    a.NS = L.NS;
    a.pieces = L.pieces;
    a.bx = L.bx;
    a.nj = (p.ny + L.JT - 1) / L.JT;
    a.total = (long long)a.nj * p.nz;
    a.ay = p.ay;
    a.az = p.az;
    a.om1 = 1.0 - c->omega;
    a.status = c->dev_status;
    cudaError_t e;
    if (L.tma) {
        int rc = BRS_OK;
        const CUtensorMap* mu = brs_tmap(c, uin, L.JT + 2, &rc);
        if (rc != BRS_OK)
            return rc;
        const CUtensorMap* mb = brs_tmap(c, b, L.JT, &rc);
        if (rc != BRS_OK)
            return rc;
        CUtensorMap tu = *mu, tbm = *mb;
        void* out = uout;
        const void* tab = L.pair ? c->line_tab2 : c->line_tab;
        void* args[] = {&tu, &tbm, &out, (void*)&tab, &a};
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(L.grid);
        cfg.blockDim = dim3(L.JT * (L.pair ? 64 : L.G));
        cfg.dynamicSmemBytes = L.smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = L.pdl ? 1 : 0;
        e = cudaLaunchKernelExC(&cfg, ktma, args);
    } else {
        const int groups = 256 / L.G;
        const long long nlines = (long long)p.ny * p.nz;
        const unsigned blocks = (unsigned)((nlines + groups - 1) / groups);
        const void* in = uin;
        void* out = uout;
        const void* tab = c->line_tab;
        void* args[] = {(void*)&in, &out, (void*)&b, (void*)&tab, &a};
        e = cudaLaunchKernel(kplain, dim3(blocks), dim3(256), args, 0, s);
    }
    return brs_cuda_status(e);
}
