// Batched x-line block sweeps over many independent patches of different sizes
// (Sec. 1.1 / Sec. 4.2: an AMR level holds many patches; the GPU processes their blocks
// as one stream of work, with no synchronisation between patches).
//
// Work items are (patch, y-block of R lines, z-chunk of KC planes).  A persistent grid
// of warps pulls items from an atomic counter (load balance across uneven patches);
// each warp marches its R lines in +z: u(j,k-1), u(j,k), u(j,k+1) stay in registers,
// the y neighbours inside the warp come by shuffle and only the two halo lines of the
// y-block are loaded.  Lines are solved exactly with the shared-pivot Thomas scan of the
// single-grid path (the factor of M_line depends only on nx and the coefficients, so one
// table per distinct nx is built once).  One launch per sweep; the sweep sequence of a
// call is captured once into a CUDA graph and replayed as a single graph launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "batched.cuh"
#include "line_impl.cuh"
#include "thomas_tables.h"

namespace {

struct PatchDesc {
    int nx, ny, nz;
    int cls;          // lanes per line G = 4 << cls (E = 4 cells per lane)
    long long off;    // element offset of the patch in the packed arrays
    int item0;        // first work item of the patch
    int njb;          // y-blocks (R = 32 / G lines each)
    int nkc;          // z-chunks
    int tab;          // element offset of the patch's line tables
    int vec;          // rows and patch start are 16-byte aligned
    int bchunk0;      // level: first 256-element chunk of the patch's ghost block
    long long g0;     // level: start of the patch's ghost block
};

struct Graph {
    const void* u;
    const void* b;
    int nsweeps;
    int mode;  // level ghost chaining at capture: bit 0 on, bit 1 ghosts valid, bit 2 parity
    cudaGraphExec_t exec;
};

struct BatchState {
    int npatch = 0;
    std::vector<int> dims;      // 3 * npatch
    long long total = 0;        // cells
    int KC = 8;                 // z-chunk
    int warps = 8;              // warps per CTA
    int grid = 0;               // persistent CTAs
    int nitems = 0;
    PatchDesc* d_desc = nullptr;
    int* d_item_patch = nullptr;
    void* d_tab = nullptr;
    int* d_counters = nullptr;  // one per sweep of a call
    int ncounters = 0;
    std::vector<PatchDesc> h_desc;
    std::vector<int> h_item_patch;
    cudaStream_t cap = nullptr; // private capture stream
    std::vector<Graph> graphs;
    bool async = false;         // cp.async kernel (every patch row is 16-byte aligned)
    // level of patches (ghost values from the face neighbours, refreshed after every step)
    bool level = false;
    int* d_nbr = nullptr;        // 6 per patch: -x, +x, -y, +y, -z, +z neighbour or -1
    int* d_chunk_patch = nullptr; // boundary-cell chunk -> patch
    int nchunks = 0;
    void* ghost = nullptr;       // ghost blocks of every patch (neighbours' face layers)
    void* ghost2 = nullptr;      // the second ghost buffer (written during a step, read by the next)
    long long* d_push = nullptr; // 6 per patch: where each face goes in a ghost buffer, or -1
    bool push = true;            // steps after a call's first write their faces themselves
    // ghosts kept across calls (brsmooth_level_keep_ghosts): the last step of a call also
    // writes its faces, and the next call's first step reads them instead of gathering;
    // gpar is the ghost buffer the next step reads (0: ghost, 1: ghost2)
    bool keep = false;
    bool gvalid = false;
    int gpar = 0;
    int stages = 4;             // its ring depth (z-steps of lookahead per warp)
};

BatchState* bs(brs_ctx* c)
{
    return static_cast<BatchState*>(c->batch);
}

constexpr int kE = 4;
// cp.async ring fields: u(k+1), b(k) and the two halo lines
constexpr int kFields = 4;
// x ghosts of one work item of a level, staged per warp: 2 faces x z-steps x lines
constexpr int kMaxKC = 32;
constexpr size_t xg_bytes(size_t esize) { return (size_t)2 * kMaxKC * 8 * esize; }
// bytes of one warp's cp.async area: stages x fields x 32 lanes x kE elements, plus the
// staged x ghosts of a level
constexpr size_t async_ring_bytes(int stages, size_t esize, bool level)
{
    return (size_t)stages * kFields * 32 * kE * esize + (level ? xg_bytes(esize) : 0);
}

// Ghost block of a patch of a level (the face neighbours' adjacent layers as they were before
// the step; zero on the physical boundary), at g0 in a ghost array: the z- and z+ faces
// ([j][i], nx*ny each), the y- and y+ faces ([k][i], nx*nz), the x- and x+ faces ([k][j],
// ny*nz), each face starting on a multiple of 4 elements.
__host__ __device__ __forceinline__ long long round4(long long v) { return (v + 3) & ~3ll; }
__host__ __device__ __forceinline__ long long ghost_block(int nx, int ny, int nz)
{
    return 2 * (round4((long long)nx * ny) + round4((long long)nx * nz) +
                round4((long long)ny * nz));
}

// Row (jj, kk) just outside the patch across a z or y face: its x = 0 element in the
// ghost block, or null (no ghosts, or not a face row).
template <typename T>
__device__ __forceinline__ const T* outside_row(const PatchDesc& d, const T* ghost, int jj, int kk)
{
    if (!ghost)
        return nullptr;
    const long long A = round4((long long)d.nx * d.ny), Bz = round4((long long)d.nx * d.nz);
    const T* g = ghost + d.g0;
    if (jj >= 0 && jj < d.ny) {
        if (kk == -1)
            return g + (long long)jj * d.nx;
        if (kk == d.nz)
            return g + A + (long long)jj * d.nx;
    } else if (kk >= 0 && kk < d.nz) {
        if (jj == -1)
            return g + 2 * A + (long long)kk * d.nx;
        if (jj == d.ny)
            return g + 2 * A + Bz + (long long)kk * d.nx;
    }
    return nullptr;
}

// x- face ghost of line (j, k); the x+ ghost is ghost_x(...) + round4(ny * nz).
template <typename T>
__device__ __forceinline__ const T* ghost_x(const PatchDesc& d, const T* ghost, int j, int k)
{
    const long long A = round4((long long)d.nx * d.ny), Bz = round4((long long)d.nx * d.nz);
    return ghost + d.g0 + 2 * A + 2 * Bz + j + (long long)d.ny * k;
}

// Level contexts, steps after the first of a call: once a work item's lines are stored, the
// warp copies the item's cells that lie on a patch face into the ghost block of the face
// neighbour, in the ghost buffer that the next step reads (the current step reads the other
// one, so every patch still sees its neighbours' values of the previous step).  Every cell
// is written once per step, so the values are final; they are re-read from the output (just
// written by this warp, L2-resident).  push[f] is the offset of the destination face in that
// buffer, -1 where face f has no neighbour; destination layouts: z faces [j][i], y faces
// [k][i], x faces [k][j].  With yz_done (the cp.async kernel) the step loop has stored the
// y- and z-face rows itself, from registers, and only the x faces (and the y faces of a
// one-line patch) are copied here.  Not inlined and kept small: the step loop keeps its
// registers; the item is re-read here.
template <typename T>
__device__ __noinline__ void push_item(const PatchDesc* __restrict__ desc,
                                       const long long* __restrict__ push_all, T* gnext,
                                       const T* uout, int pq, int item, int KC, bool yz_done)
{
    __syncwarp();  // the item's stores by every lane of the warp are visible to all lanes
    const PatchDesc d = desc[pq];
    const long long* push = push_all + 6 * pq;
    const int local = item - d.item0;
    const int R = 32 / (4 << d.cls);
    const int j0 = (local % d.njb) * R, k0 = (local / d.njb) * KC;
    const int k1 = min(d.nz, k0 + KC);
    const T* uo = uout + d.off;
    const int lane = threadIdx.x & 31;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const long long plane = (long long)nx * ny;
    const int nj = min(R, ny - j0), nk = k1 - k0;
    for (int f = 0; f < 2; ++f) {  // x faces: the item's cells at x = 0 and x = nx - 1
        const long long o = __ldg(push + f);
        if (o < 0)
            continue;
        const int xi = f ? nx - 1 : 0;
        const int lgR = 3 - d.cls;  // R = 8 >> cls
        for (int t = lane; t < nj * nk; t += 32) {
            const int kk = nj == R ? t >> lgR : t / nj;
            const int jl = t - kk * nj;
            const int j = j0 + jl, k = k0 + kk;
            gnext[o + j + (long long)ny * k] = uo[k * plane + (long long)j * nx + xi];
        }
    }
    for (int f = 2; f < 4; ++f) {  // y faces: line 0 or ny - 1, when the item holds it
        if (yz_done && ny > 1)
            break;  // written by the step loop
        const int j = f == 2 ? 0 : ny - 1;
        if (j < j0 || j >= j0 + nj)
            continue;
        const long long o = __ldg(push + f);
        if (o < 0)
            continue;
        for (int t = lane; t < nk * nx; t += 32) {
            const int kk = t / nx, i = t - kk * nx;
            const int k = k0 + kk;
            gnext[o + (long long)k * nx + i] = uo[k * plane + (long long)j * nx + i];
        }
    }
    for (int f = 4; f < 6 && !yz_done; ++f) {  // z faces: plane 0 or nz - 1, when held
        const int k = f == 4 ? 0 : nz - 1;
        if (k < k0 || k >= k1)
            continue;
        const long long o = __ldg(push + f);
        if (o < 0)
            continue;
        for (int t = lane; t < nj * nx; t += 32) {
            const int jl = t / nx, i = t - jl * nx;
            const int j = j0 + jl;
            gnext[o + (long long)j * nx + i] = uo[k * plane + (long long)j * nx + i];
        }
    }
}

template <typename T, int G, bool GS, bool LV>
__device__ __forceinline__ void batched_item(const PatchDesc& d, int jb, int kc, int KC,
                                             const T* uin, T* uout, const T* __restrict__ b,
                                             const T* __restrict__ tab, T ax, T ay, T az,
                                             T om1, const T* ghost)
{
    constexpr int R = 32 / G;
    const int lanew = threadIdx.x & 31;
    const int g = lanew / G, l = lanew % G;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int j = jb * R + g;
    const bool jin = j < ny;
    const int x0 = l * kE;
    const bool xin = x0 < nx;
    const long long plane = (long long)nx * ny;
    const T* ub = uin + d.off;
    T* uo = uout + d.off;
    const T* bb = b + d.off;
    brs::LineTables<T, kE, G> tb;
    tb.load(tab + d.tab, l);
    const int k0 = kc * KC;
    const int k1 = min(nz, k0 + KC);

    // load E cells of line (jj, kk) of `src`; outside the patch the ghost row (u only,
    // level contexts) or zero
    auto ld = [&](const T* src, int jj, int kk, T (&v)[kE]) {
        const bool in = jj >= 0 && jj < ny && kk >= 0 && kk < nz;
        const T* row = in ? src + (long long)kk * plane + (long long)jj * nx
                          : ((LV && src == ub) ? outside_row(d, ghost, jj, kk) : nullptr);
        if (xin && row) {
            const T* p = row + x0;
            if (d.vec) {
                if (sizeof(T) == 4) {
                    float4 f = *reinterpret_cast<const float4*>(p);
                    v[0] = (T)f.x; v[1] = (T)f.y; v[2] = (T)f.z; v[3] = (T)f.w;
                } else {
                    const double2* q = reinterpret_cast<const double2*>(p);
                    double2 f0 = q[0], f1 = q[1];
                    v[0] = (T)f0.x; v[1] = (T)f0.y; v[2] = (T)f1.x; v[3] = (T)f1.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kE; ++q)
                    v[q] = (x0 + q < nx) ? p[q] : T(0);
            }
        } else {
#pragma unroll
            for (int q = 0; q < kE; ++q)
                v[q] = T(0);
        }
    };

    T um[kE], uc[kE], up[kE], r[kE], bv[kE], un[kE], us[kE];
    // next step's u(k+2), b(k+1) and halo lines (y-block edges), loaded one step ahead
    T upn[kE], bvn[kE], hnn[kE], hsn[kE];
    // x ghosts of the line (level contexts): the lane holding x = 0 and the one holding
    // x = nx - 1 add ax times the neighbour's value, loaded one step ahead
    const bool xlo = LV && xin && jin && x0 == 0;
    const bool xhi = LV && xin && jin && x0 <= nx - 1 && nx - 1 < x0 + kE;
    const long long xpo = round4((long long)ny * nz);
    T gxm = T(0), gxp = T(0), gxmn = T(0), gxpn = T(0);
    if (xlo)
        gxmn = *ghost_x(d, ghost, j, k0);
    if (xhi)
        gxpn = ghost_x(d, ghost, j, k0)[xpo];
    ld(ub, j, k0 - 1, um);
    ld(ub, j, k0, uc);
    ld(ub, j, k0 + 1, upn);
    ld(bb, j, k0, bvn);
    ld(ub, g == 0 ? j - 1 : -2, k0, hnn);
    ld(ub, g == R - 1 ? j + 1 : -2, k0, hsn);
    for (int k = k0; k < k1; ++k) {
        T hn[kE], hs[kE];
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            up[q] = upn[q];
            bv[q] = bvn[q];
            hn[q] = hnn[q];
            hs[q] = hsn[q];
        }
        gxm = gxmn;
        gxp = gxpn;
        if (k + 1 < k1) {
            ld(ub, j, k + 2, upn);
            ld(bb, j, k + 1, bvn);
            // y neighbours at the block edges come from memory (row -1 reads as zero)
            ld(ub, g == 0 ? j - 1 : -2, k + 1, hnn);
            ld(ub, g == R - 1 ? j + 1 : -2, k + 1, hsn);
            if (xlo)
                gxmn = *ghost_x(d, ghost, j, k + 1);
            if (xhi)
                gxpn = ghost_x(d, ghost, j, k + 1)[xpo];
        }
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            T a = __shfl_up_sync(0xffffffffu, uc[q], G);
            T c = __shfl_down_sync(0xffffffffu, uc[q], G);
            un[q] = (g == 0) ? hn[q] : a;
            us[q] = (g == R - 1) ? hs[q] : c;
        }
#pragma unroll
        for (int q = 0; q < kE; ++q)
            r[q] = (xin && jin) ? fma(az, um[q] + up[q], fma(ay, un[q] + us[q], bv[q])) : T(0);
        if (xlo)
            r[0] = fma(ax, gxm, r[0]);
        if (xhi) {
#pragma unroll
            for (int q = 0; q < kE; ++q)
                if (x0 + q == nx - 1)
                    r[q] = fma(ax, gxp, r[q]);
        }
        brs::line_solve<T, kE, G>(r, tb, l);
        T v[kE];
#pragma unroll
        for (int q = 0; q < kE; ++q)
            v[q] = fma(tb.wp[q], r[q], om1 * uc[q]);
        if (xin && jin) {
            T* p = uo + (long long)k * plane + (long long)j * nx + x0;
            if (d.vec && sizeof(T) == 4) {
                *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1],
                                                            (float)v[2], (float)v[3]);
            } else {
#pragma unroll
                for (int q = 0; q < kE; ++q)
                    if (x0 + q < nx)
                        p[q] = v[q];
            }
        }
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            um[q] = GS ? ((xin && jin) ? v[q] : T(0)) : uc[q];
            uc[q] = up[q];
        }
    }
}

// 16-byte asynchronous copy global -> shared (per thread); src_bytes = 0 writes zeros
// without reading global memory (rows and planes outside the patch).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
// 4-byte variant (through L1), for the staged x ghosts of a level
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Same work item as batched_item, with the per-step inputs (u(k+1), b(k) and, for the
// lines at the y-block edges, the halo lines j-1 / j+1 of plane k) staged by cp.async
// through a per-warp ring of D steps in shared memory.  Every patch row is a
// multiple of 16 bytes (checked on the host).  Each lane copies and reads back only its
// own 16-byte pieces, so no cross-lane synchronisation is needed.
template <typename T, int G, bool GS, int D, bool LV>
__device__ __forceinline__ void batched_item_async(const PatchDesc& d, int jb, int kc, int KC,
                                                   const T* uin, T* uout,
                                                   const T* __restrict__ b,
                                                   const T* __restrict__ tab, T ax, T ay, T az,
                                                   T om1, const T* ghost, unsigned char* ring,
                                                   T* gnext, const long long* pp)
{
    constexpr int R = 32 / G;
    constexpr int CH = (int)(kE * sizeof(T) / 16);  // 16-byte chunks per lane and field
    const int lanew = threadIdx.x & 31;
    const int g = lanew / G, l = lanew % G;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int j = jb * R + g;
    const bool jin = j < ny;
    const int x0 = l * kE;
    const bool xin = x0 < nx;
    const long long plane = (long long)nx * ny;
    const T* ub = uin + d.off;
    T* uo = uout + d.off;
    const T* bb = b + d.off;
    brs::LineTables<T, kE, G> tb;
    tb.load(tab + d.tab, l);
    const int k0 = kc * KC;
    const int k1 = min(nz, k0 + KC);
    const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(ring);
    // byte offset of (slot, field, chunk) for this lane
    auto soff = [&](int slot, int f, int c) -> uint32_t {
        return (uint32_t)((((slot * kFields + f) * CH + c) * 32 + lanew) * 16);
    };
    // Rows of u this item may need from outside the patch (a level's ghost block, else
    // none): row j of the z- and z+ faces, and the y- / y+ face rows of its edge lines.
    const T* gzm = nullptr;
    const T* gzp = nullptr;
    const T* gym = nullptr;
    const T* gyp = nullptr;
    if (LV) {
        gzm = outside_row(d, ghost, j, -1);
        gzp = outside_row(d, ghost, j, nz);
        gym = outside_row(d, ghost, -1, 0);   // + kk * nx for plane kk
        gyp = outside_row(d, ghost, ny, 0);
    }
    // row (jj, kk) of src: inside the patch, else the ghost row (u of a level), else zeros
    auto row_of = [&](const T* src, int jj, int kk) -> const T* {
        if (jj >= 0 && jj < ny && kk >= 0 && kk < nz)
            return src + (long long)kk * plane + (long long)jj * nx;
        if (!LV || src != ub)
            return nullptr;
        if (kk == -1)
            return jj == j ? gzm : nullptr;
        if (kk == nz)
            return jj == j ? gzp : nullptr;
        if (jj == -1)
            return gym ? gym + (long long)kk * nx : nullptr;
        if (jj == ny)
            return gyp ? gyp + (long long)kk * nx : nullptr;
        return nullptr;
    };
    // The steps' rows are issued for consecutive planes k0, k0 + 1, ...: their element
    // offsets advance by one plane (a y face's ghost rows by nx) per step, and whether
    // each field's row exists is fixed per item.  (The generic selection of row_of on
    // every copy cost about a fifth of the kernel's instructions.)
    long long o_next = (long long)k0 * plane + (long long)j * nx + x0;  // row (j, k) at x0
    const bool ok_b = xin && jin;
    const bool ok_n = xin && j >= 1 && j <= ny;  // line j - 1 inside the patch
    const bool ok_s = xin && j + 1 < ny;         // line j + 1
    // a level's rows outside the patch: u(k+1) of line ny is the y+ ghost row, and the
    // halo lines at the patch's y faces are the y- / y+ ghost rows
    long long og_next = (long long)k0 * nx + x0;
    const bool ok_0 = xin && (jin || (j == ny && gyp));
    const bool ok_gn = xin && (j > 0 || gym);
    const bool ok_gs = xin && (j + 1 < ny || (j + 1 == ny && gyp));
    auto copy_at = [&](int slot, int f, const T* src, long long o, bool ok) {
        const T* p = ok ? src + o : ub;
#pragma unroll
        for (int c = 0; c < CH; ++c)
            cp_async16(ring0 + soff(slot, f, c), p + c * (16 / sizeof(T)), ok ? 16u : 0u);
    };
    // x ghosts of the line (level contexts): the lanes holding x = 0 and x = nx - 1
    const bool xlo = LV && xin && jin && x0 == 0;
    const bool xhi = LV && xin && jin && x0 <= nx - 1 && nx - 1 < x0 + kE;
    // a level step that writes the next step's ghosts (gnext set): the y- and z-face rows
    // its lines feed are stored as the steps produce them, from registers (row k of a y face
    // at o + k nx, row j of a z face at o + j nx; pp: the patch's six push offsets).  Lines
    // 0 and ny - 1 are distinct when ny > 1; a one-line patch leaves its y faces to push_item.
    long long gy = -1;  // this lane's piece of the y-face row of plane k, or -1
    if (LV && gnext && xin && ny > 1 && (j == 0 || j == ny - 1)) {
        const long long o = __ldg(pp + (j == 0 ? 2 : 3));
        if (o >= 0)
            gy = o + (long long)k0 * nx + x0;
    }
    // the item's x ghosts, staged once: xg[face][k - k0][line in the warp], copied
    // asynchronously with the first step's inputs (zero beyond the last line)
    T* xg = reinterpret_cast<T*>(ring + (size_t)D * kFields * 32 * kE * sizeof(T));
    if (LV) {
        // x faces are [k][j] in the ghost block: element (kk, jl) of the item at
        // xb + face * xpo + kk * ny + jl (R a power of two: no divisions)
        const long long xpo = round4((long long)ny * nz);
        const int nk = k1 - k0;
        const uint32_t xg0 = (uint32_t)__cvta_generic_to_shared(xg);
        const T* xb = ghost_x(d, ghost, jb * R, k0);
        for (int face = 0; face < 2; ++face)
            for (int idx = lanew; idx < nk * R; idx += 32) {
                const int kk = idx / R, jl = idx % R;
                const bool ok = jb * R + jl < ny;
                const T* src = ok ? xb + (face ? xpo : 0) + (long long)kk * ny + jl : ghost;
                cp_async4(xg0 + (uint32_t)(((face * kMaxKC + kk) * 8 + jl) * sizeof(T)), src,
                          ok ? 4u : 0u);
            }
    }
    auto issue = [&](int kk, int slot) {
        if constexpr (LV) {
            // the rows this step can need outside the patch are known per field: u(k+1)
            // crosses the z+ face on the last plane, the halo lines cross the y faces, and
            // line ny (past the patch, in the last y-block) carries the y+ ghost row that
            // its neighbour ny - 1 takes by shuffle (og: row kk of a y face, at x0)
            const long long o = o_next, og = og_next;
            o_next += plane;
            og_next += nx;
            if (kk + 1 < nz)
                copy_at(slot, 0, jin ? ub : gyp, jin ? o + plane : og + nx, ok_0);
            else
                copy_at(slot, 0, gzp, x0, xin && gzp);
            copy_at(slot, 1, bb, o, ok_b);
            if (g == 0)
                copy_at(slot, 2, j > 0 ? ub : gym, j > 0 ? o - nx : og, ok_gn);
            if (g == R - 1)
                copy_at(slot, 3, j + 1 < ny ? ub : gyp, j + 1 < ny ? o + nx : og, ok_gs);
        } else {
            const long long o = o_next;  // row (j, kk): issue runs for kk = k0, k0 + 1, ...
            o_next += plane;
            copy_at(slot, 0, ub, o + plane, ok_b && kk + 1 < nz);
            copy_at(slot, 1, bb, o, ok_b);
            if (g == 0)
                copy_at(slot, 2, ub, o - nx, ok_n);
            if (g == R - 1)
                copy_at(slot, 3, ub, o + nx, ok_s);
        }
    };
    auto read = [&](int slot, int f, T (&v)[kE]) {
#pragma unroll
        for (int c = 0; c < CH; ++c)
            reinterpret_cast<float4*>(v)[c] =
                *reinterpret_cast<const float4*>(ring + soff(slot, f, c));
    };
    auto ld = [&](const T* src, int jj, int kk, T (&v)[kE]) {
        const T* row = row_of(src, jj, kk);
        if (xin && row) {
            const T* p = row + x0;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                reinterpret_cast<float4*>(v)[c] = reinterpret_cast<const float4*>(p)[c];
        } else {
#pragma unroll
            for (int q = 0; q < kE; ++q)
                v[q] = T(0);
        }
    };

    T um[kE], uc[kE], up[kE], r[kE], bv[kE], un[kE], us[kE], hn[kE], hs[kE];
    ld(ub, j, k0 - 1, um);
    ld(ub, j, k0, uc);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (k0 + i < k1)
            issue(k0 + i, i);
        cp_async_commit();
    }
    if (LV) {  // the x ghosts (first group) have landed and every lane sees them
        cp_async_wait<D - 1>();
        __syncwarp();
    }
    int slot = 0;
    for (int k = k0; k < k1; ++k) {
        cp_async_wait<D - 1>();  // the group of step k (committed D groups ago) is complete
        read(slot, 0, up);
        read(slot, 1, bv);
        if (g == 0)
            read(slot, 2, hn);
        if (g == R - 1)
            read(slot, 3, hs);
        T gxm = T(0), gxp = T(0);
        if (LV) {
            if (xlo)
                gxm = xg[(k - k0) * 8 + g];
            if (xhi)
                gxp = xg[(kMaxKC + k - k0) * 8 + g];
        }
#pragma unroll
        for (int q = 0; q < kE; ++q) {
            T a = __shfl_up_sync(0xffffffffu, uc[q], G);
            T c = __shfl_down_sync(0xffffffffu, uc[q], G);
            un[q] = (g == 0) ? hn[q] : a;
            us[q] = (g == R - 1) ? hs[q] : c;
        }
#pragma unroll
        for (int q = 0; q < kE; ++q)
            r[q] = (xin && jin) ? fma(az, um[q] + up[q], fma(ay, un[q] + us[q], bv[q])) : T(0);
        if (xlo)
            r[0] = fma(ax, gxm, r[0]);
        if (xhi) {
#pragma unroll
            for (int q = 0; q < kE; ++q)
                if (x0 + q == nx - 1)
                    r[q] = fma(ax, gxp, r[q]);
        }
        brs::line_solve<T, kE, G>(r, tb, l);
        T v[kE];
#pragma unroll
        for (int q = 0; q < kE; ++q)
            v[q] = fma(tb.wp[q], r[q], om1 * uc[q]);
        if (xin && jin) {
            T* p = uo + (long long)k * plane + (long long)j * nx + x0;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                reinterpret_cast<float4*>(p)[c] = reinterpret_cast<const float4*>(v)[c];
        }
        if constexpr (LV) {
            if (gy >= 0) {
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    reinterpret_cast<float4*>(gnext + gy)[c] = reinterpret_cast<const float4*>(v)[c];
                gy += nx;
            }
            if (gnext && (k == 0 || k == nz - 1) && xin && jin) {  // k is the same for the warp
#pragma unroll
                for (int f = 4; f < 6; ++f) {
                    const long long o = (f == 4 ? k == 0 : k == nz - 1) ? __ldg(pp + f) : -1;
                    if (o >= 0) {
                        T* p = gnext + o + (long long)j * nx + x0;
#pragma unroll
                        for (int c = 0; c < CH; ++c)
                            reinterpret_cast<float4*>(p)[c] = reinterpret_cast<const float4*>(v)[c];
                    }
                }
            }
        }

#pragma unroll
        for (int q = 0; q < kE; ++q) {
            um[q] = GS ? ((xin && jin) ? v[q] : T(0)) : uc[q];
            uc[q] = up[q];
        }
        // refill the slot just read (its values have been consumed above)
        if (k + D < k1)
            issue(k + D, slot);
        cp_async_commit();
        slot = slot + 1 == D ? 0 : slot + 1;
    }
    cp_async_wait<0>();  // only empty groups remain; the ring is free for the next item
    __syncwarp();        // and every lane has read the staged x ghosts
}

template <typename T, bool GS, int D, bool LV>
__global__ void __launch_bounds__(512) batched_async_kernel(const PatchDesc* __restrict__ desc,
                                                            const int* __restrict__ item_patch,
                                                            int nitems, int* counter, int KC,
                                                            const T* uin, T* uout,
                                                            const T* __restrict__ b,
                                                            const T* __restrict__ tab,
                                                            double ax, double ay, double az,
                                                            double om1, const T* ghost,
                                                            T* gnext,
                                                            const long long* __restrict__ push)
{
    extern __shared__ __align__(16) unsigned char async_smem[];
    pdl_wait_trigger();
    const int lanew = threadIdx.x & 31;
    unsigned char* ring =
        async_smem + (size_t)(threadIdx.x >> 5) * async_ring_bytes(D, sizeof(T), LV);
    while (true) {
        int item = 0;
        if (lanew == 0)
            item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems)
            return;
        const int pq = item_patch[item];
        const PatchDesc d = desc[pq];
        const int local = item - d.item0;
        const int jb = local % d.njb, kc = local / d.njb;
        const long long* pp = push ? push + 6 * pq : nullptr;
        switch (d.cls) {
        case 0: batched_item_async<T, 4, GS, D, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost, ring, gnext, pp); break;
        case 1: batched_item_async<T, 8, GS, D, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost, ring, gnext, pp); break;
        case 2: batched_item_async<T, 16, GS, D, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost, ring, gnext, pp); break;
        default: batched_item_async<T, 32, GS, D, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost, ring, gnext, pp); break;
        }
        if (LV && gnext)
            push_item<T>(desc, push, gnext, uout, item_patch[item], item, KC, true);
    }
}

// Ghost exchange of a level (Sec. 2: ghost cells updated in a Jacobi fashion after each
// complete smoothing step): every patch's ghost block receives its face neighbours' adjacent
// layers of u (zero where a face is the physical boundary).  One thread per ghost element,
// chunks of 256 elements per patch; the sweep that follows reads these values wherever its
// stencil leaves the patch.
template <typename T>
__global__ void __launch_bounds__(256) level_exchange_kernel(const PatchDesc* __restrict__ desc,
                                                             const int* __restrict__ chunk_patch,
                                                             const int* __restrict__ nbr,
                                                             const T* u, T* __restrict__ ghost)
{
    pdl_wait_trigger();
    const int p = __ldg(chunk_patch + blockIdx.x);
    const int nx = __ldg(&desc[p].nx), ny = __ldg(&desc[p].ny), nz = __ldg(&desc[p].nz);
    const int t = (int)(blockIdx.x - __ldg(&desc[p].bchunk0)) * (int)blockDim.x + threadIdx.x;
    const int A = (int)round4((long long)nx * ny), Bz = (int)round4((long long)nx * nz);
    const int C = (int)round4((long long)ny * nz);
    if (t >= 2 * (A + Bz + C))
        return;
    auto at = [&](int q, int ii, int jj, int kk) -> T {
        const int qx = __ldg(&desc[q].nx), qy = __ldg(&desc[q].ny);
        return u[__ldg(&desc[q].off) + ii + (long long)qx * (jj + (long long)qy * kk)];
    };
    const int* nb = nbr + 6 * p;
    T v = T(0);
    if (t < 2 * A) {  // z faces, [j][i]
        const bool hi = t >= A;
        const int r = hi ? t - A : t;
        if (r >= nx * ny)
            return;  // padding
        const int j = r / nx, i = r - j * nx;
        const int q = __ldg(nb + (hi ? 5 : 4));
        if (q >= 0)
            v = at(q, i, j, hi ? 0 : __ldg(&desc[q].nz) - 1);
    } else if (t < 2 * A + 2 * Bz) {  // y faces, [k][i]
        const int t2 = t - 2 * A;
        const bool hi = t2 >= Bz;
        const int r = hi ? t2 - Bz : t2;
        if (r >= nx * nz)
            return;
        const int k = r / nx, i = r - k * nx;
        const int q = __ldg(nb + (hi ? 3 : 2));
        if (q >= 0)
            v = at(q, i, hi ? 0 : __ldg(&desc[q].ny) - 1, k);
    } else {  // x faces, [k][j]
        const int t3 = t - 2 * A - 2 * Bz;
        const bool hi = t3 >= C;
        const int r = hi ? t3 - C : t3;
        if (r >= ny * nz)
            return;
        const int k = r / ny, j = r - k * ny;
        const int q = __ldg(nb + (hi ? 1 : 0));
        if (q >= 0)
            v = at(q, hi ? 0 : __ldg(&desc[q].nx) - 1, j, k);
    }
    ghost[__ldg(&desc[p].g0) + t] = v;
}

template <typename T, bool GS, bool LV>
__global__ void __launch_bounds__(512) batched_line_kernel(const PatchDesc* __restrict__ desc,
                                                           const int* __restrict__ item_patch,
                                                           int nitems, int* counter, int KC,
                                                           const T* uin, T* uout,
                                                           const T* __restrict__ b,
                                                           const T* __restrict__ tab,
                                                           double ax, double ay, double az,
                                                           double om1, const T* ghost,
                                                           T* gnext,
                                                           const long long* __restrict__ push)
{
    pdl_wait_trigger();
    const int lanew = threadIdx.x & 31;
    while (true) {
        int item = 0;
        if (lanew == 0)
            item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems)
            return;
        const int pq = item_patch[item];
        const PatchDesc d = desc[pq];
        const int local = item - d.item0;
        const int jb = local % d.njb, kc = local / d.njb;
        switch (d.cls) {
        case 0: batched_item<T, 4, GS, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost); break;
        case 1: batched_item<T, 8, GS, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost); break;
        case 2: batched_item<T, 16, GS, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost); break;
        default: batched_item<T, 32, GS, LV>(d, jb, kc, KC, uin, uout, b, tab, (T)ax, (T)ay, (T)az, (T)om1, ghost); break;
        }
        if (LV && gnext)
            push_item<T>(desc, push, gnext, uout, item_patch[item], item, KC, false);
    }
}

// FP32 only (the FP64 item does not fit the register budget with its ring addressing)
template <bool LV>
const void* async_kernel_lv(bool gs, int stages)
{
    if (stages >= 8)
        return gs ? (const void*)batched_async_kernel<float, true, 8, LV>
                  : (const void*)batched_async_kernel<float, false, 8, LV>;
    if (stages >= 6)
        return gs ? (const void*)batched_async_kernel<float, true, 6, LV>
                  : (const void*)batched_async_kernel<float, false, 6, LV>;
    return gs ? (const void*)batched_async_kernel<float, true, 4, LV>
              : (const void*)batched_async_kernel<float, false, 4, LV>;
}

const void* async_kernel_for(bool gs, int stages, bool level)
{
    return level ? async_kernel_lv<true>(gs, stages) : async_kernel_lv<false>(gs, stages);
}

template <bool LV>
const void* kernel_lv(int dtype, bool gs)
{
    if (dtype == BRS_F64)
        return gs ? (const void*)batched_line_kernel<double, true, LV>
                  : (const void*)batched_line_kernel<double, false, LV>;
    return gs ? (const void*)batched_line_kernel<float, true, LV>
              : (const void*)batched_line_kernel<float, false, LV>;
}

const void* kernel_for(int dtype, bool gs, bool level)
{
    return level ? kernel_lv<true>(dtype, gs) : kernel_lv<false>(dtype, gs);
}

// Line tables of one nx for E = 4 and G lanes (same layout and recurrences as the
// single-grid line path).
std::vector<double> tables_for(int nx, int G, const brs_params& p, double omega)
{
    return scan_thomas_tables<double>(nx, p.ax, 2.0 * (p.ax + p.ay + p.az), omega, kE, G, false);
}

int build_items(brs_ctx* c, int KC)
{
    BatchState* B = bs(c);
    B->h_item_patch.clear();
    int item = 0;
    for (int q = 0; q < B->npatch; ++q) {
        PatchDesc& d = B->h_desc[q];
        const int G = 4 << d.cls, R = 32 / G;
        d.njb = (d.ny + R - 1) / R;
        d.nkc = (d.nz + KC - 1) / KC;
        d.item0 = item;
        const int n = d.njb * d.nkc;
        for (int t = 0; t < n; ++t)
            B->h_item_patch.push_back(q);
        item += n;
    }
    B->nitems = item;
    B->KC = KC;
    if (B->d_desc)
        cudaFree(B->d_desc);
    if (B->d_item_patch)
        cudaFree(B->d_item_patch);
    B->d_desc = nullptr;
    B->d_item_patch = nullptr;
    cudaError_t e = cudaMalloc(&B->d_desc, sizeof(PatchDesc) * B->npatch);
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_desc, B->h_desc.data(), sizeof(PatchDesc) * B->npatch,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&B->d_item_patch, sizeof(int) * std::max(1, item));
    if (e == cudaSuccess && item > 0)
        e = cudaMemcpy(B->d_item_patch, B->h_item_patch.data(), sizeof(int) * item,
                       cudaMemcpyHostToDevice);
    return brs_cuda_status(e);
}

int ensure_counters(BatchState* B, int n)
{
    if (B->ncounters >= n)
        return BRS_OK;
    if (B->d_counters)
        cudaFree(B->d_counters);
    B->d_counters = nullptr;
    B->ncounters = 0;
    cudaError_t e = cudaMalloc(&B->d_counters, sizeof(int) * n);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    B->ncounters = n;
    return BRS_OK;
}

int launch_one(brs_ctx* c, const void* uin, void* uout, const void* b, int* counter,
               cudaStream_t s, const void* ghost = nullptr, void* gnext = nullptr)
{
    BatchState* B = bs(c);
    const bool gs = c->p.method == BRS_CHAOTIC_GS;
    const void* k = B->async ? async_kernel_for(gs, B->stages, B->level)
                             : kernel_for(c->p.dtype, gs, B->level);
    const size_t smem =
        B->async ? (size_t)B->warps * async_ring_bytes(B->stages, c->esize, B->level) : 0;
    const PatchDesc* desc = B->d_desc;
    const int* ip = B->d_item_patch;
    int nitems = B->nitems, KC = B->KC;
    const void* tab = B->d_tab;
    double ax = c->p.ax, ay = c->p.ay, az = c->p.az, om1 = 1.0 - c->omega;
    // ghost: the buffer this step reads (null unless the context is a level); gnext: the
    // one its face pushes go to (null: no pushes)
    const long long* push = B->d_push;
    void* args[] = {(void*)&desc, (void*)&ip, &nitems, &counter, &KC, (void*)&uin, &uout,
                    (void*)&b, (void*)&tab, &ax, &ay, &az, &om1, (void*)&ghost, &gnext,
                    (void*)&push};
    return brs_cuda_status(launch_pdl_c(k, dim3(B->grid), dim3(B->warps * 32), smem, s, args));
}

int level_exchange(brs_ctx* c, const void* u, void* ghost, cudaStream_t s)
{
    BatchState* B = bs(c);
    const PatchDesc* desc = B->d_desc;
    const int* cp = B->d_chunk_patch;
    const int* nb = B->d_nbr;
    cudaError_t e;
    if (c->p.dtype == BRS_F64)
        e = launch_pdl(level_exchange_kernel<double>, dim3(B->nchunks), dim3(256), 0, s, desc, cp,
                       nb, static_cast<const double*>(u), static_cast<double*>(ghost));
    else
        e = launch_pdl(level_exchange_kernel<float>, dim3(B->nchunks), dim3(256), 0, s, desc, cp,
                       nb, static_cast<const float*>(u), static_cast<float*>(ghost));
    return brs_cuda_status(e);
}

// Enqueue one call's sweeps (counter reset + one launch per sweep) on stream s.
int enqueue_sweeps(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s)
{
    BatchState* B = bs(c);
    cudaError_t e = cudaMemsetAsync(B->d_counters, 0, sizeof(int) * nsweeps, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    const bool gs = c->p.method == BRS_CHAOTIC_GS;
    void* cur = u;
    void* nxt = gs ? u : c->scratch;
    int rc = BRS_OK;
    const bool chain = B->level && B->push && B->keep;
    const int par0 = chain ? B->gpar : 0;
    for (int k = 0; k < nsweeps && rc == BRS_OK; ++k) {
        void* gcur = nullptr;
        void* gnext = nullptr;
        if (B->level) {
            // the call's first step gathers its ghost layer from the iterate (unless the
            // previous call left it, ghosts kept across calls); every step but the last (every
            // step, when kept) then writes the next step's ghosts as it computes its faces
            // (two buffers, alternating)
            const int idx = (par0 + k) & 1;
            gcur = (B->push && idx) ? B->ghost2 : B->ghost;
            if (!B->push || (k == 0 && !(chain && B->gvalid)))
                rc = level_exchange(c, cur, gcur, s);
            if (B->push && (k + 1 < nsweeps || chain))
                gnext = idx ? B->ghost : B->ghost2;
        }
        if (rc == BRS_OK)
            rc = launch_one(c, cur, nxt, b, B->d_counters + k, s, gcur, gnext);
        if (!gs)
            std::swap(cur, nxt);
    }
    if (rc == BRS_OK && cur != u)
        rc = brs_cuda_status(cudaMemcpyAsync(u, cur, (size_t)B->total * c->esize,
                                             cudaMemcpyDeviceToDevice, s));
    return rc;
}

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

void set_shape(brs_ctx* c, int warps, int ctas_per_sm)
{
    BatchState* B = bs(c);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    B->warps = warps;
    B->grid = std::max(1, sms * ctas_per_sm);
}

// Autotuner: time each candidate (z-chunk, warps per CTA, CTAs per SM) on scratch
// arrays of the real patch set and keep the fastest.  Results are cached per process
// keyed by the patch set, dtype and method.
struct TuneKey {
    std::vector<int> dims;
    int dtype, method;
    bool operator<(const TuneKey& o) const
    {
        if (dtype != o.dtype) return dtype < o.dtype;
        if (method != o.method) return method < o.method;
        return dims < o.dims;
    }
};
struct TuneVal {
    int KC, warps, cps;
};
std::map<TuneKey, TuneVal> g_tune_cache;
std::mutex g_tune_mutex;

int autotune(brs_ctx* c)
{
    BatchState* B = bs(c);
    TuneKey key{B->dims, c->p.dtype, c->p.method};
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            set_shape(c, it->second.warps, it->second.cps);
            return build_items(c, it->second.KC);
        }
    }
    int fixed_kc = env_int("BRSMOOTH_BATCH_KC", 0);
    fixed_kc = fixed_kc > kMaxKC ? kMaxKC : fixed_kc;
    std::vector<TuneVal> cands;
    for (int kc : {4, 8, 16, 32})
        for (int w : {4, 8, 16})
            for (int cps : {2, 4, 8}) {
                if (w * cps > 64)
                    continue;
                if (B->async &&
                    ((size_t)w * cps * async_ring_bytes(B->stages, c->esize, true) > 220u * 1024u ||
                     (size_t)w * async_ring_bytes(B->stages, c->esize, true) > 227u * 1024u))
                    continue;  // the rings of every resident warp must fit one SM
                if (fixed_kc && kc != fixed_kc)
                    continue;
                cands.push_back({kc, w, cps});
            }
    const size_t bytes = (size_t)B->total * c->esize;
    void *tu = nullptr, *tb = nullptr;
    cudaError_t e = cudaMalloc(&tu, bytes);
    if (e == cudaSuccess)
        e = cudaMalloc(&tb, bytes);
    if (e == cudaSuccess)
        e = cudaMemset(tu, 0, bytes);
    if (e == cudaSuccess)
        e = cudaMemset(tb, 0, bytes);
    int rc = brs_cuda_status(e);
    if (rc == BRS_OK)
        rc = ensure_counters(B, 8);  // the timed calls run up to 5 sweeps
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == BRS_OK) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    TuneVal best{8, 8, 4};
    float best_ms = 1e30f;
    for (const TuneVal& v : cands) {
        if (rc != BRS_OK)
            break;
        set_shape(c, v.warps, v.cps);
        rc = build_items(c, v.KC);
        if (rc != BRS_OK)
            break;
        rc = enqueue_sweeps(c, tu, tb, 1, nullptr);  // warm
        // best of two 5-sweep timings: one short timing picked shapes 8 % apart run to run
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && rc == BRS_OK; ++rep) {
            cudaEventRecord(e0, nullptr);
            rc = enqueue_sweeps(c, tu, tb, 5, nullptr);
            cudaEventRecord(e1, nullptr);
            if (cudaEventSynchronize(e1) != cudaSuccess && rc == BRS_OK)
                rc = BRS_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = t < ms ? t : ms;
        }
        if (rc == BRS_OK && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (tu)
        cudaFree(tu);
    if (tb)
        cudaFree(tb);
    if (rc != BRS_OK)
        return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    set_shape(c, best.warps, best.cps);
    return build_items(c, best.KC);
}

}  // namespace

int batched_setup(brs_ctx* c, int npatch, const int* dims)
{
    BatchState* B = new BatchState();
    c->batch = B;
    B->npatch = npatch;
    B->dims.assign(dims, dims + 3 * npatch);
    std::map<int, int> tab_off;  // nx -> table offset
    std::vector<double> tabs;
    long long off = 0;
    const long long align = 16 / (long long)c->esize;
    for (int q = 0; q < npatch; ++q) {
        PatchDesc d{};
        d.nx = dims[3 * q];
        d.ny = dims[3 * q + 1];
        d.nz = dims[3 * q + 2];
        d.cls = d.nx <= 16 ? 0 : d.nx <= 32 ? 1 : d.nx <= 64 ? 2 : 3;
        d.off = off;
        d.vec = (d.nx % 4 == 0) && (off % align == 0) && (d.nx * (long long)c->esize) % 16 == 0;
        const int G = 4 << d.cls;
        const int key = d.nx;
        if (!tab_off.count(key)) {
            tab_off[key] = (int)tabs.size();
            auto t = tables_for(d.nx, G, c->p, c->omega);
            tabs.insert(tabs.end(), t.begin(), t.end());
        }
        d.tab = tab_off[key];
        B->h_desc.push_back(d);
        off += (long long)d.nx * d.ny * d.nz;
    }
    B->total = off;
    c->cells = off;
    cudaError_t e;
    if (c->p.dtype == BRS_F64) {
        e = cudaMalloc(&B->d_tab, tabs.size() * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(B->d_tab, tabs.data(), tabs.size() * sizeof(double),
                           cudaMemcpyHostToDevice);
    } else {
        std::vector<float> tf(tabs.begin(), tabs.end());
        e = cudaMalloc(&B->d_tab, tf.size() * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemcpy(B->d_tab, tf.data(), tf.size() * sizeof(float),
                           cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    if (c->p.method == BRS_JACOBI) {
        e = cudaMalloc(&c->scratch, (size_t)B->total * c->esize);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
    }
    // cp.async kernel when every patch row is a whole number of aligned 16-byte pieces
    B->async = c->p.dtype == BRS_F32 && env_int("BRSMOOTH_BATCH_ASYNC", 1) != 0;
    for (const PatchDesc& d : B->h_desc)
        B->async = B->async && d.vec;
    B->stages = env_int("BRSMOOTH_BATCH_STAGES", 4);
    B->stages = B->stages >= 8 ? 8 : B->stages >= 6 ? 6 : 4;
    if (B->async) {
        // both the plain and the level kernel (a level is set up after the tuner ran)
        for (bool lv : {false, true}) {
            const size_t want =
                std::min<size_t>(227u * 1024u, 16 * async_ring_bytes(B->stages, c->esize, lv));
            const void* k = async_kernel_for(c->p.method == BRS_CHAOTIC_GS, B->stages, lv);
            cudaFuncAttributes fa{};
            e = cudaFuncGetAttributes(&fa, k);
            if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < want)
                e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)want);
            if (e != cudaSuccess)
                return brs_cuda_status(e);
        }
    }
    int kc = env_int("BRSMOOTH_BATCH_KC", 0);
    kc = kc > kMaxKC ? kMaxKC : kc;  // a level stages at most kMaxKC z-steps of x ghosts
    if (env_int("BRSMOOTH_BATCH_NOTUNE", 0)) {
        set_shape(c, 8, B->async ? 2 : 4);
        return build_items(c, kc ? kc : 8);
    }
    return autotune(c);
}

int level_setup(brs_ctx* c, const int* nbr)
{
    BatchState* B = bs(c);
    B->level = true;
    // boundary-cell chunks per patch (every dim >= 2, checked by the caller)
    std::vector<int> chunk_patch;
    long long gtotal = 0;
    for (int q = 0; q < B->npatch; ++q) {
        PatchDesc& d = B->h_desc[q];
        const long long gb = ghost_block(d.nx, d.ny, d.nz);
        if (gb >= (1ll << 31))
            return BRS_ERR_UNSUPPORTED;  // the exchange kernel numbers ghosts in 32 bits
        d.g0 = gtotal;
        gtotal += gb;
        d.bchunk0 = (int)chunk_patch.size();
        for (long long t = 0; t < (gb + 255) / 256; ++t)
            chunk_patch.push_back(q);
    }
    B->nchunks = (int)chunk_patch.size();
    cudaError_t e = cudaMemcpy(B->d_desc, B->h_desc.data(), sizeof(PatchDesc) * B->npatch,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&B->d_chunk_patch, sizeof(int) * chunk_patch.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_chunk_patch, chunk_patch.data(), sizeof(int) * chunk_patch.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&B->d_nbr, sizeof(int) * 6 * B->npatch);
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_nbr, nbr, sizeof(int) * 6 * B->npatch, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&B->ghost, (size_t)gtotal * c->esize);
    if (e == cudaSuccess)
        e = cudaMemset(B->ghost, 0, (size_t)gtotal * c->esize);
    // face pushes: patch p's face f lands in the opposite ghost face of neighbour q
    // (x- -> q's x+, x+ -> q's x-, and so on); physical-boundary ghosts stay zero in both
    // buffers because nothing writes them
    B->push = env_int("BRSMOOTH_LEVEL_PUSH", 1) != 0;
    if (B->push) {
        std::vector<long long> push(6 * (size_t)B->npatch, -1);
        for (int p = 0; p < B->npatch; ++p)
            for (int f = 0; f < 6; ++f) {
                const int q = nbr[6 * p + f];
                if (q < 0)
                    continue;
                const PatchDesc& d = B->h_desc[q];
                const long long A = round4((long long)d.nx * d.ny);
                const long long Bz = round4((long long)d.nx * d.nz);
                const long long C = round4((long long)d.ny * d.nz);
                const long long face[6] = {2 * A + 2 * Bz + C, 2 * A + 2 * Bz, 2 * A + Bz,
                                           2 * A, A, 0};
                push[6 * (size_t)p + f] = d.g0 + face[f];
            }
        if (e == cudaSuccess)
            e = cudaMalloc(&B->ghost2, (size_t)gtotal * c->esize);
        if (e == cudaSuccess)
            e = cudaMemset(B->ghost2, 0, (size_t)gtotal * c->esize);
        if (e == cudaSuccess)
            e = cudaMalloc(&B->d_push, sizeof(long long) * push.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(B->d_push, push.data(), sizeof(long long) * push.size(),
                           cudaMemcpyHostToDevice);
    }
    return brs_cuda_status(e);
}

void batched_teardown(brs_ctx* c)
{
    BatchState* B = bs(c);
    if (!B)
        return;
    for (auto& g : B->graphs)
        cudaGraphExecDestroy(g.exec);
    for (void* q : {(void*)B->d_desc, (void*)B->d_item_patch, B->d_tab, (void*)B->d_counters,
                    (void*)B->d_nbr, (void*)B->d_chunk_patch, B->ghost, B->ghost2,
                    (void*)B->d_push})
        if (q)
            cudaFree(q);
    if (B->cap)
        cudaStreamDestroy(B->cap);
    delete B;
    c->batch = nullptr;
}

int batched_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s)
{
    BatchState* B = bs(c);
    if (nsweeps == 0)
        return BRS_OK;
    int rc = ensure_counters(B, nsweeps);
    if (rc != BRS_OK)
        return rc;
    const bool chain = B->level && B->push && B->keep;
    const int mode = chain ? (1 | (B->gvalid ? 2 : 0) | (B->gpar << 2)) : 0;
    // after this call the kept ghosts are valid and sit in the buffer its next step would read
    auto advance = [&]() {
        if (chain) {
            B->gpar = (B->gpar + nsweeps) & 1;
            B->gvalid = true;
        }
    };
    for (auto& g : B->graphs)
        if (g.u == u && g.b == b && g.nsweeps == nsweeps && g.mode == mode) {
            advance();
            return brs_cuda_status(cudaGraphLaunch(g.exec, s));
        }
    // capture this call's sweep sequence once on the private stream, replay on `s`
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    rc = enqueue_sweeps(c, u, b, nsweeps, B->cap);
    e = cudaStreamEndCapture(B->cap, &graph);
    if (rc != BRS_OK || e != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc != BRS_OK ? rc : brs_cuda_status(e);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    if (B->graphs.size() >= 8) {
        cudaGraphExecDestroy(B->graphs.front().exec);
        B->graphs.erase(B->graphs.begin());
    }
    B->graphs.push_back({u, b, nsweeps, mode, exec});
    advance();
    return brs_cuda_status(cudaGraphLaunch(exec, s));
}

int level_keep_ghosts(brs_ctx* c, int on)
{
    BatchState* B = bs(c);
    if (!B || !B->level)
        return BRS_ERR_ARG;
    B->keep = on != 0 && B->push;
    B->gvalid = false;
    B->gpar = 0;
    return BRS_OK;
}

void batched_describe(const brs_ctx* c, int* kc, int* warps, int* grid, int* nitems)
{
    const BatchState* B = static_cast<const BatchState*>(c->batch);
    *kc = B->KC;
    *warps = B->warps;
    *grid = B->grid;
    *nitems = B->nitems;
}
