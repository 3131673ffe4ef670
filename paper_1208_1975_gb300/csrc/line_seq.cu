// FP64 x-line sweeps with one thread per half line (Sec. 2, Alg. 1 / Alg. 2 with full
// x-line blocks, Thomas elimination from both ends of the line).
//
// On GB300 the FP64 pipe retires 2 fused multiply-adds per clock per SM, 1/64 of the FP32
// rate, while HBM would carry 24 bytes per cell at ~280 Gcell/s.  An FP64 line sweep is
// therefore bound by the number of FP64 operations per cell, and this path is laid out to
// need as few as the method allows:
//
//  * Sequential elimination, no cross-lane scan.  A line of nx cells is solved by two
//    threads: one eliminates from the left end (i = 0 .. m-1), one from the right end
//    (i = nx-1 .. m+1), they meet at the twist cell m = (nx-1)/2, and each then
//    back-substitutes outwards.  With the constant block M_line = tridiag(-ax, d, -ax),
//    d = 2(ax+ay+az), the pivots are the same for every line and are computed once in
//    FP64 on the host:
//        left   p_0 = 1/d,      p_i = 1/(d - ax^2 p_{i-1})      (i < m)
//        right  q_{n-1} = 1/d,  q_i = 1/(d - ax^2 q_{i+1})      (i > m)
//        twist  g_m = 1/(d - ax^2 p_{m-1} - ax^2 q_{m+1})
//    With pv_i the pivot of cell i (p_i, g_m or q_i), the damped update
//    v = (1-omega) u + omega M^{-1} rhs is computed in scaled variables
//        z_i = omega pv_i rhs_i + (ax pv_i) z_{i-1}        left elimination (z_{-1} = 0)
//        z_i = omega pv_i rhs_i + (ax pv_i) z_{i+1}        right elimination (z_n = 0)
//        y_m = omega g_m rhs_m + (ax g_m)(z_{m-1} + z_{m+1})
//        y_i = z_i + (ax pv_i) y_{i+1}   (i < m),  y_i = z_i + (ax pv_i) y_{i-1}  (i > m)
//        v_i = (1 - omega) u_i + y_i                       (y = omega M^{-1} rhs)
//    and omega pv_i rhs_i = omega pv_i b_i + (omega pv_i ay)(u_{j-1} + u_{j+1})
//    + (omega pv_i az)(u_{k-1} + u_{k+1}).  b does not change between sweeps, so
//    b'_i = omega pv_i b_i is formed once per call.  Per cell: 2 adds + 2 FMAs for the
//    gather, 1 FMA per elimination direction, 1 FMA for the update: 7 FP64 operations
//    (6 for Gauss-Seidel with omega = 1).
//  * Line-major, colour-split layout.  The call copies u and b into
//        P(i, k, c, t) = ((i nz + k) 2 + c) H + t,   c = (j + k) & 1,  t = j >> 1,
//    H = ceil(ny/2): for each cell index i along the lines, the lines of one row k are
//    stored by colour.  A warp takes 16 consecutive lines of one colour and row (two
//    threads per line), so every load and store of a step is two contiguous 128-byte runs,
//    and all four neighbour lines of a colour-c line have colour 1-c and sit in contiguous
//    runs as well.  The elimination writes z into the output buffer (Jacobi) or a scratch
//    buffer (Gauss-Seidel); back substitution reads it back in reverse order.
//  * Gauss-Seidel in two colours.  Lines with j+k even are updated first from the old
//    values of the odd lines, then the odd lines from the new even ones: the red-black
//    line order, one admissible order of the chaotic scheme (Alg. 1), deterministic, and
//    the same order as a lexicographic sweep over each colour.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>
#include <vector>

#include "brs_internal.cuh"

namespace {

constexpr int kLinesPerWarp = 16;

// Longest elimination: lines of at most 512 cells (the x-line limit), 256 steps per side.
constexpr int kSeqMaxSteps = 256;

// Launch arguments, passed in the kernel's parameter space (about 6 KB).  The pivots are
// symmetric: the right thread's pivot at step s, q_{n-1-s}, equals the left thread's p_s
// (both obey the same recurrence from 1/d), so one table indexed by the step serves both
// halves of the elimination with a warp-uniform index.
struct SeqArgs {
    int nx, ny, nz, H, m;   // grid, half-row width, twist cell
    long long SI;           // elements per i-slab: nz * 2H
    int tpb;                // 16-line blocks per (k, colour) row: ceil(H / 16)
    int colour;             // -1: all lines (Jacobi); 0/1: lines with (j+k)&1 == colour
    long long ntasks;       // warp tasks
    double om1;             // 1 - omega
    double ga, gb, gm;      // twist cell: omega g_m ay, omega g_m az, ax g_m
    double fa[kSeqMaxSteps];  // step s: omega p_s ay
    double fb[kSeqMaxSteps];  //         omega p_s az
    double fm[kSeqMaxSteps];  //         ax p_s
};

// Launch shape of one sweep launch: `grid` CTAs of `warps` warps, dependent launch or not.
struct Shape {
    int grid = 1, warps = 1;
    bool pdl = false;
};

struct SeqState {
    int H = 0;
    long long elems = 0;    // nx * nz * 2H
    double* tab = nullptr;  // per i: omega pv_i, the scale of b
    double* U0 = nullptr;   // iterate (line-major)
    double* U1 = nullptr;   // Jacobi second vector / Gauss-Seidel elimination scratch
    double* Bs = nullptr;   // b'_i = s_i b_i (line-major)
    Shape jac, gs;          // launch shapes: Jacobi sweep, one-colour launch
    int depth = 2;          // prefetch depth selector (twist_kernel)
    std::vector<double> pv; // pivots of the twisted elimination (per cell), FP64
};

SeqState* st(brs_ctx* c) { return static_cast<SeqState*>(c->lseq); }

// ---------------------------------------------------------------------------------------
// Copies between the caller's x-fastest layout and the line-major colour-split layout.
// Tiles of 32 cells along i by 32 lines along j at one k; scale (nullable) multiplies
// cell i by scale[i] on the way in.
constexpr int kTile = 32;

__global__ void __launch_bounds__(256) to_line_major(const double* __restrict__ src,
                                                     double* __restrict__ dst,
                                                     const double* __restrict__ scale, int nx,
                                                     int ny, int nz, int H, long long SI)
{
    __shared__ double tile[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int tiles_i = (nx + kTile - 1) / kTile;
    const int i0 = (blockIdx.x % tiles_i) * kTile;
    const int j0 = (blockIdx.x / tiles_i) * kTile;
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        for (int jj = ty; jj < kTile; jj += 8) {
            const int j = j0 + jj, i = i0 + tx;
            if (j < ny && i < nx)
                tile[jj][tx] = src[((size_t)k * ny + j) * nx + i];
        }
        __syncthreads();
        const int j = j0 + tx;
        const int c = (j + k) & 1, t = j >> 1;
        for (int ii = ty; ii < kTile; ii += 8) {
            const int i = i0 + ii;
            if (j < ny && i < nx) {
                double v = tile[tx][ii];
                if (scale)
                    v *= scale[i];
                dst[(size_t)i * SI + ((size_t)k * 2 + c) * H + t] = v;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) from_line_major(const double* __restrict__ src,
                                                       double* __restrict__ dst, int nx, int ny,
                                                       int nz, int H, long long SI)
{
    __shared__ double tile[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int tiles_i = (nx + kTile - 1) / kTile;
    const int i0 = (blockIdx.x % tiles_i) * kTile;
    const int j0 = (blockIdx.x / tiles_i) * kTile;
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        const int j = j0 + tx;
        const int c = (j + k) & 1, t = j >> 1;
        for (int ii = ty; ii < kTile; ii += 8) {
            const int i = i0 + ii;
            if (j < ny && i < nx)
                tile[tx][ii] = src[(size_t)i * SI + ((size_t)k * 2 + c) * H + t];
        }
        __syncthreads();
        for (int jj = ty; jj < kTile; jj += 8) {
            const int jr = j0 + jj, i = i0 + tx;
            if (jr < ny && i < nx)
                dst[((size_t)k * ny + jr) * nx + i] = tile[jj][tx];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// The sweep.  Warp task -> (k, colour, block of 16 lines); lanes 0-15 hold the left halves
// of lines t0..t0+15, lanes 16-31 the right halves of the same lines.
struct Gather {
    double b, yn, yp, zn, zp;
};

__device__ __forceinline__ double ld_if(const double* p, bool ok)
{
    return ok ? __ldg(p) : 0.0;
}

// DF / DB: cells of loads in flight per thread during elimination / back substitution.
// A CTA is any number of warps; warp w of CTA c takes tasks c + gridDim.x (w + W r).
template <bool OMEGA1, int DF, int DB>
__global__ void __launch_bounds__(1024) xline_twist_kernel(
    const double* uin, double* out, double* zs, const double* __restrict__ bs,
    const __grid_constant__ SeqArgs a)
{
    pdl_wait_trigger();
    const int lane = threadIdx.x & 31;
    const bool right = lane >= 16;
    const int nx = a.nx, m = a.m;
    const int Lc = m, Rc = nx - 1 - m;  // cells eliminated by the left / right thread
    const int cnt = right ? Rc : Lc;
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long task = blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5);
         task < a.ntasks; task += stride) {
        int k, c, tb;
        if (a.colour < 0) {
            tb = (int)(task % a.tpb);
            const long long kc = task / a.tpb;
            k = (int)(kc >> 1);
            c = (int)(kc & 1);
        } else {
            tb = (int)(task % a.tpb);
            k = (int)(task / a.tpb);
            c = a.colour;
        }
        const int t = tb * kLinesPerWarp + (lane & 15);
        const int p = (c + k) & 1;
        const int j = 2 * t + p;
        const bool ok = j < a.ny;
        const int co = c ^ 1;
        // offsets within an i-slab
        const long long own = ((long long)k * 2 + c) * a.H + t;
        const long long oyn = ((long long)k * 2 + co) * a.H + t - 1 + p;  // (j-1, k)
        const long long oyp = ((long long)k * 2 + co) * a.H + t + p;      // (j+1, k)
        const long long ozn = ((long long)(k - 1) * 2 + co) * a.H + t;    // (j, k-1)
        const long long ozp = ((long long)(k + 1) * 2 + co) * a.H + t;    // (j, k+1)
        const bool fyn = ok && j >= 1, fyp = ok && j + 1 < a.ny;
        const bool fzn = ok && k >= 1, fzp = ok && k + 1 < a.nz;

        auto load = [&](Gather& g, int i, bool on) {
            const long long o = (long long)i * a.SI;
            g.b = ld_if(bs + o + own, on && ok);
            g.yn = ld_if(uin + o + oyn, on && fyn);
            g.yp = ld_if(uin + o + oyp, on && fyp);
            g.zn = ld_if(uin + o + ozn, on && fzn);
            g.zp = ld_if(uin + o + ozp, on && fzp);
        };
        // elimination towards the twist cell, DF cells of loads in flight; step s uses the
        // pivot p_s on both sides
        double z = 0.0;
        Gather g[DF];
#pragma unroll
        for (int h = 0; h < DF; ++h)
            load(g[h], right ? nx - 1 - h : h, h < cnt);
#pragma unroll 1
        for (int s = 0; s < Rc; s += DF) {
#pragma unroll
            for (int h = 0; h < DF; ++h) {
                const int ss = s + h;
                const int i = right ? nx - 1 - ss : ss;
                if (ss < cnt) {
                    const double r =
                        fma(a.fb[ss], g[h].zn + g[h].zp, fma(a.fa[ss], g[h].yn + g[h].yp, g[h].b));
                    z = fma(a.fm[ss], z, r);
                    if (ok)
                        zs[(long long)i * a.SI + own] = z;
                }
                const int sn = ss + DF;
                load(g[h], right ? nx - 1 - sn : sn, sn < cnt);
            }
        }
        // twist cell: the left thread combines both eliminations
        const double zr = __shfl_xor_sync(0xffffffffu, z, 16);
        double y = 0.0;
        if (!right) {
            Gather gm;
            load(gm, m, true);
            const double r = fma(a.gb, gm.zn + gm.zp, fma(a.ga, gm.yn + gm.yp, gm.b));
            y = fma(a.gm, z + zr, r);
            if (ok) {
                const long long o = (long long)m * a.SI + own;
                out[o] = OMEGA1 ? y : fma(a.om1, uin[o], y);
            }
        }
        const double yo = __shfl_xor_sync(0xffffffffu, y, 16);
        if (right)
            y = yo;
        // back substitution outwards from the twist cell, DB cells of loads in flight; the
        // left thread's step s is cell m-1-s (pivot p_{m-1-s}), the right thread's is cell
        // m+1+s (pivot q_{m+1+s} = p_{nx-2-m-s})
        double zb[DB], ub[DB];
        auto loadb = [&](int h, int i, bool on) {
            const long long o = (long long)i * a.SI + own;
            zb[h] = (on && ok) ? zs[o] : 0.0;
            if (!OMEGA1)
                ub[h] = (on && ok) ? uin[o] : 0.0;
        };
        const int pb = right ? nx - 2 - m : m - 1;  // pivot index of back step 0
#pragma unroll
        for (int h = 0; h < DB; ++h)
            loadb(h, right ? m + 1 + h : m - 1 - h, h < cnt);
#pragma unroll 1
        for (int s = 0; s < Rc; s += DB) {
#pragma unroll
            for (int h = 0; h < DB; ++h) {
                const int ss = s + h;
                const int i = right ? m + 1 + ss : m - 1 - ss;
                if (ss < cnt) {
                    y = fma(a.fm[pb - ss], y, zb[h]);
                    if (ok)
                        out[(long long)i * a.SI + own] = OMEGA1 ? y : fma(a.om1, ub[h], y);
                }
                const int sn = ss + DB;
                loadb(h, right ? m + 1 + sn : m - 1 - sn, sn < cnt);
            }
        }
    }
}

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

using TwistKernel = void (*)(const double*, double*, double*, const double*, const SeqArgs);

// Prefetch depths (elimination, back substitution) selectable for measurement:
// BRSMOOTH_SEQ_DEPTH = 0: (2, 2), 1: (2, 4), 2: (2, 8), 3: (3, 8, spills at 64 registers).
// Same box, persistent CTAs, Gcell/s at 256^3 / 512^3: Jacobi 73.7 / 73.2, 75.8 / 75.4,
// 77.2 / 76.7; Gauss-Seidel (omega = 1) 61.7 / 78.9, 67.2 / 83.9, 71.6 / 86.0.  Default 2.
template <bool OM1>
TwistKernel twist_kernel(int depth)
{
    switch (depth) {
    case 0: return xline_twist_kernel<OM1, 2, 2>;
    case 1: return xline_twist_kernel<OM1, 2, 4>;
    case 3: return xline_twist_kernel<OM1, 3, 8>;
    default: return xline_twist_kernel<OM1, 2, 8>;
    }
}

int launch_twist(brs_ctx* c, bool om1, const double* uin, double* out, double* zs,
                 const SeqArgs& a, const Shape& sh, cudaStream_t s)
{
    SeqState* S = st(c);
    TwistKernel k = om1 ? twist_kernel<true>(S->depth) : twist_kernel<false>(S->depth);
    const double* bs = S->Bs;
    cudaError_t e;
    if (sh.pdl)
        e = launch_pdl(k, dim3(sh.grid), dim3(sh.warps * 32), 0, s, uin, out, zs, bs, a);
    else {
        k<<<sh.grid, sh.warps * 32, 0, s>>>(uin, out, zs, bs, a);
        e = cudaGetLastError();
    }
    return brs_cuda_status(e);
}

}  // namespace

// Pivots of the twisted elimination (see the file comment), FP64: pv_i = p_i left of the
// twist cell m = (n-1)/2, g_m at it, q_i = p_{n-1-i} right of it.
std::vector<double> seq_line_pivots(int n, double ax, double ay, double az)
{
    const double d = 2.0 * (ax + ay + az);
    const int m = (n - 1) / 2;
    std::vector<double> pv(n, 0.0);
    for (int i = 0; i < m; ++i)
        pv[i] = 1.0 / (d - (i ? ax * ax * pv[i - 1] : 0.0));
    for (int i = n - 1; i > m; --i)
        pv[i] = 1.0 / (d - (i < n - 1 ? ax * ax * pv[i + 1] : 0.0));
    const double pl = m >= 1 ? pv[m - 1] : 0.0;
    const double qr = m + 1 <= n - 1 ? pv[m + 1] : 0.0;
    pv[m] = 1.0 / (d - ax * ax * pl - ax * ax * qr);
    return pv;
}

namespace {

// Shape of a launch over `tasks` warp tasks.  Default: one warp per CTA, one CTA per task,
// placed by the block scheduler.  persist: one CTA per SM of up to 32 warps striding over
// the tasks (every SM receives the same share, also when the launch is dependent).
// A dependent launch places the next sweep's CTAs while this one runs; when the two grids
// do not fit on the GPU together, the early CTAs land wherever slots free up first and
// unbalance the next sweep (256^3 FP64 Jacobi, 4096 one-warp CTAs on 152 x 32 slots: 59.8
// Gcell/s with dependent launches, 68.8 without; one-colour launches of half the size:
// 64.1 with, 63.2 without, same box), so one-warp CTAs are dependent only when two grids fit.
int pick_shape(brs_ctx* c, long long tasks, bool persist, Shape* sh)
{
    SeqState* S = st(c);
    const void* k = (const void*)twist_kernel<false>(S->depth);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const bool pdl_env = env_int("BRSMOOTH_LINE_PDL", 1) != 0;
    if (persist && tasks >= sms) {
        int w = (int)std::min<long long>(32, (tasks + sms - 1) / sms);
        int occ = 0;
        while (w > 1) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, w * 32, 0);
            if (e != cudaSuccess)
                return brs_cuda_status(e);
            if (occ >= 1)
                break;
            --w;
        }
        sh->grid = sms;
        sh->warps = w;
        sh->pdl = pdl_env;
        return BRS_OK;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 32, 0);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    const long long big = 1ll << 30;
    sh->grid = (int)std::max<long long>(1, std::min(tasks, big));
    sh->warps = 1;
    sh->pdl = pdl_env && 2ll * sh->grid <= (long long)occ * sms;
    return BRS_OK;
}

}  // namespace

int line_seq_setup(brs_ctx* c)
{
    const brs_params& p = c->p;
    SeqState* S = new (std::nothrow) SeqState();
    if (!S)
        return BRS_ERR_NOMEM;
    c->lseq = S;
    S->H = (p.ny + 1) / 2;
    S->elems = (long long)p.nx * p.nz * 2 * S->H;
    S->depth = env_int("BRSMOOTH_SEQ_DEPTH", 2);
    const size_t bytes = (size_t)S->elems * sizeof(double);
    if (p.nx > 2 * kSeqMaxSteps)
        return BRS_ERR_UNSUPPORTED;
    S->pv = seq_line_pivots(p.nx, p.ax, p.ay, p.az);
    // per cell: b is scaled by omega pv_i on its way into the line-major layout
    std::vector<double> scale(p.nx);
    for (int i = 0; i < p.nx; ++i)
        scale[i] = c->omega * S->pv[i];
    cudaError_t e = cudaMalloc(&S->tab, scale.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpy(S->tab, scale.data(), scale.size() * sizeof(double),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&S->U0, bytes);
    if (e == cudaSuccess)
        e = cudaMalloc(&S->U1, bytes);
    if (e == cudaSuccess)
        e = cudaMalloc(&S->Bs, bytes);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    const long long tpb = (S->H + kLinesPerWarp - 1) / kLinesPerWarp;
    const long long tasks = (long long)p.nz * 2 * tpb;
    // one CTA per SM (same box, Gcell/s, one-warp CTAs vs persistent): 256^3 Jacobi 75.3 vs
    // 77.2, Gauss-Seidel 71.8 vs 71.6; 512^3 Jacobi 76.1 vs 76.7, Gauss-Seidel 85.7 vs 86.0
    const bool persist = env_int("BRSMOOTH_SEQ_PERSIST", 1) != 0;
    int rc = pick_shape(c, tasks, persist, &S->jac);
    if (rc == BRS_OK)
        rc = pick_shape(c, tasks / 2, persist, &S->gs);
    return rc;
    return BRS_OK;
}

void line_seq_teardown(brs_ctx* c)
{
    SeqState* S = st(c);
    if (!S)
        return;
    if (S->tab)
        cudaFree(S->tab);
    if (S->U0)
        cudaFree(S->U0);
    if (S->U1)
        cudaFree(S->U1);
    if (S->Bs)
        cudaFree(S->Bs);
    delete S;
    c->lseq = nullptr;
}

int line_seq_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s)
{
    if (nsweeps == 0)
        return BRS_OK;
    SeqState* S = st(c);
    const brs_params& p = c->p;
    const long long SI = (long long)p.nz * 2 * S->H;
    const int tiles = ((p.nx + kTile - 1) / kTile) * ((p.ny + kTile - 1) / kTile);
    const dim3 pgrid(tiles, p.nz < 65535 ? p.nz : 65535);
    to_line_major<<<pgrid, 256, 0, s>>>(static_cast<const double*>(u), S->U0, nullptr, p.nx,
                                        p.ny, p.nz, S->H, SI);
    to_line_major<<<pgrid, 256, 0, s>>>(static_cast<const double*>(b), S->Bs, S->tab, p.nx,
                                        p.ny, p.nz, S->H, SI);
    int rc = brs_cuda_status(cudaGetLastError());
    if (rc != BRS_OK)
        return rc;
    SeqArgs a{};
    a.nx = p.nx;
    a.ny = p.ny;
    a.nz = p.nz;
    a.H = S->H;
    a.m = (p.nx - 1) / 2;
    a.SI = SI;
    a.tpb = (S->H + kLinesPerWarp - 1) / kLinesPerWarp;
    a.om1 = 1.0 - c->omega;
    const bool om1 = a.om1 == 0.0;
    const double* pv = S->pv.data();
    const int Rc = p.nx - 1 - a.m;
    for (int q = 0; q < kSeqMaxSteps; ++q) {
        // step q on either side uses p_q (pv[q] for q < m; the right side's q_{nx-1-q})
        const double pq = q < Rc ? pv[p.nx - 1 - q] : 0.0;
        a.fa[q] = c->omega * pq * p.ay;
        a.fb[q] = c->omega * pq * p.az;
        a.fm[q] = p.ax * pq;
    }
    a.ga = c->omega * pv[a.m] * p.ay;
    a.gb = c->omega * pv[a.m] * p.az;
    a.gm = p.ax * pv[a.m];
    double* cur = S->U0;
    if (p.method == BRS_CHAOTIC_GS) {
        // red-black line order: colour 0 from the old colour-1 values, then colour 1 from the
        // new colour-0 values; in place, elimination values in U1
        a.ntasks = (long long)p.nz * a.tpb;
        for (int q = 0; q < nsweeps && rc == BRS_OK; ++q)
            for (int col = 0; col < 2 && rc == BRS_OK; ++col) {
                a.colour = col;
                rc = launch_twist(c, om1, cur, cur, S->U1, a, S->gs, s);
            }
    } else {
        a.colour = -1;
        a.ntasks = (long long)p.nz * 2 * a.tpb;
        double* nxt = S->U1;
        for (int q = 0; q < nsweeps && rc == BRS_OK; ++q) {
            rc = launch_twist(c, om1, cur, nxt, nxt, a, S->jac, s);
            double* t = cur;
            cur = nxt;
            nxt = t;
        }
    }
    if (rc != BRS_OK)
        return rc;
    from_line_major<<<pgrid, 256, 0, s>>>(cur, static_cast<double*>(u), p.nx, p.ny, p.nz,
                                          S->H, SI);
    return brs_cuda_status(cudaGetLastError());
}
