// FP64 xy-plane sweeps in the x-sine basis with the twisted elimination (Sec. 2 with one
// block per xy-plane; the basis change is described in plane_modes.cu).
//
// In the x-sine basis a plane sweep is, for every x-mode p on its own, a sweep of y-lines
// with the block M_p = tridiag(-ay, d_p, -ay), d_p = ax s_p + 2 ay + 2 az, and the z coupling
// az (u^_{k-1} + u^_{k+1}).  FP64 is bound by the FP64 pipe (2 FMAs per clock per SM), so this
// form solves each line the way the FP64 x-line sweep does: two threads per line, one
// eliminating from each end, meeting at the twist cell m = (ny-1)/2, then back-substituting
// outwards, with the pivots of M_p factored once per mode (twist_pivots).  In scaled
// variables (pv_y the pivot of cell y of mode p)
//   z_y = b'_y + fb_s (u^_{k-1,y} + u^_{k+1,y}) + fm_s z_{y-1}     (left; right mirrored)
//   y_m = b'_m + gb (u^_{k-1,m} + u^_{k+1,m}) + gm (z_{m-1} + z_{m+1})
//   y_y = z_y + fm y_{y+1}  (left),  v = (1 - omega) u^ + y
// with b'_y = omega pv_y b^_y formed by the forward transform's epilogue, fb_s = omega p_s az,
// fm_s = ay p_s (step s of either side uses p_s: the pivots are symmetric).  5 FP64
// operations per cell.  The arrays are [k][y][p] (p fastest): a warp takes 16 consecutive
// modes of one plane, lanes 0-15 the left halves and 16-31 the right halves of their lines,
// so every load and store of a step is a 128-byte run, and so are the per-mode tables
// fm[s][p], fb[s][p] (L2-resident).  The elimination writes z to the output array (Jacobi) or
// a scratch array (Gauss-Seidel, in place) and the back substitution reads it back.
// Gauss-Seidel: one launch per colour (planes k % 2 == colour), the other colour's planes
// read as they are: even planes, then odd planes.
#include "plane.cuh"

namespace {

struct TwistModeArgs {
    int nx, ny, nz;      // modes (p), line length (y), planes
    int m;               // twist cell
    int npb;             // 16-mode blocks per plane
    int colour;          // -1: every plane (Jacobi); 0 / 1: planes with k % 2 == colour
    long long ntasks;    // warp tasks
    double om1;          // 1 - omega
};

template <bool OMEGA1, int DF, int DB>
__global__ void __launch_bounds__(256, 4) mode_twist_kernel(
    const double* uin, double* out, double* zs, const double* __restrict__ bs,
    const double* __restrict__ fm, const double* __restrict__ fb,
    const double* __restrict__ gm, const double* __restrict__ gb, const TwistModeArgs a)
{
    pdl_wait_trigger();
    const long long task = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (task >= a.ntasks)
        return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const bool right = lane >= 16;
    const int n = a.ny, m = a.m, nx = a.nx;
    const int Rc = n - 1 - m;            // steps of the right side (>= the left side's m)
    const int cnt = right ? Rc : m;
    const int pb = (int)(task % a.npb);
    const long long kk = task / a.npb;
    const int k = a.colour < 0 ? (int)kk : (int)(2 * kk + a.colour);
    const int p = pb * 16 + (lane & 15);
    const bool ok = p < nx;
    const long long plane = (long long)n * nx;
    const long long base = (long long)k * plane + p;  // cell (k, y, p) at base + y nx
    const bool fzn = ok && k >= 1, fzp = ok && k + 1 < a.nz;

    struct Step {
        double b, zn, zp, f, g;
    };
    auto load = [&](Step& v, int ss, bool on) {
        const int y = right ? n - 1 - ss : ss;
        const long long o = base + (long long)y * nx;
        const bool q = on && ok;
        v.b = q ? __ldg(bs + o) : 0.0;
        v.zn = (on && fzn) ? __ldg(uin + o - plane) : 0.0;
        v.zp = (on && fzp) ? __ldg(uin + o + plane) : 0.0;
        v.f = q ? __ldg(fm + (long long)ss * nx + p) : 0.0;
        v.g = q ? __ldg(fb + (long long)ss * nx + p) : 0.0;
    };
    // elimination towards the twist cell, DF cells of loads in flight
    double z = 0.0;
    Step st[DF];
#pragma unroll
    for (int h = 0; h < DF; ++h)
        load(st[h], h, h < cnt);
#pragma unroll 1
    for (int s = 0; s < Rc; s += DF) {
#pragma unroll
        for (int h = 0; h < DF; ++h) {
            const int ss = s + h;
            if (ss < cnt) {
                const double r = fma(st[h].g, st[h].zn + st[h].zp, st[h].b);
                z = fma(st[h].f, z, r);
                if (ok)
                    zs[base + (long long)(right ? n - 1 - ss : ss) * nx] = z;
            }
            load(st[h], ss + DF, ss + DF < cnt);
        }
    }
    // twist cell: the left thread combines both eliminations
    const double zr = __shfl_xor_sync(0xffffffffu, z, 16);
    double y = 0.0;
    if (!right) {
        const long long o = base + (long long)m * nx;
        const double bm = ok ? __ldg(bs + o) : 0.0;
        const double zn = fzn ? __ldg(uin + o - plane) : 0.0;
        const double zp = fzp ? __ldg(uin + o + plane) : 0.0;
        const double gmv = ok ? __ldg(gm + p) : 0.0, gbv = ok ? __ldg(gb + p) : 0.0;
        y = fma(gmv, z + zr, fma(gbv, zn + zp, bm));
        if (ok)
            out[o] = OMEGA1 ? y : fma(a.om1, uin[o], y);
    }
    const double yo = __shfl_xor_sync(0xffffffffu, y, 16);
    if (right)
        y = yo;
    // back substitution outwards from the twist cell; the left thread's step s is cell
    // m-1-s (pivot p_{m-1-s}), the right thread's cell m+1+s (pivot p_{n-2-m-s})
    const int p0 = right ? n - 2 - m : m - 1;
    double zb[DB], ub[DB], fbk[DB];
    auto loadb = [&](int h, int ss, bool on) {
        const long long o = base + (long long)(right ? m + 1 + ss : m - 1 - ss) * nx;
        const bool q = on && ok;
        zb[h] = q ? zs[o] : 0.0;
        if (!OMEGA1)
            ub[h] = q ? uin[o] : 0.0;
        fbk[h] = q ? __ldg(fm + (long long)(p0 - ss) * nx + p) : 0.0;
    };
#pragma unroll
    for (int h = 0; h < DB; ++h)
        loadb(h, h, h < cnt);
#pragma unroll 1
    for (int s = 0; s < Rc; s += DB) {
#pragma unroll
        for (int h = 0; h < DB; ++h) {
            const int ss = s + h;
            if (ss < cnt) {
                y = fma(fbk[h], y, zb[h]);
                if (ok)
                    out[base + (long long)(right ? m + 1 + ss : m - 1 - ss) * nx] =
                        OMEGA1 ? y : fma(a.om1, ub[h], y);
            }
            loadb(h, ss + DB, ss + DB < cnt);
        }
    }
}

// ---------------------------------------------------------------------------------------
// x-DST along rows with the sine basis's even/odd symmetry.  For the orthonormal DST-I of
// length n, S[p][n-1-x] = (-1)^p S[p][x], so with h = floor(n/2), Ks = ceil(n/2), Kd = h,
//   forward  u^_p = sum_{x<h} S[p][x] (u_x + (-1)^p u_{n-1-x})  (+ S[p][h] u_h, p even, n odd)
//   inverse  u_x = E_x + O_x,  u_{n-1-x} = E_x - O_x,  E_x = sum_q S[x][2q] u^_{2q},
//            O_x = sum_q S[x][2q+1] u^_{2q+1}  (u_h = E_h for odd n)
// so each transform is two dense products of half the size (Ks x Ks and Kd x Kd): half the
// FP64 multiply-adds of the plain product, plus one elementwise pass before (fold,
// de-interleave) and, for the inverse, one after (combine).

// dst[row][0..Ks) = u_x + u_{n-1-x} (x < h; u_h last for odd n), dst[row][Ks..n) = u_x - u_{n-1-x}
__global__ void __launch_bounds__(256) fold_rows_kernel(const double* __restrict__ src,
                                                        double* __restrict__ dst, int n,
                                                        long long rows)
{
    pdl_wait_trigger();
    const int h = n / 2, Ks = n - h;
    const long long total = rows * (long long)Ks;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / Ks;
        const int x = (int)(t - r * Ks);
        const double* a = src + r * n;
        double* d = dst + r * n;
        if (x < h) {
            const double lo = a[x], hi = a[n - 1 - x];
            d[x] = lo + hi;
            d[Ks + x] = lo - hi;
        } else {
            d[x] = a[x];  // the middle element of an odd length
        }
    }
}

// dst[row][q] = src[row][2q] (q < Ks), dst[row][Ks + q] = src[row][2q+1] (q < Kd)
__global__ void __launch_bounds__(256) deinterleave_rows_kernel(const double* __restrict__ src,
                                                                double* __restrict__ dst, int n,
                                                                long long rows)
{
    pdl_wait_trigger();
    const int Ks = n - n / 2;
    const long long total = rows * (long long)n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / n;
        const int p = (int)(t - r * n);
        dst[r * n + (p & 1 ? Ks + (p >> 1) : (p >> 1))] = src[t];
    }
}

// src[row] = [E_0..E_{Ks-1} | O_0..O_{Kd-1}] -> dst[row][x] = E_x + O_x, dst[row][n-1-x] = E_x - O_x
__global__ void __launch_bounds__(256) combine_rows_kernel(const double* __restrict__ src,
                                                           double* __restrict__ dst, int n,
                                                           long long rows)
{
    pdl_wait_trigger();
    const int h = n / 2, Ks = n - h;
    const long long total = rows * (long long)Ks;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / Ks;
        const int x = (int)(t - r * Ks);
        const double* a = src + r * n;
        double* d = dst + r * n;
        if (x < h) {
            const double e = a[x], o = a[Ks + x];
            d[x] = e + o;
            d[n - 1 - x] = e - o;
        } else {
            d[x] = a[x];
        }
    }
}

// C[m][n] at C + b sC + m ldc + n ccs = sum_k A[b sA + m lda + k] B[n ldb + k] (times scale at
// C's offset when scale is set); 64 x 64 tiles, 4 x 4 outputs per thread.
struct StridedGemm {
    int M, N, K;
    long long lda, ldb, ldc, ccs, sA, sC;
    const double* scale;
};

constexpr int kTM = 64, kTN = 64, kTK = 16;

__global__ void __launch_bounds__(256) gemm_strided_kernel(const double* __restrict__ A,
                                                           const double* __restrict__ B,
                                                           double* C, StridedGemm g)
{
    pdl_wait_trigger();
    __shared__ double As[kTK][kTM + 1];
    __shared__ double Bs[kTK][kTN + 1];
    const double* Ab = A + (long long)blockIdx.z * g.sA;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            acc[i][j] = 0.0;
    for (int k0 = 0; k0 < g.K; k0 += kTK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = threadIdx.x + r * 256;
            const int row = idx / kTK, kk = idx % kTK;
            const int gm = m0 + row, gn = n0 + row, gk = k0 + kk;
            As[kk][row] = (gm < g.M && gk < g.K) ? Ab[(long long)gm * g.lda + gk] : 0.0;
            Bs[kk][row] = (gn < g.N && gk < g.K) ? B[(long long)gn * g.ldb + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            double a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty + 16 * i];
                bv[i] = Bs[kk][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* Cb = C + (long long)blockIdx.z * g.sC;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m < g.M && n < g.N) {
                const long long o = (long long)m * g.ldc + (long long)n * g.ccs;
                Cb[o] = g.scale ? acc[i][j] * g.scale[o] : acc[i][j];
            }
        }
}

cudaError_t launch_strided(const double* A, const double* B, double* C, const StridedGemm& g,
                           int batch, cudaStream_t s)
{
    if (g.M == 0 || g.N == 0 || batch == 0)
        return cudaSuccess;
    dim3 grid((g.N + kTN - 1) / kTN, (g.M + kTM - 1) / kTM, batch);
    return launch_pdl(gemm_strided_kernel, grid, dim3(256), 0, s, A, B, C, g);
}

unsigned row_grid(long long work)
{
    long long b = (work + 255) / 256;
    return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

int dst_fold_forward(const double* u, double* out, const double* scale, double* work,
                     const double* Se, const double* So, int nx, int ny, int nz, cudaStream_t s)
{
    const int h = nx / 2, Ks = nx - h, Kd = h;
    const long long rows = (long long)ny * nz, plane = (long long)nx * ny;
    cudaError_t e = launch_pdl(fold_rows_kernel, dim3(row_grid(rows * Ks)), dim3(256), 0, s, u,
                               work, nx, rows);
    StridedGemm g{};
    g.M = ny; g.lda = nx; g.ldc = nx; g.ccs = 2; g.sA = plane; g.sC = plane;
    // even modes p = 2q: the folded sums against Se[q][x'] = S[2q][x'] (x' < Ks)
    g.N = Ks; g.K = Ks; g.ldb = Ks; g.scale = scale;
    if (e == cudaSuccess)
        e = launch_strided(work, Se, out, g, nz, s);
    // odd modes p = 2q+1: the folded differences against So[q][x'] = S[2q+1][x'] (x' < Kd)
    g.N = Kd; g.K = Kd; g.ldb = Kd; g.scale = scale ? scale + 1 : nullptr;
    if (e == cudaSuccess && Kd > 0)
        e = launch_strided(work + Ks, So, out + 1, g, nz, s);
    return brs_cuda_status(e);
}

int dst_fold_inverse(const double* uh, double* out, double* work1, double* work2,
                     const double* SeT, const double* SoT, int nx, int ny, int nz, cudaStream_t s)
{
    const int h = nx / 2, Ks = nx - h, Kd = h;
    const long long rows = (long long)ny * nz, plane = (long long)nx * ny;
    cudaError_t e = launch_pdl(deinterleave_rows_kernel, dim3(row_grid(rows * nx)), dim3(256), 0,
                               s, uh, work1, nx, rows);
    StridedGemm g{};
    g.M = ny; g.lda = nx; g.ldc = nx; g.ccs = 1; g.sA = plane; g.sC = plane; g.scale = nullptr;
    // E_x = sum_q S[x][2q] u^_{2q}: B[x][q] = SeT[x][q] (x < Ks)
    g.N = Ks; g.K = Ks; g.ldb = Ks;
    if (e == cudaSuccess)
        e = launch_strided(work1, SeT, work2, g, nz, s);
    // O_x = sum_q S[x][2q+1] u^_{2q+1}: B[x][q] = SoT[x][q] (x < Kd)
    g.N = Kd; g.K = Kd; g.ldb = Kd;
    if (e == cudaSuccess && Kd > 0)
        e = launch_strided(work1 + Ks, SoT, work2 + Ks, g, nz, s);
    if (e == cudaSuccess)
        e = launch_pdl(combine_rows_kernel, dim3(row_grid(rows * Ks)), dim3(256), 0, s,
                       (const double*)work2, out, nx, rows);
    return brs_cuda_status(e);
}

int mode_twist_launch(const double* uin, double* out, double* zs, const double* bs,
                      const double* fm, const double* fb, const double* gm, const double* gb,
                      int nx, int ny, int nz, double omega, int colour, cudaStream_t s)
{
    TwistModeArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.m = (ny - 1) / 2;
    a.npb = (nx + 15) / 16;
    a.colour = colour;
    const long long planes = colour < 0 ? nz : (nz - colour + 1) / 2;
    a.ntasks = planes * a.npb;
    a.om1 = 1.0 - omega;
    if (a.ntasks == 0)
        return BRS_OK;
    const unsigned grid = (unsigned)((a.ntasks + 7) / 8);
    cudaError_t e =
        a.om1 == 0.0
            ? launch_pdl(mode_twist_kernel<true, 2, 4>, dim3(grid), dim3(256), 0, s, uin, out, zs,
                         bs, fm, fb, gm, gb, a)
            : launch_pdl(mode_twist_kernel<false, 2, 4>, dim3(grid), dim3(256), 0, s, uin, out,
                         zs, bs, fm, fb, gm, gb, a);
    return brs_cuda_status(e);
}
