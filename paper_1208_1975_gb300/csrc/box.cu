// Box blocks: the grid is cut into bx*by*bz spatial blocks (Sec. 2; the block sizes of
// Sec. 3), every block is solved with the one precomputed inverse Ahat_b of the diagonal
// block (Sec. 4.3), applied as a dense product (Alg. 2 step 2).
//
// One sweep runs all blocks of a pass as one matrix product.  R holds one row per block:
// its n = bx*by*bz right-hand sides rhs = b + N u (the gather form of the update, with N the
// couplings that leave the block), local cells numbered x fastest.  Then D = R Ahat^T
// (Ahat is symmetric, so both operands are K-major rows), and the epilogue writes
//   u'[cell] = (1 - omega) u[cell] + omega D[block][l]
// back into the grid.  Block Jacobi reads u and writes the second vector; block
// Gauss-Seidel visits the blocks in two colours (bi+bj+bk even, then odd): blocks of one
// colour share no face, so each colour is one product that reads the other colour's
// newest values.
//
// Arithmetic: FP64 and FP32 on CUDA cores (a tiled SIMT product), or FP32 on the tensor
// cores (tcgen05.mma kind::tf32, single TF32 or split-TF32 hi*hi + hi*lo + lo*hi) through the
// persistent product kernel of plane_tc.cuh with its EPI_BOX epilogue.
//
// Parity classes (CUDA-core path).  With constant coefficients the block matrix, and so its
// inverse, is unchanged by the reflections x -> bx-1-x, y -> by-1-y, z -> bz-1-z of the box.
// In the basis of sums and differences of mirrored cells (G, one 2 x 2 butterfly per
// mirrored pair and axis) the inverse is block diagonal: one dense block per parity class
// (symmetric or antisymmetric along each axis), 8 classes of about n/8 cells.  So
//   Ahat r = G^T (W G Ahat G^T W) (G r),  W = diag(1/2 per mirrored pair along each axis)
// with the class blocks of P = W G Ahat G^T W precomputed in FP64: fold the rows of R (G),
// one dense product per class (about n^2/8 multiply-adds per block instead of n^2), and
// unfold (G^T) in the update.  The product is still the one precomputed inverse, applied
// exactly.
#include <cmath>
#include <cstdlib>
#include <vector>

#include "box.cuh"
#include "box_parity.h"
#include "plane_tc.cuh"
#include "tc_host.cuh"

namespace {

struct BoxState {
    int bx = 1, by = 1, bz = 1, n = 1;
    long long nbx = 1, nby = 1, nbz = 1, nblk = 1;
    int math = BRS_PLANE_SIMT;   // SIMT, TF32 or 3XTF32
    int split = 0;               // tensor path: 1 or 3
    int bn = 32;                 // tensor path: tile N
    int sms = 1;
    void* inv = nullptr;         // SIMT: Ahat in the context dtype, [n][n]
    void* inv_lo = nullptr;      // tensor path: inv = TF32 hi part, inv_lo = lo part
    void* R = nullptr;           // [nblk][n]: context dtype (SIMT) or TF32 hi (tensor)
    void* R_lo = nullptr;
    long long* rows = nullptr;   // packed block coordinates of each R row, in pass order
    long long cnt[2] = {0, 0};   // rows per pass (Jacobi: one pass of nblk)
    int* off = nullptr;          // local cell l -> lx + nx (ly + ny lz)
    CUtensorMap mR_hi, mR_lo, mA_hi, mA_lo;
    // parity classes (CUDA-core path): class sizes and offsets in the folded row, the class
    // blocks of P (class c at pc_off[c], nc x nc), the folded rows, and the butterfly passes
    int fold = 0;
    int cls_n[8] = {0}, cls_off[8] = {0};
    long long pc_off[8] = {0};
    void* Pc = nullptr;
    void* Rf = nullptr;
    void* ftab = nullptr; // [3][n] int2: the fold's passes (x, y, z), the last into class order
    void* utab = nullptr; // [3][n] int2: the unfold's passes (z, y, x), the first from class order
};

BoxState* bs(brs_ctx* c) { return static_cast<BoxState*>(c->box); }

// 16-byte vector of T (float4 / double2), and the 8-byte one for float.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// W consecutive values at p, in 16-byte vectors where W and the element size allow it
// (callers guarantee the matching alignment).
template <typename T, int W>
__device__ __forceinline__ void ld_vec(T (&v)[W], const T* p)
{
    using V = typename Vec16<T>::type;
    constexpr int PER = (int)(16 / sizeof(T));
    if constexpr (W % PER == 0) {
#pragma unroll
        for (int m = 0; m < W / PER; ++m)
            reinterpret_cast<V*>(v)[m] = __ldg(reinterpret_cast<const V*>(p) + m);
    } else if constexpr (sizeof(T) == 4 && W == 2) {
        *reinterpret_cast<float2*>(v) = __ldg(reinterpret_cast<const float2*>(p));
    } else {
#pragma unroll
        for (int m = 0; m < W; ++m)
            v[m] = p[m];
    }
}

template <typename T, int W>
__device__ __forceinline__ void st_vec(T* p, const T (&v)[W])
{
    using V = typename Vec16<T>::type;
    constexpr int PER = (int)(16 / sizeof(T));
    if constexpr (W % PER == 0) {
#pragma unroll
        for (int m = 0; m < W / PER; ++m)
            reinterpret_cast<V*>(p)[m] = reinterpret_cast<const V*>(v)[m];
    } else if constexpr (sizeof(T) == 4 && W == 2) {
        *reinterpret_cast<float2*>(p) = *reinterpret_cast<const float2*>(v);
    } else {
#pragma unroll
        for (int m = 0; m < W; ++m)
            p[m] = v[m];
    }
}

// One x-row r = ly + by lz of the block with packed coordinates pk into R row q.
template <typename T, int SPLIT, int BX>
__device__ __forceinline__ void box_gather_row(const T* __restrict__ u, const T* __restrict__ b,
                                               T* __restrict__ rhi, float* __restrict__ rlo,
                                               long long q, long long pk, int r, int n, int by,
                                               int bz, int nx, int ny, int nz, long long plane,
                                               T ax, T ay, T az)
{
    const int ly = r % by, lz = r / by;  // uniform per CTA
    const int i0 = (int)(pk & 0x1FFFFF) * BX;
    const int j = (int)((pk >> 21) & 0x1FFFFF) * by + ly;
    const int k = (int)(pk >> 42) * bz + lz;
    const long long cell = i0 + (long long)nx * j + plane * k;
    T v[BX], t[BX];
    ld_vec<T, BX>(v, b + cell);
    if (ly == 0 && j > 0) {
        ld_vec<T, BX>(t, u + cell - nx);
#pragma unroll
        for (int m = 0; m < BX; ++m)
            v[m] = fma(ay, t[m], v[m]);
    }
    if (ly == by - 1 && j + 1 < ny) {
        ld_vec<T, BX>(t, u + cell + nx);
#pragma unroll
        for (int m = 0; m < BX; ++m)
            v[m] = fma(ay, t[m], v[m]);
    }
    if (lz == 0 && k > 0) {
        ld_vec<T, BX>(t, u + cell - plane);
#pragma unroll
        for (int m = 0; m < BX; ++m)
            v[m] = fma(az, t[m], v[m]);
    }
    if (lz == bz - 1 && k + 1 < nz) {
        ld_vec<T, BX>(t, u + cell + plane);
#pragma unroll
        for (int m = 0; m < BX; ++m)
            v[m] = fma(az, t[m], v[m]);
    }
    if (i0 > 0)
        v[0] = fma(ax, u[cell - 1], v[0]);
    if (i0 + BX < nx)
        v[BX - 1] = fma(ax, u[cell + BX], v[BX - 1]);
    const long long o = q * n + (long long)BX * r;
    if constexpr (SPLIT == 0) {
        st_vec<T, BX>(rhi + o, v);
    } else {
        float h[BX], l[BX];
#pragma unroll
        for (int m = 0; m < BX; ++m) {
            const uint32_t hb = brs_tc::tf32_rn((float)v[m]);
            h[m] = __uint_as_float(hb);
            l[m] = __uint_as_float(brs_tc::tf32_rn((float)v[m] - h[m]));
        }
        st_vec<float, BX>(rhi + o, h);
        if (SPLIT == 3)
            st_vec<float, BX>(rlo + o, l);
    }
}


// rhs of RPT consecutive x-rows of a block: b + ax/ay/az times the neighbours that lie
// outside the block and inside the grid (zero Dirichlet values outside).  Thread = R row q
// (one block); the CTA's row group gives the first row's index r = ly + by lz inside the
// block, so adjacent threads read adjacent blocks' rows (one contiguous grid row per warp in the
// Jacobi order) and write R[q][BX r .. BX (r + RPT)), at least one 32-byte sector.  BX is
// the block's x size (a template for 1, 2, 4, 8).
// SPLIT 0: store in T; 1: TF32 hi only; 3: TF32 hi and lo.
template <typename T, int SPLIT, int BX, int RPT>
__global__ void __launch_bounds__(256) box_gather_kernel(
    const T* __restrict__ u, const T* __restrict__ b, T* __restrict__ rhi, float* __restrict__ rlo,
    const long long* __restrict__ rows, long long cnt, int n, int by, int bz, int nx, int ny,
    int nz, T ax, T ay, T az)
{
    // CTA order: the row groups of one set of 256 blocks are consecutive CTAs, so the grid
    // is read once, front to back
    pdl_wait_trigger();
    const int groups = by * bz / RPT;
    const unsigned qc = blockIdx.x / groups;
    const int r0 = (int)(blockIdx.x - qc * groups) * RPT;
    const long long q = (long long)qc * blockDim.x + threadIdx.x;
    if (q >= cnt)
        return;
    const long long pk = __ldg(rows + q);
    const long long plane = (long long)nx * ny;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr)
        box_gather_row<T, SPLIT, BX>(u, b, rhi, rlo, q, pk, r0 + rr, n, by, bz, nx, ny, nz, plane,
                                     ax, ay, az);
}

// The same for any bx (one cell per loop step, scalar accesses).
template <typename T, int SPLIT>
__global__ void __launch_bounds__(256) box_gather_any_kernel(
    const T* __restrict__ u, const T* __restrict__ b, T* __restrict__ rhi, float* __restrict__ rlo,
    const long long* __restrict__ rows, long long cnt, int n, int bx, int by, int bz, int nx,
    int ny, int nz, T ax, T ay, T az)
{
    pdl_wait_trigger();
    const int groups = by * bz;
    const unsigned qc = blockIdx.x / groups;
    const int r = (int)(blockIdx.x - qc * groups);
    const long long q = (long long)qc * blockDim.x + threadIdx.x;
    if (q >= cnt)
        return;
    const int ly = r % by, lz = r / by;
    const long long plane = (long long)nx * ny;
    const long long pk = __ldg(rows + q);
    const int i0 = (int)(pk & 0x1FFFFF) * bx;
    const int j = (int)((pk >> 21) & 0x1FFFFF) * by + ly;
    const int k = (int)(pk >> 42) * bz + lz;
    const long long cell0 = i0 + (long long)nx * j + plane * k;
    const long long o = q * n + (long long)bx * r;
    for (int lx = 0; lx < bx; ++lx) {
        const long long cell = cell0 + lx;
        T v = b[cell];
        if (ly == 0 && j > 0)
            v = fma(ay, u[cell - nx], v);
        if (ly == by - 1 && j + 1 < ny)
            v = fma(ay, u[cell + nx], v);
        if (lz == 0 && k > 0)
            v = fma(az, u[cell - plane], v);
        if (lz == bz - 1 && k + 1 < nz)
            v = fma(az, u[cell + plane], v);
        if (lx == 0 && i0 > 0)
            v = fma(ax, u[cell - 1], v);
        if (lx == bx - 1 && i0 + bx < nx)
            v = fma(ax, u[cell + 1], v);
        if constexpr (SPLIT == 0) {
            rhi[o + lx] = v;
        } else {
            const uint32_t hb = brs_tc::tf32_rn((float)v);
            rhi[o + lx] = __uint_as_float(hb);
            if (SPLIT == 3)
                rlo[o + lx] = __uint_as_float(brs_tc::tf32_rn((float)v - __uint_as_float(hb)));
        }
    }
}

template <typename T, int SPLIT>
cudaError_t launch_gather(const BoxState* B, const brs_params& p, const T* u, const T* b, T* rhi,
                          float* rlo, const long long* rows, long long M, cudaStream_t s)
{
    const dim3 grid((unsigned)(((M + 255) / 256) * (B->by * B->bz)));
    const T ax = (T)p.ax, ay = (T)p.ay, az = (T)p.az;
    // the vector paths need the row start aligned to the vector: bx | nx makes every row
    // start a multiple of bx
    // rows per thread: enough for 32 bytes of R per store, dividing the block's row count
    const int rows_in_block = B->by * B->bz;
    int want = (int)(32 / (B->bx * sizeof(T)));
    int rpt = 1;
    while (rpt * 2 <= want && rows_in_block % (rpt * 2) == 0)
        rpt *= 2;
#define BRS_BOX_GATHER(BXV, RPTV)                                                            \
    if (B->bx == BXV && rpt == RPTV) {                                                       \
        const dim3 g2((unsigned)(((M + 255) / 256) * (rows_in_block / RPTV)));              \
        return launch_pdl(box_gather_kernel<T, SPLIT, BXV, RPTV>, g2, dim3(256), 0, s, u, b,  \
                          rhi, rlo, rows, M, B->n, B->by, B->bz, p.nx, p.ny, p.nz, ax, ay,    \
                          az);                                                               \
    }
    BRS_BOX_GATHER(1, 1)
    BRS_BOX_GATHER(1, 2)
    BRS_BOX_GATHER(1, 4)
    BRS_BOX_GATHER(1, 8)
    BRS_BOX_GATHER(2, 1)
    BRS_BOX_GATHER(2, 2)
    BRS_BOX_GATHER(2, 4)
    BRS_BOX_GATHER(4, 1)
    BRS_BOX_GATHER(4, 2)
    BRS_BOX_GATHER(8, 1)
#undef BRS_BOX_GATHER
    return launch_pdl(box_gather_any_kernel<T, SPLIT>, grid, dim3(256), 0, s, u, b, rhi, rlo,
                      rows, M, B->n, B->bx, B->by, B->bz, p.nx, p.ny, p.nz, ax, ay, az);
}

// D = R Ahat^T on CUDA cores, fused with the update.  Tile 64 blocks x BN local cells,
// K in steps of 16; thread (tx, ty) owns rows ty + 16 i (i < 4) and columns tx + 16 j.
// Grid: x = row tiles, y = column tiles.
template <typename T, int BN>
__global__ void __launch_bounds__(256) box_gemm_simt(
    const T* __restrict__ R, const T* __restrict__ Ainv, const T* u, T* uout,
    const long long* __restrict__ rows, const int* __restrict__ off, long long M, int n, int bx,
    int by, int bz, int nx, int ny, double omega)
{
    pdl_wait_trigger();
    constexpr int BMS = 64, BKS = 16, TN = BN / 16;
    __shared__ T As[BKS][BMS + 1];
    __shared__ T Bs[BKS][BN + 1];
    const long long m0 = (long long)blockIdx.x * BMS;
    const int n0 = blockIdx.y * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
            acc[i][j] = T(0);
    for (int k0 = 0; k0 < n; k0 += BKS) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = threadIdx.x + r * 256;
            const int row = idx / BKS, kk = idx % BKS;
            const long long gm = m0 + row;
            const int gk = k0 + kk;
            As[kk][row] = (gm < M && gk < n) ? R[gm * n + gk] : T(0);
        }
#pragma unroll
        for (int r = 0; r < TN; ++r) {
            const int idx = threadIdx.x + r * 256;
            const int row = idx / BKS, kk = idx % BKS;
            const int gl = n0 + row, gk = k0 + kk;
            Bs[kk][row] = (gl < n && gk < n) ? Ainv[(long long)gl * n + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BKS; ++kk) {
            T a[4], bv[TN];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j)
                bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    const T om = (T)omega, om1 = (T)(1.0 - omega);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long m = m0 + ty + 16 * i;
        if (m >= M)
            continue;
        const long long pk = rows[m];
        const long long base = (pk & 0x1FFFFF) * bx +
                               (long long)nx * (((pk >> 21) & 0x1FFFFF) * by + (long long)ny * (pk >> 42) * bz);
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int l = n0 + tx + 16 * j;
            if (l < n) {
                const long long cell = base + off[l];
                uout[cell] = fma(om, acc[i][j], om1 * u[cell]);
            }
        }
    }
}

template <typename T, int BN>
cudaError_t launch_simt(const BoxState* B, const T* R, const T* inv, const T* u, T* uout,
                        const long long* rows, long long M, int nx, int ny, double omega,
                        cudaStream_t s)
{
    const long long tm = (M + 63) / 64;
    dim3 grid((unsigned)tm, (unsigned)((B->n + BN - 1) / BN));
    return launch_pdl(box_gemm_simt<T, BN>, grid, dim3(256), 0, s, R, inv, u, uout, rows,
                      (const int*)B->off, M, B->n, B->bx, B->by, B->bz, nx, ny, omega);
}

// ---------------------------------------------------------------- parity classes
// G and G^T are separable: one 2 x 2 butterfly per mirrored pair along each axis, so each is
// applied in three passes (x, y, z for G; z, y, x for G^T) with one addition per element and
// pass.  A pass is a table over its output positions o: out[o] = in[t.x] + sign in[|t.y| - 1]
// (t.y = 0: out[o] = in[t.x]).  The fold's last pass writes the class-major order, the unfold's
// first pass reads it.  A CTA stages kRowsPerCta rows and the three tables in shared memory.
constexpr int kRowsPerCta = 4;

template <typename T>
__device__ __forceinline__ T butterfly(const T* in, int2 t)
{
    const T a = in[t.x];
    return t.y == 0 ? a : t.y > 0 ? a + in[t.y - 1] : a - in[-t.y - 1];
}

// Rf[row] = G R[row] in class-major order
template <typename T>
__global__ void __launch_bounds__(256) box_fold_kernel(const T* __restrict__ R, T* __restrict__ Rf,
                                                       const int2* __restrict__ tabs, long long M,
                                                       int n)
{
    extern __shared__ __align__(16) unsigned char fold_smem[];
    int2* tab = reinterpret_cast<int2*>(fold_smem);  // [3][n]
    T* A = reinterpret_cast<T*>(fold_smem + (size_t)3 * n * sizeof(int2));
    T* Bf = A + (size_t)kRowsPerCta * n;
    pdl_wait_trigger();
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x)
        tab[i] = tabs[i];
    const long long chunks = (M + kRowsPerCta - 1) / kRowsPerCta;
    for (long long ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const long long r0 = ch * kRowsPerCta;
        const int nr = (int)(M - r0 < kRowsPerCta ? M - r0 : kRowsPerCta);
        __syncthreads();  // the previous chunk is consumed (and the tables are staged)
        for (int i = threadIdx.x; i < nr * n; i += blockDim.x)
            A[i] = R[r0 * n + i];
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr)
            for (int o = threadIdx.x; o < n; o += blockDim.x)
                Bf[rr * n + o] = butterfly(A + rr * n, tab[o]);
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr)
            for (int o = threadIdx.x; o < n; o += blockDim.x)
                A[rr * n + o] = butterfly(Bf + rr * n, tab[n + o]);
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr)
            for (int o = threadIdx.x; o < n; o += blockDim.x)
                Rf[(r0 + rr) * n + o] = butterfly(A + rr * n, tab[2 * n + o]);
    }
}

// Df[row][off + j] = sum_k Rf[row][off + k] Pc[j][k] for one parity class (nc x nc block);
// 64 rows x BN columns per tile.
template <typename T, int BN>
__global__ void __launch_bounds__(256) box_class_gemm(const T* __restrict__ Rf,
                                                      const T* __restrict__ Pc, T* Df, long long M,
                                                      int n, int off, int nc)
{
    pdl_wait_trigger();
    constexpr int BMS = 64, BKS = 16, TN = BN / 16;
    __shared__ T As[BKS][BMS + 1];
    __shared__ T Bs[BKS][BN + 1];
    const long long m0 = (long long)blockIdx.x * BMS;
    const int n0 = blockIdx.y * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
            acc[i][j] = T(0);
    for (int k0 = 0; k0 < nc; k0 += BKS) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = threadIdx.x + r * 256;
            const int row = idx / BKS, kk = idx % BKS;
            const long long gm = m0 + row;
            const int gk = k0 + kk;
            As[kk][row] = (gm < M && gk < nc) ? Rf[gm * n + off + gk] : T(0);
        }
#pragma unroll
        for (int r = 0; r < TN; ++r) {
            const int idx = threadIdx.x + r * 256;
            const int row = idx / BKS, kk = idx % BKS;
            const int gl = n0 + row, gk = k0 + kk;
            Bs[kk][row] = (gl < nc && gk < nc) ? Pc[(long long)gl * nc + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BKS; ++kk) {
            T a[4], bv[TN];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j)
                bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long m = m0 + ty + 16 * i;
        if (m >= M)
            continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int l = n0 + tx + 16 * j;
            if (l < nc)
                Df[m * n + off + l] = acc[i][j];
        }
    }
}

// uout[cell] = (1 - omega) u[cell] + omega D[l], D = G^T Df[row] (class-major in), for every
// cell l of every block row of the pass
template <typename T>
__global__ void __launch_bounds__(256) box_unfold_kernel(const T* __restrict__ Df,
                                                         const int2* __restrict__ tabs,
                                                         const T* u, T* uout,
                                                         const long long* __restrict__ rows,
                                                         const int* __restrict__ off, long long M,
                                                         int n, int bx, int by, int bz, int nx,
                                                         int ny, double omega)
{
    extern __shared__ __align__(16) unsigned char fold_smem[];
    int2* tab = reinterpret_cast<int2*>(fold_smem);
    T* A = reinterpret_cast<T*>(fold_smem + (size_t)3 * n * sizeof(int2));
    T* Bf = A + (size_t)kRowsPerCta * n;
    pdl_wait_trigger();
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x)
        tab[i] = tabs[i];
    const T om = (T)omega, om1 = (T)(1.0 - omega);
    const long long chunks = (M + kRowsPerCta - 1) / kRowsPerCta;
    for (long long ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const long long r0 = ch * kRowsPerCta;
        const int nr = (int)(M - r0 < kRowsPerCta ? M - r0 : kRowsPerCta);
        __syncthreads();
        for (int i = threadIdx.x; i < nr * n; i += blockDim.x)
            A[i] = Df[r0 * n + i];
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr)
            for (int o = threadIdx.x; o < n; o += blockDim.x)
                Bf[rr * n + o] = butterfly(A + rr * n, tab[o]);
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr)
            for (int o = threadIdx.x; o < n; o += blockDim.x)
                A[rr * n + o] = butterfly(Bf + rr * n, tab[n + o]);
        __syncthreads();
        for (int rr = 0; rr < nr; ++rr) {
            const long long pk = rows[r0 + rr];
            const long long base = (pk & 0x1FFFFF) * bx +
                                   (long long)nx * (((pk >> 21) & 0x1FFFFF) * by +
                                                    (long long)ny * (pk >> 42) * bz);
            for (int l = threadIdx.x; l < n; l += blockDim.x) {
                const T d = butterfly(A + rr * n, tab[2 * n + l]);
                const long long cell = base + __ldg(off + l);
                uout[cell] = fma(om, d, om1 * u[cell]);
            }
        }
    }
}

unsigned chunk_grid(long long M)
{
    const long long ch = (M + kRowsPerCta - 1) / kRowsPerCta;
    return (unsigned)(ch < 152 * 8 ? (ch > 0 ? ch : 1) : 152 * 8);
}

template <typename T>
size_t fold_smem(int n)
{
    return (size_t)3 * n * sizeof(int2) + (size_t)2 * kRowsPerCta * n * sizeof(T);
}

// gather, fold, one product per class, unfold with the update
template <typename T>
int box_pass_fold(brs_ctx* c, const T* uin, T* uout, const T* b, const long long* rows,
                  long long M, cudaStream_t s)
{
    BoxState* B = bs(c);
    const brs_params& p = c->p;
    T* R = static_cast<T*>(B->R);
    T* Rf = static_cast<T*>(B->Rf);
    cudaError_t e = launch_gather<T, 0>(B, p, uin, b, R, nullptr, rows, M, s);
    const int n = B->n;
    if (e == cudaSuccess)
        e = launch_pdl(box_fold_kernel<T>, dim3(chunk_grid(M)), dim3(256), fold_smem<T>(n), s,
                       (const T*)R, Rf, (const int2*)B->ftab, M, n);
    const T* Pc = static_cast<const T*>(B->Pc);
    for (int cl = 0; cl < 8 && e == cudaSuccess; ++cl) {
        const int nc = B->cls_n[cl];
        if (nc == 0)
            continue;
        const unsigned gx = (unsigned)((M + 63) / 64);
        // the products write D~ into R (consumed by the fold)
        if (nc <= 16)
            e = launch_pdl(box_class_gemm<T, 16>, dim3(gx, (nc + 15) / 16), dim3(256), 0, s,
                           (const T*)Rf, Pc + B->pc_off[cl], R, M, n, B->cls_off[cl], nc);
        else if (nc <= 32)
            e = launch_pdl(box_class_gemm<T, 32>, dim3(gx, (nc + 31) / 32), dim3(256), 0, s,
                           (const T*)Rf, Pc + B->pc_off[cl], R, M, n, B->cls_off[cl], nc);
        else
            e = launch_pdl(box_class_gemm<T, 64>, dim3(gx, (nc + 63) / 64), dim3(256), 0, s,
                           (const T*)Rf, Pc + B->pc_off[cl], R, M, n, B->cls_off[cl], nc);
    }
    if (e == cudaSuccess)
        e = launch_pdl(box_unfold_kernel<T>, dim3(chunk_grid(M)), dim3(256), fold_smem<T>(n), s,
                       (const T*)R, (const int2*)B->utab, uin, uout, rows, (const int*)B->off, M,
                       n, B->bx, B->by, B->bz, p.nx, p.ny, c->omega);
    return brs_cuda_status(e);
}

template <int SPLIT, int BN>
const void* tc_kernel()
{
    return (const void*)brs_tc::tc_gemm_persistent<SPLIT, brs_tc::EPI_BOX, BN,
                                                   brs_tc::pers_nst(SPLIT, BN)>;
}

const void* tc_kernel_for(int split, int bn)
{
    if (split == 3)
        return bn == 256 ? tc_kernel<3, 256>() : bn == 128 ? tc_kernel<3, 128>()
             : bn == 64  ? tc_kernel<3, 64>()  : tc_kernel<3, 32>();
    return bn == 256 ? tc_kernel<1, 256>() : bn == 128 ? tc_kernel<1, 128>()
         : bn == 64  ? tc_kernel<1, 64>()  : tc_kernel<1, 32>();
}

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return v ? std::atoi(v) : dflt;
}

// One pass: gather the rows of `rows[0..M)` from uin, then the product and update into uout.
template <typename T>
int box_pass(brs_ctx* c, const T* uin, T* uout, const T* b, const long long* rows, long long M,
             cudaStream_t s)
{
    BoxState* B = bs(c);
    const brs_params& p = c->p;
    if (M == 0)
        return BRS_OK;
    cudaError_t e = cudaSuccess;
    if (B->split == 0 && B->fold)
        return box_pass_fold<T>(c, uin, uout, b, rows, M, s);
    if (B->split == 0) {
        e = launch_gather<T, 0>(B, p, uin, b, static_cast<T*>(B->R), nullptr, rows, M, s);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        const T* R = static_cast<const T*>(B->R);
        const T* inv = static_cast<const T*>(B->inv);
        if (B->n <= 16)
            e = launch_simt<T, 16>(B, R, inv, uin, uout, rows, M, p.nx, p.ny, c->omega, s);
        else if (B->n <= 32)
            e = launch_simt<T, 32>(B, R, inv, uin, uout, rows, M, p.nx, p.ny, c->omega, s);
        else
            e = launch_simt<T, 64>(B, R, inv, uin, uout, rows, M, p.nx, p.ny, c->omega, s);
        return brs_cuda_status(e);
    }
    if constexpr (sizeof(T) == 4) {
        float* rhi = static_cast<float*>(B->R);
        float* rlo = static_cast<float*>(B->R_lo);
        if (B->split == 3)
            e = launch_gather<float, 3>(B, p, uin, b, rhi, rlo, rows, M, s);
        else
            e = launch_gather<float, 1>(B, p, uin, b, rhi, nullptr, rows, M, s);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        brs_tc::TcArgs g{};
        g.M = (int)M;
        g.N = B->n;
        g.K = B->n;
        g.u = uin;
        g.uout = uout;
        g.omega = (float)c->omega;
        g.status = c->dev_status;
        g.box_rows = rows;
        g.box_off = B->off;
        g.box_bx = B->bx;
        g.box_by = B->by;
        g.box_bz = B->bz;
        g.box_nx = p.nx;
        g.box_ny = p.ny;
        g.box_vec4 = (B->bx % 4 == 0 && p.nx % 4 == 0) ? 1 : 0;
        int tn = (B->n + B->bn - 1) / B->bn;
        int tm = (int)((M + brs_tc::BM - 1) / brs_tc::BM);
        int nb = 1;
        const long long ntiles = (long long)tn * tm;
        const int grid = (int)(ntiles < B->sms ? ntiles : B->sms);
        CUtensorMap a0 = B->mR_hi, a1 = B->mR_lo, b0 = B->mA_hi, b1 = B->mA_lo;
        void* args[] = {&a0, &a1, &b0, &b1, &g, &tn, &tm, &nb};
        e = launch_pdl_c(tc_kernel_for(B->split, B->bn), dim3(grid), dim3(192),
                         brs_tc::pers_smem(B->split, B->bn), s, args);
        return brs_cuda_status(e);
    }
    return BRS_ERR_UNSUPPORTED;
}

// Ahat = A_b^{-1} in FP64 from the block's own sine basis: A_b (zero values outside the
// block) is ax Tx + ay Ty + az Tz on the block, diagonal in the 3D DST-I of the block with
// eigenvalues ax s_p + ay s_q + az s_r, s_p = 2 - 2 cos((p+1) pi / (b+1)).
std::vector<double> block_inverse(int bx, int by, int bz, double ax, double ay, double az)
{
    auto basis = [](int m) {
        std::vector<double> S((size_t)m * m);
        const double sc = std::sqrt(2.0 / (m + 1));
        for (int p = 0; p < m; ++p)
            for (int i = 0; i < m; ++i)
                S[(size_t)p * m + i] = sc * std::sin(M_PI * (p + 1) * (i + 1) / (m + 1));
        return S;
    };
    auto eig = [](int m, int p) { return 2.0 - 2.0 * std::cos(M_PI * (p + 1) / (m + 1)); };
    const int n = bx * by * bz;
    const std::vector<double> Sx = basis(bx), Sy = basis(by), Sz = basis(bz);
    std::vector<double> Q((size_t)n * n), lam(n);
    for (int r = 0; r < bz; ++r)
        for (int q = 0; q < by; ++q)
            for (int p = 0; p < bx; ++p) {
                const int kk = p + bx * (q + by * r);
                lam[kk] = ax * eig(bx, p) + ay * eig(by, q) + az * eig(bz, r);
                for (int l = 0; l < n; ++l) {
                    const int lx = l % bx, ly = (l / bx) % by, lz = l / (bx * by);
                    Q[(size_t)l * n + kk] = Sx[(size_t)p * bx + lx] * Sy[(size_t)q * by + ly] *
                                            Sz[(size_t)r * bz + lz];
                }
            }
    std::vector<double> inv((size_t)n * n, 0.0);
    for (int l = 0; l < n; ++l)
        for (int m = 0; m <= l; ++m) {
            double s = 0.0;
            for (int kk = 0; kk < n; ++kk)
                s += Q[(size_t)l * n + kk] * Q[(size_t)m * n + kk] / lam[kk];
            inv[(size_t)l * n + m] = s;
            inv[(size_t)m * n + l] = s;
        }
    return inv;
}

template <typename T>
int upload(void** dst, const std::vector<T>& v)
{
    cudaError_t e = cudaMalloc(dst, v.size() * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return brs_cuda_status(e);
}

}  // namespace

// Parity classes of the box (box_parity.h builds the tables on the host in FP64).
template <typename T>
int parity_setup(BoxState* B, const std::vector<double>& inv)
{
    const ParityTables pt = parity_tables(B->bx, B->by, B->bz, inv);
    if (!pt.use)
        return BRS_OK;
    for (int cl = 0; cl < 8; ++cl) {
        B->cls_n[cl] = pt.cls_n[cl];
        B->cls_off[cl] = pt.cls_off[cl];
        B->pc_off[cl] = pt.pc_off[cl];
    }
    const std::vector<T> pc(pt.pc.begin(), pt.pc.end());
    const std::vector<int>& ftab = pt.ftab;  // [3][n] (x, y) pairs: the layout of int2
    const std::vector<int>& utab = pt.utab;
    int rc = upload(&B->Pc, pc);
    if (rc == BRS_OK)
        rc = upload(&B->ftab, ftab);
    if (rc == BRS_OK)
        rc = upload(&B->utab, utab);
    if (rc == BRS_OK)
        rc = brs_cuda_status(cudaMalloc(&B->Rf, (size_t)B->nblk * B->n * sizeof(T)));
    if (rc == BRS_OK)
        B->fold = 1;
    return rc;
}

int box_setup(brs_ctx* c)
{
    const brs_params& p = c->p;
    if (p.bx < 1 || p.by < 1 || p.bz < 1)
        return BRS_ERR_ARG;
    if (p.nx % p.bx || p.ny % p.by || p.nz % p.bz)
        return BRS_ERR_ARG;
    const int n = p.bx * p.by * p.bz;
    if (n > 512 || p.bx > 512 || p.by > 512 || p.bz > 512)
        return BRS_ERR_UNSUPPORTED;
    BoxState* B = new (std::nothrow) BoxState();
    if (!B)
        return BRS_ERR_NOMEM;
    c->box = B;
    B->bx = p.bx;
    B->by = p.by;
    B->bz = p.bz;
    B->n = n;
    B->nbx = p.nx / p.bx;
    B->nby = p.ny / p.by;
    B->nbz = p.nz / p.bz;
    B->nblk = B->nbx * B->nby * B->nbz;
    if (B->nbx >= (1 << 21) || B->nby >= (1 << 21) || B->nbz >= (1 << 21) ||
        (long long)p.nx * p.ny * p.bz >= (1ll << 31) ||
        (B->nblk + 255) / 256 * (long long)(p.by * p.bz) >= (1ll << 31))
        return BRS_ERR_UNSUPPORTED;  // packed block coordinates, int offsets, gather grid
    // arithmetic
    int math = p.plane_math;
    if (p.dtype == BRS_F64) {
        if (math == BRS_PLANE_TF32 || math == BRS_PLANE_3XTF32)
            return BRS_ERR_UNSUPPORTED;
        math = BRS_PLANE_SIMT;
    } else if (math == BRS_PLANE_AUTO) {
        math = (n % 4 == 0 && n >= 32) ? BRS_PLANE_3XTF32 : BRS_PLANE_SIMT;
    } else if ((math == BRS_PLANE_TF32 || math == BRS_PLANE_3XTF32) && (n % 4 != 0 || n < 32)) {
        // K-major rows of n FP32 must be 16-byte multiples and span one 32-value TMA box
        return BRS_ERR_UNSUPPORTED;
    }
    B->math = math;
    B->split = math == BRS_PLANE_3XTF32 ? 3 : math == BRS_PLANE_TF32 ? 1 : 0;
    B->bn = n >= 128 ? 128 : n >= 64 ? 64 : 32;
    if (n >= 256 && env_int("BRSMOOTH_BOX_BN", 0) == 256)
        B->bn = 256;
    cudaError_t e = cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    // the inverse, once (Sec. 4.3)
    const std::vector<double> inv = block_inverse(p.bx, p.by, p.bz, p.ax, p.ay, p.az);
    int rc = BRS_OK;
    if (B->split) {
        rc = brs_tc::upload_split(&B->inv, &B->inv_lo, inv);
    } else if (p.dtype == BRS_F64) {
        rc = upload(&B->inv, inv);
    } else {
        rc = upload(&B->inv, std::vector<float>(inv.begin(), inv.end()));
    }
    if (rc != BRS_OK)
        return rc;
    // row tables: lexicographic for Jacobi, colour 0 then colour 1 for Gauss-Seidel
    std::vector<long long> rows;
    rows.reserve((size_t)B->nblk);
    auto pack = [](long long i, long long j, long long k) { return i | (j << 21) | (k << 42); };
    if (p.method == BRS_JACOBI) {
        for (long long k = 0; k < B->nbz; ++k)
            for (long long j = 0; j < B->nby; ++j)
                for (long long i = 0; i < B->nbx; ++i)
                    rows.push_back(pack(i, j, k));
        B->cnt[0] = B->nblk;
    } else {
        for (int colour = 0; colour < 2; ++colour) {
            for (long long k = 0; k < B->nbz; ++k)
                for (long long j = 0; j < B->nby; ++j)
                    for (long long i = 0; i < B->nbx; ++i)
                        if (((i + j + k) & 1) == colour)
                            rows.push_back(pack(i, j, k));
            B->cnt[colour] = (long long)rows.size() - (colour ? B->cnt[0] : 0);
        }
    }
    rc = upload(reinterpret_cast<void**>(&B->rows), rows);
    std::vector<int> off(n);
    for (int l = 0; l < n; ++l) {
        const int lx = l % p.bx, ly = (l / p.bx) % p.by, lz = l / (p.bx * p.by);
        off[l] = lx + p.nx * (ly + p.ny * lz);
    }
    if (rc == BRS_OK)
        rc = upload(reinterpret_cast<void**>(&B->off), off);
    if (rc != BRS_OK)
        return rc;
    // CUDA-core path: the product by parity classes (BRSMOOTH_BOX_FOLD=0: the full product)
    if (B->split == 0 && env_int("BRSMOOTH_BOX_FOLD", 1) != 0) {
        rc = p.dtype == BRS_F64 ? parity_setup<double>(B, inv) : parity_setup<float>(B, inv);
        if (rc != BRS_OK)
            return rc;
    }
    // R buffers (rows of the largest pass)
    const size_t relem = (size_t)B->nblk * n;
    e = cudaMalloc(&B->R, relem * (B->split ? 4 : c->esize));
    if (e == cudaSuccess && B->split == 3)
        e = cudaMalloc(&B->R_lo, relem * 4);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    if (B->split) {
        const int nrows = (int)B->nblk;
        if (B->nblk >= (1ll << 31))
            return BRS_ERR_UNSUPPORTED;
        rc = brs_tc::encode_map(&B->mR_hi, B->R, n, nrows, 0, brs_tc::BM);
        if (rc == BRS_OK)
            rc = brs_tc::encode_map(&B->mR_lo, B->split == 3 ? B->R_lo : B->R, n, nrows, 0, brs_tc::BM);
        if (rc == BRS_OK)
            rc = brs_tc::encode_map(&B->mA_hi, B->inv, n, n, 0, B->bn);
        if (rc == BRS_OK)
            rc = brs_tc::encode_map(&B->mA_lo, B->split == 3 ? B->inv_lo : B->inv, n, n, 0, B->bn);
        if (rc != BRS_OK)
            return rc;
        const void* k = tc_kernel_for(B->split, B->bn);
        const size_t smem = brs_tc::pers_smem(B->split, B->bn);
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, k);
        if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < smem)
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
    }
    return BRS_OK;
}

void box_teardown(brs_ctx* c)
{
    BoxState* B = bs(c);
    if (!B)
        return;
    void* bufs[] = {B->inv, B->inv_lo, B->R, B->R_lo, B->rows, B->off, B->Pc, B->Rf, B->ftab,
                    B->utab};
    for (void* q : bufs)
        if (q)
            cudaFree(q);
    delete B;
    c->box = nullptr;
}

int box_sweep_launch(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s)
{
    BoxState* B = bs(c);
    if (c->p.method == BRS_JACOBI) {
        if (c->p.dtype == BRS_F64)
            return box_pass<double>(c, static_cast<const double*>(uin), static_cast<double*>(uout),
                                    static_cast<const double*>(b), B->rows, B->cnt[0], s);
        return box_pass<float>(c, static_cast<const float*>(uin), static_cast<float*>(uout),
                               static_cast<const float*>(b), B->rows, B->cnt[0], s);
    }
    // two colours, in place
    int rc = BRS_OK;
    for (int colour = 0; colour < 2 && rc == BRS_OK; ++colour) {
        const long long* rows = B->rows + (colour ? B->cnt[0] : 0);
        if (c->p.dtype == BRS_F64)
            rc = box_pass<double>(c, static_cast<const double*>(uout), static_cast<double*>(uout),
                                  static_cast<const double*>(b), rows, B->cnt[colour], s);
        else
            rc = box_pass<float>(c, static_cast<const float*>(uout), static_cast<float*>(uout),
                                 static_cast<const float*>(b), rows, B->cnt[colour], s);
    }
    return rc;
}
