// xy-plane block sweeps (Sec. 2 with one block per xy-plane).
//
// For plane k the sweep gathers the off-block (z) neighbours into the block right-hand
// side and solves the plane block exactly:
//   R_k = b_k + az (u_{k-1} + u_{k+1})
//   M_plane X = R_k,  M_plane(X) = ax X Tx + ay Ty X + 2 az X   (X indexed [y][x])
//   new u_k = (1-omega) u_k + omega X
// M_plane is diagonal in the orthonormal DST-I basis S (S = S^T = S^{-1},
// S T S = diag(s), s_p = 2 - 2 cos(p pi/(n+1))), so
//   X = S_y [ (S_y R S_x) ./ L ] S_x,   L[q][p] = ax s_p + ay s_q + 2 az.
// The basis and 1/L are built once per context on the host in FP64 (the constant block
// is factored once and reused, Sec. 4.3).
//
// The four contractions run as batched "TN" products C = A B^T (both operands K-major,
// one plane per batch index) chosen so that each pass's output is the next pass's
// K-major operand:
//   P1  C1[p][y] = sum_x Sx[p][x] R[y][x]
//   P2  Q[p][q]  = (sum_y C1[p][y] Sy[q][y]) / L[q][p]
//   P3  W[y][p]  = sum_q Sy[y][q] Q[p][q]
//   P4  X[y][x]  = sum_p W[y][p] Sx[x][p]      -> fused Jacobi / GS update of plane k
// Block Jacobi reads only old planes and writes the second vector.  Chaotic block GS
// updates in place, even planes first and odd planes second, so odd planes read their
// neighbours' new values (one admissible outcome of the unordered update of Alg. 1).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "line_impl.cuh"
#include "plane.cuh"
#include "plane_tc.cuh"
#include "tc_host.cuh"
#include "thomas_tables.h"

namespace {

struct PlaneState {
    int nx = 0, ny = 0;
    int math = BRS_PLANE_SIMT;
    void* sx = nullptr;    // [nx][nx] DST-I (context dtype; tensor path: TF32 hi part)
    void* sy = nullptr;    // [ny][ny]
    void* ilam = nullptr;  // [nx][ny]: 1 / (ax s_p + ay s_q + 2 az) at [p][q]
    void* t1 = nullptr;    // grid-sized intermediates (tensor path: hi parts)
    void* t2 = nullptr;
    // tensor path: TF32 lo parts and the TMA maps of the four products
    void* sx_lo = nullptr;
    void* sy_lo = nullptr;
    void* t1_lo = nullptr;
    void* t2_lo = nullptr;
    CUtensorMap m_sx_hi, m_sx_lo, m_sy_hi, m_sy_lo;  // 2D, box (32, 128)
    CUtensorMap m_R_hi, m_R_lo;    // t2 as [k][y][x]  (B of P1, box rows BN)
    CUtensorMap m_C1_hi, m_C1_lo;  // t1 as [k][p][y]  (A of P2, box rows 128)
    CUtensorMap m_Q_hi, m_Q_lo;    // t2 as [k][p][q]  (B of P3, box rows BN)
    CUtensorMap m_W_hi, m_W_lo;    // t1 as [k][y][p]  (A of P4, box rows 128)
    CUtensorMap m_sxB_hi, m_sxB_lo, m_syB_hi, m_syB_lo;  // S as B operands, box rows BN
    int tc_bn = 128, tc_nst = 3;
    int tc_persistent = 0, tc_pbn = 128, sms = 152;
    // x-DST + y-Thomas form: per-mode scan-Thomas tables along y and the map of t2 as the
    // [k][y][p] A operand of the inverse x-transform
    int form = 2;          // 2: 2D sine basis (four products); 1: x-DST + y-Thomas
    int yE = 0;            // cells per lane of the y solve (32 lanes per line)
    int ytab_len = 0;      // table entries per x-mode
    void* ytab = nullptr;  // [nx][ytab_len], context dtype (FP32 on the tensor path)
    CUtensorMap m_W2_hi, m_W2_lo;
    // fused x-DST + y-Thomas product (tensor path, ny <= 256): tile N = fbn covers a whole
    // y line, the epilogue eliminates along it; ym[y][p] are the reciprocal pivots
    int fused = 0, fbn = 0, fbk = 16;  // tile N, K block (16: 64-byte swizzle, deeper ring)
    void* ym = nullptr;
    CUtensorMap m_Rf_hi, m_Rf_lo;    // t2 as [k][y][x], box (fbk, fbn) (B of the fused product)
    CUtensorMap m_sxf_hi, m_sxf_lo;  // Sx, box (fbk, 128) (A of the fused product)
    // gather form of the fused product (R formed in shared memory from u and b): maps of the
    // grids it reads, [k][y][x] with box (16, fbn), cached by address
    int fgather = 0;
    struct GridMap {
        const void* ptr = nullptr;
        CUtensorMap map;
    };
    GridMap gmaps[4];
    int gnext = 0;
    // x-sine form of calls of several sweeps (plane_modes.cu): b^ and u^ as [k][p][y], the
    // per-mode factor tables with omega folded in, and the tensor maps of the mode arrays
    int modes = 0;          // available for this context
    int modes_min = 2;      // smallest sweep count per call that takes it
    ModeCfg mcfg;
    void* mb = nullptr;     // b^
    void* mu = nullptr;     // u^
    void* mtab = nullptr;   // [nx][mcfg.tab_len], context dtype
    void* mv = nullptr;     // second vector of Gauss-Seidel in one launch per sweep
    int gs_fused = 1;       // GS: one launch per sweep (zebra order into mv), else two in place
    CUtensorMap mm_b, mm_u, mm_v;  // maps of mb, mu and the second vector (mv or scratch)
    const void* mm_v_ptr = nullptr;
    // FP64: the twisted-elimination form of the mode-line sweep, arrays [k][y][p]
    // (plane_modes_f64.cu); b^ is stored scaled by omega pv (tscale) by the forward product
    int twist = 0;
    void* tfm = nullptr;     // [Rc][nx]: ay p_s of mode p
    void* tfb = nullptr;     // [Rc][nx]: omega p_s az
    void* tgm = nullptr;     // [nx]: ay g_m (twist cell)
    void* tgb = nullptr;     // [nx]: omega g_m az
    void* tscale = nullptr;  // [ny][nx]: omega pv_y
    void* mz = nullptr;      // Gauss-Seidel: the elimination's values
    // the x-DST products of this form by the even/odd symmetry (dst_fold_forward / _inverse)
    void* tSe = nullptr;     // [Ks][Ks]: S[2q][x]
    void* tSo = nullptr;     // [Kd][Kd]: S[2q+1][x]
    void* tSeT = nullptr;    // transposes
    void* tSoT = nullptr;
    int fold = 1;            // BRSMOOTH_MODE_FOLD=0: the plain products
};

// Map of a grid for the gather form, encoded on first use of its address.
const CUtensorMap* grid_map(PlaneState* P, const brs_params& p, const void* ptr)
{
    for (auto& e : P->gmaps)
        if (e.ptr == ptr)
            return &e.map;
    PlaneState::GridMap& e = P->gmaps[P->gnext];
    e.ptr = nullptr;
    if (brs_tc::encode_map(&e.map, ptr, p.nx, p.ny, p.nz, P->fbn, 16) != BRS_OK)
        return nullptr;
    e.ptr = ptr;
    P->gnext = (P->gnext + 1) % 4;
    return &e.map;
}

// Tile shapes of the tensor-core products (N per CTA, ring stages): 128 x 128 tiles with a
// deep ring at one CTA per SM, or 128 x 64 tiles at two CTAs per SM (one CTA's epilogue
// overlaps the other's main loop).
struct TcShape {
    int bn, nst;
};

size_t tc_smem(int split, int bn, int nst)
{
    const size_t stage = (size_t)(split == 3 ? 2 : 1) * (brs_tc::BM + bn) * brs_tc::BK * 4;
    return 1024 + nst * stage + (2 * nst + 1) * 8 + 16;
}

PlaneState* ps(brs_ctx* c)
{
    return static_cast<PlaneState*>(c->plane);
}

// ------------------------------------------------------------------- gather kernel
// R_k = b_k + az (u_{k-1} + u_{k+1}) for planes k = k0, k0 + kstep, ...; R is packed by
// batch index (batch i holds plane k0 + i*kstep).
template <typename T>
__global__ void plane_gather_kernel(const T* __restrict__ u, const T* __restrict__ b,
                                    T* __restrict__ R, int nx, int ny, int nz, double az,
                                    int k0, int kstep, int nbatch)
{
    pdl_wait_trigger();
    const long long plane = (long long)nx * ny;
    const long long total = plane * nbatch;
    const T cz = (T)az;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long bi = t / plane;
        const long long o = t - bi * plane;
        const int k = k0 + (int)bi * kstep;
        const long long g = (long long)k * plane + o;
        const T s = (k > 0 ? u[g - plane] : T(0)) + (k + 1 < nz ? u[g + plane] : T(0));
        R[t] = fma(cz, s, b[g]);
    }
}

// ------------------------------------------------------------------- SIMT batched GEMM
// C_b[m][n] = sum_k A_b[m][k] * B_b[n][k]  (both operands K-major), 64x64 tiles,
// 256 threads, 4x4 outputs per thread.  Batch b uses A + b*strideA (strideA = 0 for a
// shared basis matrix), likewise B and C.
enum Epi { EPI_STORE = 0, EPI_SCALE = 1, EPI_UPDATE = 2 };

struct GemmArgs {
    int M, N, K;
    long long strideA, strideB, strideC;  // elements per batch
    const void* scale;                    // EPI_SCALE: [M][N] factors
    const void* u;                        // EPI_UPDATE: old plane values, [M][N]
    long long strideU;
    int k0, kstep;                        // EPI_UPDATE: batch b -> plane k0 + b*kstep
    double omega;
};

constexpr int BM = 64, BN = 64, BK = 16;

template <typename T, int EPI>
__global__ void __launch_bounds__(256) gemm_tn_simt(const T* __restrict__ A,
                                                    const T* __restrict__ B, T* C, GemmArgs g)
{
    pdl_wait_trigger();
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int bidx = blockIdx.z;
    const T* Ab = A + (long long)bidx * g.strideA;
    const T* Bb = B + (long long)bidx * g.strideB;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            acc[i][j] = T(0);
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        // each thread loads 4 elements of A's and of B's 64x16 tile
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = threadIdx.x + r * 256;
            const int row = idx / BK, kk = idx % BK;
            const int gm = m0 + row, gn = n0 + row, gk = k0 + kk;
            As[kk][row] = (gm < g.M && gk < g.K) ? Ab[(long long)gm * g.K + gk] : T(0);
            Bs[kk][row] = (gn < g.N && gk < g.K) ? Bb[(long long)gn * g.K + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], bv[4];
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
    T* Cb = C + (long long)bidx * g.strideC;
    const T om = (T)g.omega, om1 = (T)(1.0 - g.omega);
    const T* Ub = nullptr;
    if (EPI == EPI_UPDATE)
        Ub = static_cast<const T*>(g.u) + (long long)(g.k0 + bidx * g.kstep) * g.strideU;
    if (EPI == EPI_UPDATE)
        Cb = C + (long long)(g.k0 + bidx * g.kstep) * g.strideC;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m < g.M && n < g.N) {
                const long long o = (long long)m * g.N + n;
                T v = acc[i][j];
                if (EPI == EPI_SCALE)
                    v *= static_cast<const T*>(g.scale)[o];
                if (EPI == EPI_UPDATE)
                    v = fma(om, v, om1 * Ub[o]);
                Cb[o] = v;
            }
        }
}

template <typename T, int EPI>
cudaError_t launch_gemm(const T* A, const T* B, T* C, const GemmArgs& g, int batch,
                        cudaStream_t s)
{
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch);
    return launch_pdl(gemm_tn_simt<T, EPI>, grid, dim3(256), 0, s, A, B, C, g);
}

// R_k = b_k + az (u_{k-1} + u_{k+1}) split into TF32 hi/lo parts, stored at plane k.
// Four cells per thread with 16-byte accesses (nx * ny is a multiple of 4 on this path).
__global__ void plane_gather_split_kernel(const float* __restrict__ u, const float* __restrict__ b,
                                          float* __restrict__ rhi, float* __restrict__ rlo,
                                          int nx, int ny, int nz, float az, int k0, int kstep,
                                          int nbatch, int split)
{
    pdl_wait_trigger();
    const long long plane = (long long)nx * ny;
    const long long plane4 = plane / 4;
    const long long total4 = plane4 * nbatch;
    const float4* u4 = reinterpret_cast<const float4*>(u);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    float4* hi4 = reinterpret_cast<float4*>(rhi);
    float4* lo4 = reinterpret_cast<float4*>(rlo);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total4;
         t += (long long)gridDim.x * blockDim.x) {
        const long long bi = t / plane4;
        const long long o = t - bi * plane4;
        const int k = k0 + (int)bi * kstep;
        const long long gi = (long long)k * plane4 + o;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 um = k > 0 ? u4[gi - plane4] : z4;
        const float4 up = k + 1 < nz ? u4[gi + plane4] : z4;
        const float4 bb = b4[gi];
        float r[4] = {fmaf(az, um.x + up.x, bb.x), fmaf(az, um.y + up.y, bb.y),
                      fmaf(az, um.z + up.z, bb.z), fmaf(az, um.w + up.w, bb.w)};
        float h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t hb = brs_tc::tf32_rn(r[q]);
            h[q] = __uint_as_float(hb);
            l[q] = __uint_as_float(brs_tc::tf32_rn(r[q] - h[q]));
        }
        hi4[gi] = make_float4(h[0], h[1], h[2], h[3]);
        if (split == 3)
            lo4[gi] = make_float4(l[0], l[1], l[2], l[3]);
    }
}

template <int SPLIT, int EPI, int BNT, int NST>
const void* tc_kernel()
{
    return (const void*)brs_tc::tc_gemm_kernel<SPLIT, EPI, BNT, NST>;
}

template <int SPLIT, int EPI>
const void* tc_kernel_for(int bn, int nst)
{
    if (bn == 64)
        return SPLIT == 3 ? tc_kernel<SPLIT, EPI, 64, 2>() : tc_kernel<SPLIT, EPI, 64, 4>();
    return tc_kernel<SPLIT, EPI, 128, 3>();
}

using brs_tc::pers_nst;
using brs_tc::pers_smem;

template <int SPLIT, int EPI>
const void* pers_kernel_for(int bn)
{
    if (bn == 64)
        return (const void*)brs_tc::tc_gemm_persistent<SPLIT, EPI, 64, pers_nst(SPLIT, 64)>;
    if (bn == 256)
        return (const void*)brs_tc::tc_gemm_persistent<SPLIT, EPI, 256, pers_nst(SPLIT, 256)>;
    return (const void*)brs_tc::tc_gemm_persistent<SPLIT, EPI, 128, pers_nst(SPLIT, 128)>;
}

using brs_tc::ring_nst;

template <int SPLIT, int BKT>
const void* fused_kernel_bk(int bn)
{
    using brs_tc::EPI_YTHOMAS;
    if (bn == 64)
        return (const void*)
            brs_tc::tc_gemm_persistent<SPLIT, EPI_YTHOMAS, 64, ring_nst(SPLIT, 64, BKT), BKT>;
    if (bn == 128)
        return (const void*)
            brs_tc::tc_gemm_persistent<SPLIT, EPI_YTHOMAS, 128, ring_nst(SPLIT, 128, BKT), BKT>;
    return (const void*)
        brs_tc::tc_gemm_persistent<SPLIT, EPI_YTHOMAS, 256, ring_nst(SPLIT, 256, BKT), BKT>;
}

template <int SPLIT>
const void* fused_kernel_for(int bn, int bk)
{
    return bk == 16 ? fused_kernel_bk<SPLIT, 16>(bn) : fused_kernel_bk<SPLIT, 32>(bn);
}

template <int SPLIT>
const void* gather_kernel_for(int bn)
{
    using brs_tc::EPI_YGATHER;
    using brs_tc::gather_nst;
    if (bn == 64)
        return (const void*)
            brs_tc::tc_gemm_persistent<SPLIT, EPI_YGATHER, 64, gather_nst(SPLIT, 64), 16>;
    if (bn == 128)
        return (const void*)
            brs_tc::tc_gemm_persistent<SPLIT, EPI_YGATHER, 128, gather_nst(SPLIT, 128), 16>;
    return (const void*)
        brs_tc::tc_gemm_persistent<SPLIT, EPI_YGATHER, 256, gather_nst(SPLIT, 256), 16>;
}

// ring + barriers (full, empty, 2 accf, 2 acce, done, 4 pair, nst converted) + TMEM slot and
// abort flag + exchange area, after 1024 bytes of alignment slack
size_t gather_smem(int split, int bn)
{
    const int nst = brs_tc::gather_nst(split, bn);
    return 1024 + (size_t)nst * brs_tc::gather_stage(split, bn) + (size_t)(3 * nst + 9) * 8 + 8 +
           2 * 4 * 64 * 4 + 16;
}

size_t fused_smem(int split, int bn, int bk)
{
    const int nst = split == 3 ? (bk == 16 ? ring_nst(3, bn, 16) : ring_nst(3, bn, 32))
                               : (bk == 16 ? ring_nst(1, bn, 16) : ring_nst(1, bn, 32));
    return pers_smem(split, bn, nst, bk) + brs_tc::kTwistExtra;
}

template <int SPLIT, int EPI>
cudaError_t launch_tc(const PlaneState* P, const CUtensorMap& ah, const CUtensorMap& al,
                      const CUtensorMap& bh, const CUtensorMap& bl, const brs_tc::TcArgs& g,
                      int nbatch, cudaStream_t s)
{
    if (P->tc_persistent) {
        const int bn = P->tc_pbn;
        int tn = (g.N + bn - 1) / bn, tm = (g.M + brs_tc::BM - 1) / brs_tc::BM, nb = nbatch;
        const long long ntiles = (long long)tn * tm * nb;
        const int grid = (int)(ntiles < P->sms ? ntiles : P->sms);
        CUtensorMap a0 = ah, a1 = al, b0 = bh, b1 = bl;
        brs_tc::TcArgs gg = g;
        void* args[] = {&a0, &a1, &b0, &b1, &gg, &tn, &tm, &nb};
        return launch_pdl_c(pers_kernel_for<SPLIT, EPI>(bn), dim3(grid), dim3(192),
                            pers_smem(SPLIT, bn), s, args);
    }
    const int bn = P->tc_bn, nst = P->tc_nst;
    const void* k = tc_kernel_for<SPLIT, EPI>(bn, nst);
    dim3 grid((g.N + bn - 1) / bn, (g.M + brs_tc::BM - 1) / brs_tc::BM, nbatch);
    CUtensorMap a0 = ah, a1 = al, b0 = bh, b1 = bl;
    brs_tc::TcArgs gg = g;
    void* args[] = {&a0, &a1, &b0, &b1, &gg};
    return launch_pdl_c(k, grid, dim3(128), tc_smem(SPLIT, bn, nst), s, args);
}

template <int SPLIT>
int plane_pass_tc(brs_ctx* c, const float* uin, float* uout, const float* b, int k0, int kstep,
                  int nbatch, cudaStream_t s)
{
    PlaneState* P = ps(c);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const long long plane = (long long)nx * ny;
    {
        int blocks = (int)((plane / 4 * nbatch + 255) / 256);
        if (blocks > 152 * 16)
            blocks = 152 * 16;
        cudaError_t e = launch_pdl(plane_gather_split_kernel, dim3(blocks), dim3(256), 0, s, uin,
                                   b, (float*)P->t2, (float*)P->t2_lo, nx, ny, nz,
                                   (float)c->p.az, k0, kstep, nbatch, SPLIT);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
    }
    brs_tc::TcArgs g{};
    g.k0 = k0;
    g.kstep = kstep;
    g.plane = plane;
    g.status = c->dev_status;
    cudaError_t e;
    // P1: C1[p][y] = sum_x Sx[p][x] R[y][x]
    g.M = nx; g.N = ny; g.K = nx; g.a_batched = 0; g.b_batched = 1;
    g.out_hi = (float*)P->t1; g.out_lo = (float*)P->t1_lo;
    e = launch_tc<SPLIT, brs_tc::EPI_SPLIT>(P, P->m_sx_hi, P->m_sx_lo, P->m_R_hi, P->m_R_lo, g, nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    // P2: Q[p][q] = (sum_y C1[p][y] Sy[q][y]) / L[q][p]
    g.M = nx; g.N = ny; g.K = ny; g.a_batched = 1; g.b_batched = 0;
    g.out_hi = (float*)P->t2; g.out_lo = (float*)P->t2_lo; g.scale = (const float*)P->ilam;
    e = launch_tc<SPLIT, brs_tc::EPI_SCALE_SPLIT>(P, P->m_C1_hi, P->m_C1_lo, P->m_syB_hi, P->m_syB_lo, g,
                                           nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    // P3: W[y][p] = sum_q Sy[y][q] Q[p][q]
    g.M = ny; g.N = nx; g.K = ny; g.a_batched = 0; g.b_batched = 1;
    g.out_hi = (float*)P->t1; g.out_lo = (float*)P->t1_lo; g.scale = nullptr;
    e = launch_tc<SPLIT, brs_tc::EPI_SPLIT>(P, P->m_sy_hi, P->m_sy_lo, P->m_Q_hi, P->m_Q_lo, g, nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    // P4: X[y][x] = sum_p W[y][p] Sx[x][p]; u_k <- (1-omega) u_k + omega X
    g.M = ny; g.N = nx; g.K = nx; g.a_batched = 1; g.b_batched = 0;
    g.out_hi = nullptr; g.out_lo = nullptr; g.u = uin; g.uout = uout; g.omega = (float)c->omega;
    e = launch_tc<SPLIT, brs_tc::EPI_UPDATE>(P, P->m_W_hi, P->m_W_lo, P->m_sxB_hi, P->m_sxB_lo, g, nbatch, s);
    return brs_cuda_status(e);
}

// y-Thomas of the x-DST form: for x-mode p the plane block reduces to the tridiagonal system
//   (ay Ty + (ax s_p + 2 az) I) w = C1[p][:]   (along y),
// solved exactly with the cross-lane scan Thomas (32 lanes per line, E cells per lane) and
// pivots factored once per mode.  A CTA owns 8 consecutive modes (one warp each, tables
// loaded once) over a chunk of planes; each plane's 8 solved lines are written transposed,
// W[k][y][p], through a padded shared-memory tile (32-byte row segments).
// SPLIT = 3/1: input and output are TF32 hi (+lo) pairs; SPLIT = 0: plain T.
constexpr int kYModes = 8;     // modes (warps) per CTA
constexpr int kYPlanes = 8;    // planes per CTA

__host__ __device__ inline int ythomas_stride(int ny)
{
    const int s0 = ny + (ny >> 3) + 1;
    return s0 + (((4 - s0) % 32) + 32) % 32;
}

// FP32: at most 80 registers for lanes of <= 8 cells (3 CTAs per SM), 128 for 12-16 (2 CTAs
// per SM: ny = 512 went from one CTA at 167 registers to two at 128 without spills, and the
// 512^3 split-TF32 plane sweep from 60.4 to 65.5 Gcell/s on the same box).
template <typename T, int E, int SPLIT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (E <= 8 ? 3 : 2) : 1) plane_ythomas_kernel(const T* __restrict__ cin_hi,
                                                               const T* __restrict__ cin_lo,
                                                               T* __restrict__ w_hi,
                                                               T* __restrict__ w_lo,
                                                               const T* __restrict__ ytab,
                                                               int tab_len, int nx, int ny, int k0,
                                                               int kstep, int nbatch)
{
    extern __shared__ __align__(16) unsigned char ysm[];
    // two tiles, alternating by plane: a plane's transposed write reads one tile while the
    // next plane's solves fill the other, so one barrier per plane suffices.
    // tile[m][y] at m * stride + y + y / 8: a pad word after every 8 cells makes a lane's
    // 8-cell chunk writes hit distinct banks, and stride = 4 (mod 32) does the same for the
    // transposed reads of 8 modes x 4 consecutive y
    const int stride = ythomas_stride(ny);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kYModes + warp;
    const bool pin = p < nx;  // warp-uniform
    const long long plane = (long long)nx * ny;
    const bool vec = sizeof(T) == 4 && (ny % 4) == 0 && (E % 4) == 0;  // 16-byte FP32 pieces
    brs::LineTables<T, E, 32> tb;
    tb.load(ytab + (long long)(pin ? p : 0) * tab_len, lane);
    pdl_wait_trigger();
    const int b0 = blockIdx.y * kYPlanes;
    const int b1 = min(nbatch, b0 + kYPlanes);
    // this lane's E cells of mode p's row in the plane of batch index bi
    auto load_row = [&](int bi, T (&v)[E]) {
        const long long row = (long long)(k0 + bi * kstep) * plane + (long long)p * ny;
        const int y0 = lane * E;
        if constexpr (sizeof(T) == 4 && E % 4 == 0) {
            if (vec && y0 + E <= ny) {
#pragma unroll
                for (int q = 0; q < E; q += 4) {
                    const float4 h = __ldg(reinterpret_cast<const float4*>(cin_hi + row + y0 + q));
                    v[q] = h.x;
                    v[q + 1] = h.y;
                    v[q + 2] = h.z;
                    v[q + 3] = h.w;
                }
                if (SPLIT == 3 && cin_lo) {
#pragma unroll
                    for (int q = 0; q < E; ++q)
                        v[q] += cin_lo[row + y0 + q];
                }
                return;
            }
        }
        {
#pragma unroll
            for (int q = 0; q < E; ++q)
                v[q] = (y0 + q < ny) ? cin_hi[row + y0 + q] : T(0);
        }
        if (SPLIT == 3 && cin_lo) {
#pragma unroll
            for (int q = 0; q < E; ++q)
                if (y0 + q < ny)
                    v[q] += cin_lo[row + y0 + q];
        }
    };
    T rn[E];
    if (pin && b0 < b1)
        load_row(b0, rn);
    for (int bi = b0; bi < b1; ++bi) {
        const int k = k0 + bi * kstep;
        T* tile = reinterpret_cast<T*>(ysm) + (size_t)((bi - b0) & 1) * kYModes * stride;
        if (pin) {
            T r[E];
#pragma unroll
            for (int q = 0; q < E; ++q)
                r[q] = rn[q];
            if (bi + 1 < b1)
                load_row(bi + 1, rn);  // the next plane's row, in flight during this solve
            brs::line_solve<T, E, 32>(r, tb, lane);
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const int y = lane * E + q;
                if (y < ny)
                    tile[warp * stride + y + (y >> 3)] = tb.wp[q] * r[q];
            }
        }
        __syncthreads();
        // transposed write: thread (y-row, mode) pairs, 8 consecutive modes per row
        for (int t = threadIdx.x; t < ny * kYModes; t += blockDim.x) {
            const int y = t / kYModes, m = t % kYModes;
            const int pp = blockIdx.x * kYModes + m;
            if (pp < nx) {
                const T v = tile[m * stride + y + (y >> 3)];
                const long long o = (long long)k * plane + (long long)y * nx + pp;
                if (SPLIT == 0) {
                    w_hi[o] = v;
                } else {
                    const uint32_t hi = brs_tc::tf32_rn((float)v);
                    w_hi[o] = __uint_as_float(hi);
                    if (SPLIT == 3)
                        w_lo[o] = __uint_as_float(brs_tc::tf32_rn((float)v - __uint_as_float(hi)));
                }
            }
        }
    }
}

template <typename T, int SPLIT>
cudaError_t launch_ythomas(const PlaneState* P, const T* cin_hi, const T* cin_lo, T* w_hi,
                           T* w_lo, int nx, int ny, int k0, int kstep, int nbatch, cudaStream_t s)
{
    const size_t smem = 2 * (size_t)kYModes * ythomas_stride(ny) * sizeof(T);
    dim3 grid((nx + kYModes - 1) / kYModes, (nbatch + kYPlanes - 1) / kYPlanes);
    const T* tab = static_cast<const T*>(P->ytab);
    const int tl = P->ytab_len;
#define BRS_YT_CASE(EE)                                                                          \
    if (P->yE == EE) {                                                                           \
        return launch_pdl(plane_ythomas_kernel<T, EE, SPLIT>, grid, dim3(256), smem, s, cin_hi,  \
                          cin_lo, w_hi, w_lo, tab, tl, nx, ny, k0, kstep, nbatch);               \
    }
    BRS_YT_CASE(4)
    BRS_YT_CASE(8)
    BRS_YT_CASE(12)
    BRS_YT_CASE(16)
#undef BRS_YT_CASE
    return cudaErrorInvalidConfiguration;
}

template <typename T, int SPLIT>
const void* ythomas_kernel_for(int E)
{
    if (E == 4) return (const void*)plane_ythomas_kernel<T, 4, SPLIT>;
    if (E == 8) return (const void*)plane_ythomas_kernel<T, 8, SPLIT>;
    if (E == 12) return (const void*)plane_ythomas_kernel<T, 12, SPLIT>;
    return (const void*)plane_ythomas_kernel<T, 16, SPLIT>;
}

// x-DST + y-Thomas form on the tensor path: gather, P1 (x-DST), y-Thomas, P4 (inverse x-DST
// fused with the update).
template <int SPLIT>
int plane_pass_tc_xdst(brs_ctx* c, const float* uin, float* uout, const float* b, int k0,
                       int kstep, int nbatch, cudaStream_t s)
{
    PlaneState* P = ps(c);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const long long plane = (long long)nx * ny;
    brs_tc::TcArgs g{};
    g.k0 = k0;
    g.kstep = kstep;
    g.plane = plane;
    g.status = c->dev_status;
    const CUtensorMap* mu = P->fgather ? grid_map(P, c->p, uin) : nullptr;
    const CUtensorMap* mb = mu ? grid_map(P, c->p, b) : nullptr;
    if (mu && mb) {
        // R_k formed in shared memory, the x-DST, and the y-Thomas in one kernel -> t1 (W)
        g.M = nx; g.N = ny; g.K = nx; g.a_batched = 0; g.b_batched = 1;
        g.out_hi = (float*)P->t1; g.out_lo = (float*)P->t1_lo;
        g.ym = (const float*)P->ym; g.ay = (float)c->p.ay; g.az = (float)c->p.az;
        int tn = 1, tm = (nx + brs_tc::BM - 1) / brs_tc::BM, nb = nbatch;
        const long long ntiles = (long long)tm * nb;
        const int grid = (int)(ntiles < P->sms ? ntiles : P->sms);
        CUtensorMap a0 = P->m_sxf_hi, a1 = P->m_sxf_lo, b0 = *mu, b1 = *mb;
        brs_tc::TcArgs gg = g;
        void* args[] = {&a0, &a1, &b0, &b1, &gg, &tn, &tm, &nb};
        cudaError_t e = launch_pdl_c(gather_kernel_for<SPLIT>(P->fbn), dim3(grid),
                                     dim3(brs_tc::pers_threads<brs_tc::EPI_YGATHER>()),
                                     gather_smem(SPLIT, P->fbn), s, args);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        g.ym = nullptr;
        g.M = ny; g.N = nx; g.K = nx; g.a_batched = 1; g.b_batched = 0;
        g.out_hi = nullptr; g.out_lo = nullptr; g.u = uin; g.uout = uout;
        g.omega = (float)c->omega;
        e = launch_tc<SPLIT, brs_tc::EPI_UPDATE>(P, P->m_W_hi, P->m_W_lo, P->m_sxB_hi,
                                                 P->m_sxB_lo, g, nbatch, s);
        return brs_cuda_status(e);
    }
    {
        int blocks = (int)((plane / 4 * nbatch + 255) / 256);
        if (blocks > 152 * 16)
            blocks = 152 * 16;
        cudaError_t e = launch_pdl(plane_gather_split_kernel, dim3(blocks), dim3(256), 0, s, uin,
                                   b, (float*)P->t2, (float*)P->t2_lo, nx, ny, nz,
                                   (float)c->p.az, k0, kstep, nbatch, SPLIT);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
    }
    if (P->fused) {
        // P1 with the y-Thomas in its epilogue: t1 <- W[k][y][p] (split)
        g.M = nx; g.N = ny; g.K = nx; g.a_batched = 0; g.b_batched = 1;
        g.out_hi = (float*)P->t1; g.out_lo = (float*)P->t1_lo;
        g.ym = (const float*)P->ym; g.ay = (float)c->p.ay;
        int tn = 1, tm = (nx + brs_tc::BM - 1) / brs_tc::BM, nb = nbatch;
        const long long ntiles = (long long)tm * nb;
        const int grid = (int)(ntiles < P->sms ? ntiles : P->sms);
        CUtensorMap a0 = P->m_sxf_hi, a1 = P->m_sxf_lo, b0 = P->m_Rf_hi, b1 = P->m_Rf_lo;
        brs_tc::TcArgs gg = g;
        void* args[] = {&a0, &a1, &b0, &b1, &gg, &tn, &tm, &nb};
        cudaError_t e = launch_pdl_c(fused_kernel_for<SPLIT>(P->fbn, P->fbk), dim3(grid),
                                     dim3(brs_tc::pers_threads<brs_tc::EPI_YTHOMAS>()),
                                     fused_smem(SPLIT, P->fbn, P->fbk), s, args);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        g.ym = nullptr;
        // P4: X[y][x] = sum_p W[y][p] Sx[x][p]; u_k <- (1-omega) u_k + omega X
        g.M = ny; g.N = nx; g.K = nx; g.a_batched = 1; g.b_batched = 0;
        g.out_hi = nullptr; g.out_lo = nullptr; g.u = uin; g.uout = uout;
        g.omega = (float)c->omega;
        e = launch_tc<SPLIT, brs_tc::EPI_UPDATE>(P, P->m_W_hi, P->m_W_lo, P->m_sxB_hi,
                                                 P->m_sxB_lo, g, nbatch, s);
        return brs_cuda_status(e);
    }
    // P1: C1[p][y] = sum_x Sx[p][x] R[y][x]  -> t1, plain FP32 (the y solve is not a
    // tensor-core operand, so it needs no TF32 split)
    g.M = nx; g.N = ny; g.K = nx; g.a_batched = 0; g.b_batched = 1;
    g.out_hi = (float*)P->t1; g.out_lo = nullptr; g.out_plain = 1;
    cudaError_t e = launch_tc<SPLIT, brs_tc::EPI_SPLIT>(P, P->m_sx_hi, P->m_sx_lo, P->m_R_hi,
                                                        P->m_R_lo, g, nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    g.out_plain = 0;
    // y-Thomas per x-mode: t1 [p][y] -> t2 [y][p], split for P4
    e = launch_ythomas<float, SPLIT>(P, (const float*)P->t1, nullptr, (float*)P->t2,
                                     (float*)P->t2_lo, nx, ny, k0, kstep, nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    // P4: X[y][x] = sum_p W[y][p] Sx[x][p]; u_k <- (1-omega) u_k + omega X
    g.M = ny; g.N = nx; g.K = nx; g.a_batched = 1; g.b_batched = 0;
    g.out_hi = nullptr; g.out_lo = nullptr; g.u = uin; g.uout = uout; g.omega = (float)c->omega;
    e = launch_tc<SPLIT, brs_tc::EPI_UPDATE>(P, P->m_W2_hi, P->m_W2_lo, P->m_sxB_hi, P->m_sxB_lo,
                                             g, nbatch, s);
    return brs_cuda_status(e);
}

// One plane-block solve + update for planes k0, k0+kstep, ... (nbatch of them), reading
// neighbours from `uin` and writing the updated planes to `uout`.
template <typename T>
int plane_pass(brs_ctx* c, const T* uin, T* uout, const T* b, int k0, int kstep, int nbatch,
               cudaStream_t s)
{
    PlaneState* P = ps(c);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const long long plane = (long long)nx * ny;
    T* R = static_cast<T*>(P->t2);
    T* T1 = static_cast<T*>(P->t1);
    T* T2 = static_cast<T*>(P->t2);
    const T* Sx = static_cast<const T*>(P->sx);
    const T* Sy = static_cast<const T*>(P->sy);
    {
        const long long total = plane * nbatch;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 152 * 16)
            blocks = 152 * 16;
        cudaError_t e = launch_pdl(plane_gather_kernel<T>, dim3(blocks), dim3(256), 0, s, uin, b,
                                   R, nx, ny, nz, c->p.az, k0, kstep, nbatch);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
    }
    cudaError_t e;
    GemmArgs g{};
    // P1: C1[p][y] = sum_x Sx[p][x] R[y][x]
    g.M = nx; g.N = ny; g.K = nx; g.strideA = 0; g.strideB = plane; g.strideC = plane;
    e = launch_gemm<T, EPI_STORE>(Sx, R, T1, g, nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    if (P->form == 1) {
        // y-Thomas per x-mode (T1 [p][y] -> T2 [y][p]), then the inverse x-DST fused with the
        // update; P1 wrote plane b of T1 at b*plane, so pass k0 = 0, kstep = 1 here
        e = launch_ythomas<T, 0>(P, T1, nullptr, T2, nullptr, nx, ny, 0, 1, nbatch, s);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        g = GemmArgs{};
        g.M = ny; g.N = nx; g.K = nx; g.strideA = plane; g.strideB = 0; g.strideC = plane;
        g.u = uin; g.strideU = plane; g.k0 = k0; g.kstep = kstep; g.omega = c->omega;
        e = launch_gemm<T, EPI_UPDATE>(T2, Sx, uout, g, nbatch, s);
        return brs_cuda_status(e);
    }
    // P2: Q[p][q] = (sum_y C1[p][y] Sy[q][y]) / L[q][p]
    g = GemmArgs{};
    g.M = nx; g.N = ny; g.K = ny; g.strideA = plane; g.strideB = 0; g.strideC = plane;
    g.scale = P->ilam;
    e = launch_gemm<T, EPI_SCALE>(T1, Sy, T2, g, nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    // P3: W[y][p] = sum_q Sy[y][q] Q[p][q]
    g = GemmArgs{};
    g.M = ny; g.N = nx; g.K = ny; g.strideA = 0; g.strideB = plane; g.strideC = plane;
    e = launch_gemm<T, EPI_STORE>(Sy, T2, T1, g, nbatch, s);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    // P4: X[y][x] = sum_p W[y][p] Sx[x][p], then u_k <- (1-omega) u_k + omega X
    g = GemmArgs{};
    g.M = ny; g.N = nx; g.K = nx; g.strideA = plane; g.strideB = 0; g.strideC = plane;
    g.u = uin; g.strideU = plane; g.k0 = k0; g.kstep = kstep; g.omega = c->omega;
    e = launch_gemm<T, EPI_UPDATE>(T1, Sx, uout, g, nbatch, s);
    return brs_cuda_status(e);
}

// ------------------------------------------------------------------- x-sine form
// A call of several sweeps runs in the x-sine basis (plane_modes.cu): u^ = S_x u and
// b^ = S_x b once (layout [k][p][y]), the sweeps as mode-line sweeps of u^, then u = S_x u^.
// The transforms are the x-DST products of the per-sweep form: P1 (A = Sx, B = the grid) for
// the forward one, P4 (A = u^ as [k][y][p], B = Sx) for the inverse one.

// TF32 split of an FP32 array, four values per thread with 16-byte accesses.
__global__ void split_tf32_kernel(const float* __restrict__ x, float* __restrict__ hi,
                                  float* __restrict__ lo, long long n4, int split)
{
    pdl_wait_trigger();
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* h4 = reinterpret_cast<float4*>(hi);
    float4* l4 = reinterpret_cast<float4*>(lo);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n4;
         t += (long long)gridDim.x * blockDim.x) {
        const float4 v = x4[t];
        const float r[4] = {v.x, v.y, v.z, v.w};
        float h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = __uint_as_float(brs_tc::tf32_rn(r[q]));
            l[q] = __uint_as_float(brs_tc::tf32_rn(r[q] - h[q]));
        }
        h4[t] = make_float4(h[0], h[1], h[2], h[3]);
        if (split == 3)
            l4[t] = make_float4(l[0], l[1], l[2], l[3]);
    }
}

// [k][p][y] -> [k][y][p] through 32 x 32 shared-memory tiles.  SPLIT = 3 / 1: TF32 hi (+ lo)
// outputs for a tensor-core operand; 0: a plain copy.
template <typename T, int SPLIT>
__global__ void __launch_bounds__(256) modes_to_rows_kernel(const T* __restrict__ src,
                                                            T* __restrict__ hi,
                                                            T* __restrict__ lo, int nm, int ny,
                                                            int nz)
{
    __shared__ T tile[32][33];
    pdl_wait_trigger();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int tiles_y = (ny + 31) / 32;
    const int y0 = (blockIdx.x % tiles_y) * 32, p0 = (blockIdx.x / tiles_y) * 32;
    const long long plane = (long long)nm * ny;
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        const T* sk = src + (long long)k * plane;
        for (int pp = ty; pp < 32; pp += 8) {
            const int p = p0 + pp, y = y0 + tx;
            if (p < nm && y < ny)
                tile[pp][tx] = sk[(long long)p * ny + y];
        }
        __syncthreads();
        for (int yy = ty; yy < 32; yy += 8) {
            const int y = y0 + yy, p = p0 + tx;
            if (p < nm && y < ny) {
                const T v = tile[tx][yy];
                const long long o = (long long)k * plane + (long long)y * nm + p;
                if constexpr (SPLIT == 0) {
                    hi[o] = v;
                } else {
                    const float hb = __uint_as_float(brs_tc::tf32_rn((float)v));
                    hi[o] = hb;
                    if (SPLIT == 3)
                        lo[o] = __uint_as_float(brs_tc::tf32_rn((float)v - hb));
                }
            }
        }
        __syncthreads();
    }
}

bool modes_simt(const brs_ctx* c, const PlaneState* P)
{
    return c->p.dtype == BRS_F64 || P->math == BRS_PLANE_SIMT;
}

// dst[k][p][y] = sum_x Sx[p][x] src[k][y][x]
int modes_forward(brs_ctx* c, const void* src, void* dst, cudaStream_t s)
{
    PlaneState* P = ps(c);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const long long plane = (long long)nx * ny;
    cudaError_t e;
    if (modes_simt(c, P)) {
        GemmArgs g{};
        g.M = nx; g.N = ny; g.K = nx; g.strideA = 0; g.strideB = plane; g.strideC = plane;
        if (c->p.dtype == BRS_F64)
            e = launch_gemm<double, EPI_STORE>(static_cast<const double*>(P->sx),
                                               static_cast<const double*>(src),
                                               static_cast<double*>(dst), g, nz, s);
        else
            e = launch_gemm<float, EPI_STORE>(static_cast<const float*>(P->sx),
                                              static_cast<const float*>(src),
                                              static_cast<float*>(dst), g, nz, s);
        return brs_cuda_status(e);
    }
    const int split = P->math == BRS_PLANE_3XTF32 ? 3 : 1;
    const long long n4 = c->cells / 4;  // nx is a multiple of 32 on the tensor path
    long long blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    e = launch_pdl(split_tf32_kernel, dim3((unsigned)blocks), dim3(256), 0, s,
                   static_cast<const float*>(src), (float*)P->t2, (float*)P->t2_lo, n4, split);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    brs_tc::TcArgs g{};
    g.k0 = 0; g.kstep = 1; g.plane = plane; g.status = c->dev_status;
    g.M = nx; g.N = ny; g.K = nx; g.a_batched = 0; g.b_batched = 1;
    g.out_hi = static_cast<float*>(dst); g.out_lo = nullptr; g.out_plain = 1;
    e = split == 3
            ? launch_tc<3, brs_tc::EPI_SPLIT>(P, P->m_sx_hi, P->m_sx_lo, P->m_R_hi, P->m_R_lo, g, nz, s)
            : launch_tc<1, brs_tc::EPI_SPLIT>(P, P->m_sx_hi, P->m_sx_lo, P->m_R_hi, P->m_R_lo, g, nz, s);
    return brs_cuda_status(e);
}

// dst[k][y][x] = sum_p Sx[x][p] src[k][p][y]  (S is symmetric)
int modes_inverse(brs_ctx* c, const void* src, void* dst, cudaStream_t s)
{
    PlaneState* P = ps(c);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const long long plane = (long long)nx * ny;
    const dim3 tgrid((unsigned)(((ny + 31) / 32) * ((nx + 31) / 32)), (unsigned)(nz < 65535 ? nz : 65535));
    cudaError_t e;
    if (modes_simt(c, P)) {
        GemmArgs g{};
        g.M = ny; g.N = nx; g.K = nx; g.strideA = plane; g.strideB = 0; g.strideC = plane;
        if (c->p.dtype == BRS_F64) {
            e = launch_pdl(modes_to_rows_kernel<double, 0>, tgrid, dim3(256), 0, s,
                           static_cast<const double*>(src), (double*)P->t2, (double*)nullptr, nx,
                           ny, nz);
            if (e == cudaSuccess)
                e = launch_gemm<double, EPI_STORE>((const double*)P->t2,
                                                   static_cast<const double*>(P->sx),
                                                   static_cast<double*>(dst), g, nz, s);
        } else {
            e = launch_pdl(modes_to_rows_kernel<float, 0>, tgrid, dim3(256), 0, s,
                           static_cast<const float*>(src), (float*)P->t2, (float*)nullptr, nx,
                           ny, nz);
            if (e == cudaSuccess)
                e = launch_gemm<float, EPI_STORE>((const float*)P->t2,
                                                  static_cast<const float*>(P->sx),
                                                  static_cast<float*>(dst), g, nz, s);
        }
        return brs_cuda_status(e);
    }
    const int split = P->math == BRS_PLANE_3XTF32 ? 3 : 1;
    e = split == 3 ? launch_pdl(modes_to_rows_kernel<float, 3>, tgrid, dim3(256), 0, s,
                                static_cast<const float*>(src), (float*)P->t2, (float*)P->t2_lo,
                                nx, ny, nz)
                   : launch_pdl(modes_to_rows_kernel<float, 1>, tgrid, dim3(256), 0, s,
                                static_cast<const float*>(src), (float*)P->t2, (float*)P->t2_lo,
                                nx, ny, nz);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    brs_tc::TcArgs g{};
    g.k0 = 0; g.kstep = 1; g.plane = plane; g.status = c->dev_status;
    g.M = ny; g.N = nx; g.K = nx; g.a_batched = 1; g.b_batched = 0;
    g.out_hi = static_cast<float*>(dst); g.out_lo = nullptr; g.out_plain = 1;
    e = split == 3 ? launch_tc<3, brs_tc::EPI_SPLIT>(P, P->m_W2_hi, P->m_W2_lo, P->m_sxB_hi,
                                                     P->m_sxB_lo, g, nz, s)
                   : launch_tc<1, brs_tc::EPI_SPLIT>(P, P->m_W2_hi, P->m_W2_lo, P->m_sxB_hi,
                                                     P->m_sxB_lo, g, nz, s);
    return brs_cuda_status(e);
}

// Orthonormal DST-I matrix S[i][j] = sqrt(2/(n+1)) sin((i+1)(j+1) pi/(n+1)).
std::vector<double> dst1(int n)
{
    std::vector<double> S((size_t)n * n);
    const double sc = std::sqrt(2.0 / (n + 1));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            // reduce the angle index mod 2(n+1) before the sine for accuracy
            const long long q = ((long long)(i + 1) * (j + 1)) % (2LL * (n + 1));
            S[(size_t)i * n + j] = sc * std::sin(M_PI * (double)q / (n + 1));
        }
    return S;
}

template <typename T>
int upload(void** dst, const std::vector<double>& src)
{
    std::vector<T> h(src.size());
    for (size_t i = 0; i < src.size(); ++i)
        h[i] = (T)src[i];
    cudaError_t e = cudaMalloc(dst, h.size() * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return brs_cuda_status(e);
}

using brs_tc::encode_map;
using brs_tc::upload_split;

// Scan-Thomas tables of the y systems of every x-mode p:
//   tridiag(-ay, ax s_p + 2 ay + 2 az, -ay) of size ny,  s_p = 2 - 2 cos((p+1) pi/(nx+1)).
template <typename T>
int ythomas_setup(brs_ctx* c)
{
    PlaneState* P = ps(c);
    const brs_params& p = c->p;
    const int ny = p.ny;
    P->yE = ny <= 128 ? 4 : ny <= 256 ? 8 : ny <= 384 ? 12 : 16;
    std::vector<T> all;
    for (int q = 0; q < p.nx; ++q) {
        const double sp = 2.0 - 2.0 * std::cos(M_PI * (q + 1) / (p.nx + 1));
        auto t = scan_thomas_tables<T>(ny, p.ay, p.ax * sp + 2.0 * p.ay + 2.0 * p.az, 1.0, P->yE,
                                       32, false);
        P->ytab_len = (int)t.size();
        all.insert(all.end(), t.begin(), t.end());
    }
    cudaError_t e = cudaMalloc(&P->ytab, all.size() * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMemcpy(P->ytab, all.data(), all.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    const size_t smem = 2 * (size_t)kYModes * ythomas_stride(ny) * sizeof(T);
    const void* ks[2];
    if (sizeof(T) == 8) {
        ks[0] = ythomas_kernel_for<T, 0>(P->yE);
        ks[1] = ks[0];
    } else {
        ks[0] = ythomas_kernel_for<T, 3>(P->yE);
        ks[1] = ythomas_kernel_for<T, 1>(P->yE);
    }
    const void* k0s[] = {ks[0], ks[1], ythomas_kernel_for<T, 0>(P->yE)};
    for (const void* k : k0s) {
        cudaFuncAttributes fa{};
        cudaError_t ce = cudaFuncGetAttributes(&fa, k);
        if (ce == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < smem)
            ce = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ce != cudaSuccess)
            return brs_cuda_status(ce);
    }
    return BRS_OK;
}

int tc_setup(brs_ctx* c, const std::vector<double>& sx, const std::vector<double>& sy)
{
    PlaneState* P = ps(c);
    if (!brs_encoder())
        return BRS_ERR_CUDA;
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    int rc = upload_split(&P->sx, &P->sx_lo, sx);
    if (rc == BRS_OK)
        rc = upload_split(&P->sy, &P->sy_lo, sy);
    const size_t bytes = (size_t)c->cells * 4;
    for (void** q : {&P->t1, &P->t2, &P->t1_lo, &P->t2_lo})
        if (rc == BRS_OK)
            rc = brs_cuda_status(cudaMalloc(q, bytes));
    if (rc != BRS_OK)
        return rc;
    const char* env = std::getenv("BRSMOOTH_TC_BN");
    // measured defaults: split-TF32 128x64 tiles (2 stages, 2 CTAs/SM); single TF32 128x128
    // tiles (3 stages, 2 CTAs/SM)
    const int dflt = P->math == BRS_PLANE_3XTF32 ? 64 : 128;
    const int want = env ? std::atoi(env) : dflt;
    P->tc_bn = (want == 64 || want == 128) ? want : dflt;
    P->tc_nst = P->tc_bn == 64 ? (P->math == BRS_PLANE_3XTF32 ? 2 : 4) : 3;
    // persistent warp-specialised products (double-buffered TMEM accumulator)
    const char* penv = std::getenv("BRSMOOTH_TC_PERSISTENT");
    // measured at 256^3 (x-sine form, same box): the persistent kernel, which overlaps a
    // tile's epilogue with the next tile's MMAs, beats two per-tile CTAs per SM for split
    // TF32 and, narrowly, for single TF32 (96.4 vs 95.0 Gcell/s).  Tiles of N = 128 beat
    // N = 256, whose two-stage split-TF32 ring starves the MMA issue (76.0 vs 71.2).
    P->tc_persistent = penv ? std::atoi(penv) != 0 : 1;
    const char* pbn = std::getenv("BRSMOOTH_TC_PBN");
    P->tc_pbn = pbn ? (std::atoi(pbn) == 64 ? 64 : std::atoi(pbn) == 256 ? 256 : 128) : 128;
    cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (P->tc_persistent)
        P->tc_bn = P->tc_pbn;  // B maps' box rows follow the tile N in use
    const int BN = P->tc_bn, BMr = brs_tc::BM;
    int e = BRS_OK;
    auto enc = [&](CUtensorMap* m, const void* p, int k, int r, int pl, int br) {
        if (e == BRS_OK)
            e = encode_map(m, p, k, r, pl, br);
    };
    enc(&P->m_sx_hi, P->sx, nx, nx, 0, BMr);
    enc(&P->m_sx_lo, P->sx_lo, nx, nx, 0, BMr);
    enc(&P->m_sy_hi, P->sy, ny, ny, 0, BMr);
    enc(&P->m_sy_lo, P->sy_lo, ny, ny, 0, BMr);
    enc(&P->m_sxB_hi, P->sx, nx, nx, 0, BN);
    enc(&P->m_sxB_lo, P->sx_lo, nx, nx, 0, BN);
    enc(&P->m_syB_hi, P->sy, ny, ny, 0, BN);
    enc(&P->m_syB_lo, P->sy_lo, ny, ny, 0, BN);
    enc(&P->m_R_hi, P->t2, nx, ny, nz, BN);
    enc(&P->m_R_lo, P->t2_lo, nx, ny, nz, BN);
    enc(&P->m_C1_hi, P->t1, ny, nx, nz, BMr);
    enc(&P->m_C1_lo, P->t1_lo, ny, nx, nz, BMr);
    enc(&P->m_Q_hi, P->t2, ny, nx, nz, BN);
    enc(&P->m_Q_lo, P->t2_lo, ny, nx, nz, BN);
    enc(&P->m_W_hi, P->t1, nx, ny, nz, BMr);
    enc(&P->m_W_lo, P->t1_lo, nx, ny, nz, BMr);
    enc(&P->m_W2_hi, P->t2, nx, ny, nz, BMr);
    enc(&P->m_W2_lo, P->t2_lo, nx, ny, nz, BMr);
    if (e != BRS_OK)
        return e;
    // raise the kernels' dynamic shared-memory limit (never lower it)
    const int split = P->math == BRS_PLANE_3XTF32 ? 3 : 1;
    const void* kern[3];
    if (split == 3) {
        kern[0] = tc_kernel_for<3, brs_tc::EPI_SPLIT>(P->tc_bn, P->tc_nst);
        kern[1] = tc_kernel_for<3, brs_tc::EPI_SCALE_SPLIT>(P->tc_bn, P->tc_nst);
        kern[2] = tc_kernel_for<3, brs_tc::EPI_UPDATE>(P->tc_bn, P->tc_nst);
    } else {
        kern[0] = tc_kernel_for<1, brs_tc::EPI_SPLIT>(P->tc_bn, P->tc_nst);
        kern[1] = tc_kernel_for<1, brs_tc::EPI_SCALE_SPLIT>(P->tc_bn, P->tc_nst);
        kern[2] = tc_kernel_for<1, brs_tc::EPI_UPDATE>(P->tc_bn, P->tc_nst);
    }
    size_t need = tc_smem(split, P->tc_bn, P->tc_nst);
    if (P->tc_persistent) {
        need = pers_smem(split, P->tc_pbn);
        if (split == 3) {
            kern[0] = pers_kernel_for<3, brs_tc::EPI_SPLIT>(P->tc_pbn);
            kern[1] = pers_kernel_for<3, brs_tc::EPI_SCALE_SPLIT>(P->tc_pbn);
            kern[2] = pers_kernel_for<3, brs_tc::EPI_UPDATE>(P->tc_pbn);
        } else {
            kern[0] = pers_kernel_for<1, brs_tc::EPI_SPLIT>(P->tc_pbn);
            kern[1] = pers_kernel_for<1, brs_tc::EPI_SCALE_SPLIT>(P->tc_pbn);
            kern[2] = pers_kernel_for<1, brs_tc::EPI_UPDATE>(P->tc_pbn);
        }
    }
    for (int i = 0; i < 3; ++i) {
        cudaFuncAttributes fa{};
        cudaError_t ce = cudaFuncGetAttributes(&fa, kern[i]);
        if (ce == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < need)
            ce = cudaFuncSetAttribute(kern[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)need);
        if (ce != cudaSuccess)
            return brs_cuda_status(ce);
    }
    return BRS_OK;
}

// Fused x-DST + y-Thomas product: on for the persistent tensor path when one tile's N (64,
// 128 or 256) holds a whole y line.  Reciprocal pivots of tridiag(-ay, d_p, -ay), d_p =
// ax s_p + 2 ay + 2 az, factored in FP64: m_0 = 1 / d_p, m_y = 1 / (d_p - ay^2 m_{y-1}).
int fused_setup(brs_ctx* c)
{
    PlaneState* P = ps(c);
    const brs_params& p = c->p;
    const char* env = std::getenv("BRSMOOTH_PLANE_FUSE");
    const bool want = env ? std::atoi(env) != 0 : true;
    if (!want || !P->tc_persistent || p.ny > 256)
        return BRS_OK;
    P->fbn = p.ny <= 64 ? 64 : p.ny <= 128 ? 128 : 256;
    std::vector<float> m((size_t)p.ny * p.nx);
    for (int q = 0; q < p.nx; ++q) {
        const double sp = 2.0 - 2.0 * std::cos(M_PI * (q + 1) / (p.nx + 1));
        const double d = p.ax * sp + 2.0 * p.ay + 2.0 * p.az;
        double piv = 1.0 / d;
        for (int y = 0; y < p.ny; ++y) {
            if (y > 0)
                piv = 1.0 / (d - p.ay * p.ay * piv);
            m[(size_t)y * p.nx + q] = (float)piv;
        }
    }
    cudaError_t e = cudaMalloc(&P->ym, m.size() * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(P->ym, m.data(), m.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    const char* kenv = std::getenv("BRSMOOTH_PLANE_FUSE_BK");
    P->fbk = (kenv && std::atoi(kenv) == 32) ? 32 : 16;
    int rc = encode_map(&P->m_Rf_hi, P->t2, p.nx, p.ny, p.nz, P->fbn, P->fbk);
    if (rc == BRS_OK)
        rc = encode_map(&P->m_Rf_lo, P->t2_lo, p.nx, p.ny, p.nz, P->fbn, P->fbk);
    if (rc == BRS_OK)
        rc = encode_map(&P->m_sxf_hi, P->sx, p.nx, p.nx, 0, brs_tc::BM, P->fbk);
    if (rc == BRS_OK)
        rc = encode_map(&P->m_sxf_lo, P->sx_lo, p.nx, p.nx, 0, brs_tc::BM, P->fbk);
    if (rc != BRS_OK)
        return rc;
    const int split = P->math == BRS_PLANE_3XTF32 ? 3 : 1;
    const void* k = split == 3 ? fused_kernel_for<3>(P->fbn, P->fbk)
                               : fused_kernel_for<1>(P->fbn, P->fbk);
    const size_t need = fused_smem(split, P->fbn, P->fbk);
    cudaFuncAttributes fa{};
    cudaError_t ce = cudaFuncGetAttributes(&fa, k);
    if (ce == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < need)
        ce = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (ce != cudaSuccess)
        return brs_cuda_status(ce);
    P->fused = 1;
    // gather form: on unless BRSMOOTH_PLANE_FGATHER=0 (K blocks of 16 only)
    const char* genv = std::getenv("BRSMOOTH_PLANE_FGATHER");
    if ((genv ? std::atoi(genv) != 0 : true) && P->fbk == 16) {
        const void* kg = split == 3 ? gather_kernel_for<3>(P->fbn) : gather_kernel_for<1>(P->fbn);
        const size_t gneed = gather_smem(split, P->fbn);
        cudaFuncAttributes ga{};
        cudaError_t ge = cudaFuncGetAttributes(&ga, kg);
        if (ge == cudaSuccess && (size_t)ga.maxDynamicSharedSizeBytes < gneed)
            ge = cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gneed);
        if (ge != cudaSuccess)
            return brs_cuda_status(ge);
        P->fgather = 1;
    }
    return BRS_OK;
}

// FP64 x-sine form with the twisted elimination: per-mode pivots of tridiag(-ay, d_p, -ay),
// d_p = ax s_p + 2 ay + 2 az (twist_pivots, FP64), as the tables the kernel reads per step,
// and the mode arrays; any ny.
int twist_setup(brs_ctx* c)
{
    PlaneState* P = ps(c);
    const brs_params& p = c->p;
    const int nx = p.nx, ny = p.ny, m = (ny - 1) / 2, Rc = ny - 1 - m;
    const double om = c->omega;
    std::vector<double> fm((size_t)(Rc > 0 ? Rc : 1) * nx, 0.0), fb(fm.size(), 0.0);
    std::vector<double> gm(nx), gb(nx), sc((size_t)ny * nx);
    for (int q = 0; q < nx; ++q) {
        const double sp = 2.0 - 2.0 * std::cos(M_PI * (q + 1) / (nx + 1));
        const std::vector<double> pv = twist_pivots(ny, p.ay, p.ax * sp + 2.0 * p.ay + 2.0 * p.az);
        for (int s = 0; s < Rc; ++s) {
            const double ps_ = pv[ny - 1 - s];  // p_s: the right side's pivot at step s
            fm[(size_t)s * nx + q] = p.ay * ps_;
            fb[(size_t)s * nx + q] = om * ps_ * p.az;
        }
        gm[q] = p.ay * pv[m];
        gb[q] = om * pv[m] * p.az;
        for (int y = 0; y < ny; ++y)
            sc[(size_t)y * nx + q] = om * pv[y];
    }
    auto up = [&](void** dst, const std::vector<double>& v) {
        cudaError_t e = cudaMalloc(dst, v.size() * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
        return brs_cuda_status(e);
    };
    // S's even and odd rows on the first ceil(nx/2) / floor(nx/2) columns, and transposes
    const int Kd = nx / 2, Ks = nx - Kd;
    const std::vector<double> S = dst1(nx);
    std::vector<double> se((size_t)Ks * Ks), so((size_t)(Kd > 0 ? Kd : 1) * (Kd > 0 ? Kd : 1), 0.0);
    std::vector<double> set(se.size()), sot(so.size(), 0.0);
    for (int q = 0; q < Ks; ++q)
        for (int x = 0; x < Ks; ++x) {
            se[(size_t)q * Ks + x] = S[(size_t)(2 * q) * nx + x];
            set[(size_t)x * Ks + q] = S[(size_t)(2 * q) * nx + x];
        }
    for (int q = 0; q < Kd; ++q)
        for (int x = 0; x < Kd; ++x) {
            so[(size_t)q * Kd + x] = S[(size_t)(2 * q + 1) * nx + x];
            sot[(size_t)x * Kd + q] = S[(size_t)(2 * q + 1) * nx + x];
        }
    const char* fenv = std::getenv("BRSMOOTH_MODE_FOLD");
    P->fold = !(fenv && *fenv && std::atoi(fenv) == 0);
    int rc = up(&P->tfm, fm);
    if (rc == BRS_OK)
        rc = up(&P->tfb, fb);
    if (rc == BRS_OK)
        rc = up(&P->tSe, se);
    if (rc == BRS_OK)
        rc = up(&P->tSo, so);
    if (rc == BRS_OK)
        rc = up(&P->tSeT, set);
    if (rc == BRS_OK)
        rc = up(&P->tSoT, sot);
    if (rc == BRS_OK)
        rc = up(&P->tgm, gm);
    if (rc == BRS_OK)
        rc = up(&P->tgb, gb);
    if (rc == BRS_OK)
        rc = up(&P->tscale, sc);
    const size_t bytes = (size_t)c->cells * sizeof(double);
    for (void** q : {&P->mb, &P->mu})
        if (rc == BRS_OK)
            rc = brs_cuda_status(cudaMalloc(q, bytes));
    if (rc == BRS_OK && p.method == BRS_CHAOTIC_GS)
        rc = brs_cuda_status(cudaMalloc(&P->mz, bytes));
    if (rc != BRS_OK)
        return rc;
    P->twist = 1;
    P->modes = 1;
    return BRS_OK;
}

// The twisted FP64 form of a call: b^' = (b Sx^T) .* omega pv and u^ = u Sx^T ([k][y][p]), the
// sweeps, u = u^ Sx^T (Sx is symmetric, so one product form serves both directions).
int twist_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s, bool u_zero)
{
    PlaneState* P = ps(c);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const long long plane = (long long)nx * ny;
    const double* Sx = static_cast<const double*>(P->sx);
    GemmArgs g{};
    g.M = ny; g.N = nx; g.K = nx; g.strideA = plane; g.strideB = 0; g.strideC = plane;
    GemmArgs gs_ = g;
    gs_.scale = P->tscale;
    double* mb = static_cast<double*>(P->mb);
    double* mu = static_cast<double*>(P->mu);
    double* w1 = static_cast<double*>(P->t1);
    double* w2 = static_cast<double*>(P->t2);
    const double* Se = static_cast<const double*>(P->tSe);
    const double* So = static_cast<const double*>(P->tSo);
    int rc;
    if (P->fold) {
        rc = dst_fold_forward(static_cast<const double*>(b), mb,
                              static_cast<const double*>(P->tscale), w1, Se, So, nx, ny, nz, s);
        if (rc == BRS_OK)
            rc = u_zero ? brs_cuda_status(cudaMemsetAsync(mu, 0, (size_t)c->cells * sizeof(double), s))
                        : dst_fold_forward(static_cast<const double*>(u), mu, nullptr, w1, Se, So,
                                           nx, ny, nz, s);
    } else {
        cudaError_t e =
            launch_gemm<double, EPI_SCALE>(static_cast<const double*>(b), Sx, mb, gs_, nz, s);
        if (e == cudaSuccess)
            e = u_zero ? cudaMemsetAsync(mu, 0, (size_t)c->cells * sizeof(double), s)
                       : launch_gemm<double, EPI_STORE>(static_cast<const double*>(u), Sx, mu, g,
                                                        nz, s);
        rc = brs_cuda_status(e);
    }
    const double* fm = static_cast<const double*>(P->tfm);
    const double* fb = static_cast<const double*>(P->tfb);
    const double* gm = static_cast<const double*>(P->tgm);
    const double* gb = static_cast<const double*>(P->tgb);
    double* cur = mu;
    if (c->p.method == BRS_CHAOTIC_GS) {
        // even planes, then odd planes, in place; the elimination's values in mz
        double* zs = static_cast<double*>(P->mz);
        for (int it = 0; it < nsweeps && rc == BRS_OK; ++it)
            for (int col = 0; col < 2 && rc == BRS_OK; ++col)
                rc = mode_twist_launch(cur, cur, zs, mb, fm, fb, gm, gb, nx, ny, nz, c->omega,
                                       col, s);
    } else {
        double* nxt = static_cast<double*>(c->scratch);
        for (int it = 0; it < nsweeps && rc == BRS_OK; ++it) {
            rc = mode_twist_launch(cur, nxt, nxt, mb, fm, fb, gm, gb, nx, ny, nz, c->omega, -1, s);
            std::swap(cur, nxt);
        }
    }
    if (rc == BRS_OK)
        rc = P->fold ? dst_fold_inverse(cur, static_cast<double*>(u), w1, w2,
                                        static_cast<const double*>(P->tSeT),
                                        static_cast<const double*>(P->tSoT), nx, ny, nz, s)
                     : brs_cuda_status(
                           launch_gemm<double, EPI_STORE>(cur, Sx, static_cast<double*>(u), g, nz, s));
    return rc;
}

// x-sine form: per-mode scan-Thomas tables of tridiag(-ay, ax s_p + 2 ay + 2 az, -ay) along y
// with the context's omega folded in (factored once in FP64), the mode arrays and their
// maps.  Leaves the form off (per-sweep form only) when BRSMOOTH_PLANE_MODES=0 or the y rows
// cannot be staged by TMA.
template <typename T>
int modes_setup(brs_ctx* c)
{
    PlaneState* P = ps(c);
    const brs_params& p = c->p;
    const char* env = std::getenv("BRSMOOTH_PLANE_MODES");
    if (env && *env && std::atoi(env) == 0)
        return BRS_OK;
    // measured at 256^3 (same box): two split-TF32 sweeps per call take 0.350 ms in this form
    // against 0.304 ms per-sweep (three transforms against four products), ten take 0.61 ms
    // against 1.5; on the SIMT and FP64 paths, whose products are slower, two already gain
    const char* menv = std::getenv("BRSMOOTH_PLANE_MODES_MIN");
    const int dflt = (P->math == BRS_PLANE_TF32 || P->math == BRS_PLANE_3XTF32) ? 3 : 2;
    P->modes_min = (menv && *menv && std::atoi(menv) >= 1) ? std::atoi(menv) : dflt;
    const char* tenv = std::getenv("BRSMOOTH_MODE_TWIST");
    if (sizeof(T) == 8 && !(tenv && *tenv && std::atoi(tenv) == 0))
        return twist_setup(c);
    ModeCfg m;
    int rc = mode_config(p.ny, p.nx, p.nz, p.dtype, c->device, &m);
    if (rc == BRS_ERR_UNSUPPORTED)
        return BRS_OK;
    if (rc != BRS_OK)
        return rc;
    std::vector<T> all;
    all.reserve((size_t)p.nx * m.tab_len);
    for (int q = 0; q < p.nx; ++q) {
        const double sp = 2.0 - 2.0 * std::cos(M_PI * (q + 1) / (p.nx + 1));
        auto t = scan_thomas_tables<T>(p.ny, p.ay, p.ax * sp + 2.0 * p.ay + 2.0 * p.az, c->omega,
                                       m.E, m.G, false);
        if ((int)t.size() != m.tab_len)
            return BRS_ERR_UNSUPPORTED;
        all.insert(all.end(), t.begin(), t.end());
    }
    cudaError_t e = cudaMalloc(&P->mtab, all.size() * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMemcpy(P->mtab, all.data(), all.size() * sizeof(T), cudaMemcpyHostToDevice);
    const size_t bytes = (size_t)c->cells * sizeof(T);
    if (e == cudaSuccess)
        e = cudaMalloc(&P->mb, bytes);
    if (e == cudaSuccess)
        e = cudaMalloc(&P->mu, bytes);
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    rc = mode_encode_map(m, &P->mm_b, P->mb);
    if (rc == BRS_OK)
        rc = mode_encode_map(m, &P->mm_u, P->mu);
    if (rc != BRS_OK)
        return rc;
    // Gauss-Seidel in one launch per sweep writes a second vector (measured at 256^3 FP32:
    // two in-place colour launches per sweep, 16 bytes per cell, 57 us; one launch, 12 bytes
    // per cell: see the x-sine row of the design notes); BRSMOOTH_MODE_GS_FUSED=0 keeps the
    // two launches
    const char* genv = std::getenv("BRSMOOTH_MODE_GS_FUSED");
    P->gs_fused = !(genv && *genv && std::atoi(genv) == 0);
    if (p.method == BRS_CHAOTIC_GS && P->gs_fused) {
        rc = brs_cuda_status(cudaMalloc(&P->mv, bytes));
        if (rc == BRS_OK)
            rc = mode_encode_map(m, &P->mm_v, P->mv);
        if (rc != BRS_OK)
            return rc;
        P->mm_v_ptr = P->mv;
    }
    P->mcfg = m;
    P->modes = 1;
    return BRS_OK;
}

}  // namespace

int plane_setup(brs_ctx* c)
{
    const brs_params& p = c->p;
    if (p.nx > 1024 || p.ny > 1024)
        return BRS_ERR_UNSUPPORTED;
    int math = p.plane_math;
    if (p.dtype == BRS_F64 && (math == BRS_PLANE_TF32 || math == BRS_PLANE_3XTF32))
        return BRS_ERR_UNSUPPORTED;
    // tensor-core path: FP32, both plane sides whole 32-element K blocks
    const bool tc_shape = p.dtype == BRS_F32 && p.nx % 32 == 0 && p.ny % 32 == 0;
    if (math == BRS_PLANE_AUTO)
        math = tc_shape ? BRS_PLANE_3XTF32 : BRS_PLANE_SIMT;
    if ((math == BRS_PLANE_TF32 || math == BRS_PLANE_3XTF32) && !tc_shape)
        return BRS_ERR_UNSUPPORTED;
    PlaneState* P = new PlaneState();
    c->plane = P;
    P->nx = p.nx;
    P->ny = p.ny;
    P->math = math;
    {
        const char* fenv = std::getenv("BRSMOOTH_PLANE_FORM");
        // x-DST + y-Thomas (half the transform work) unless asked for the 2D sine basis or the
        // y lines exceed the scan-Thomas limit of 512 cells
        const int want = fenv ? std::atoi(fenv) : 1;
        P->form = (want == 1 && p.ny <= 512) ? 1 : 2;
    }
    std::vector<double> sx = dst1(p.nx), sy = dst1(p.ny), il((size_t)p.nx * p.ny);
    for (int pp = 0; pp < p.nx; ++pp)
        for (int q = 0; q < p.ny; ++q) {
            const double spx = 2.0 - 2.0 * std::cos(M_PI * (pp + 1) / (p.nx + 1));
            const double sqy = 2.0 - 2.0 * std::cos(M_PI * (q + 1) / (p.ny + 1));
            il[(size_t)pp * p.ny + q] = 1.0 / (p.ax * spx + p.ay * sqy + 2.0 * p.az);
        }
    int rc;
    if (math == BRS_PLANE_TF32 || math == BRS_PLANE_3XTF32) {
        std::vector<float> ilf(il.begin(), il.end());
        rc = brs_cuda_status(cudaMalloc(&P->ilam, ilf.size() * 4));
        if (rc == BRS_OK)
            rc = brs_cuda_status(
                cudaMemcpy(P->ilam, ilf.data(), ilf.size() * 4, cudaMemcpyHostToDevice));
        if (rc == BRS_OK)
            rc = tc_setup(c, sx, sy);
        if (rc == BRS_OK && P->form == 1)
            rc = ythomas_setup<float>(c);
        if (rc == BRS_OK && P->form == 1)
            rc = fused_setup(c);
        if (rc == BRS_OK)
            rc = modes_setup<float>(c);
        return rc;
    }
    if (p.dtype == BRS_F64)
        rc = upload<double>(&P->sx, sx);
    else
        rc = upload<float>(&P->sx, sx);
    if (rc == BRS_OK)
        rc = p.dtype == BRS_F64 ? upload<double>(&P->sy, sy) : upload<float>(&P->sy, sy);
    if (rc == BRS_OK)
        rc = p.dtype == BRS_F64 ? upload<double>(&P->ilam, il) : upload<float>(&P->ilam, il);
    const size_t bytes = (size_t)c->cells * c->esize;
    if (rc == BRS_OK)
        rc = brs_cuda_status(cudaMalloc(&P->t1, bytes));
    if (rc == BRS_OK)
        rc = brs_cuda_status(cudaMalloc(&P->t2, bytes));
    if (rc == BRS_OK && P->form == 1)
        rc = p.dtype == BRS_F64 ? ythomas_setup<double>(c) : ythomas_setup<float>(c);
    if (rc == BRS_OK)
        rc = p.dtype == BRS_F64 ? modes_setup<double>(c) : modes_setup<float>(c);
    return rc;
}

void plane_teardown(brs_ctx* c)
{
    PlaneState* P = ps(c);
    if (!P)
        return;
    for (void* q : {P->sx, P->sy, P->ilam, P->t1, P->t2, P->sx_lo, P->sy_lo, P->t1_lo, P->t2_lo,
                    P->ytab, P->ym, P->mb, P->mu, P->mtab, P->mv, P->tfm, P->tfb, P->tgm,
                    P->tgb, P->tscale, P->mz, P->tSe, P->tSo, P->tSeT, P->tSoT})
        if (q)
            cudaFree(q);
    delete P;
    c->plane = nullptr;
}

int plane_sweep_launch(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s)
{
    const int nz = c->p.nz;
    const bool gs = c->p.method == BRS_CHAOTIC_GS;
    auto run = [&](auto tag) -> int {
        using T = decltype(tag);
        const T* ui = static_cast<const T*>(uin);
        T* uo = static_cast<T*>(uout);
        const T* bb = static_cast<const T*>(b);
        if (!gs)
            return plane_pass<T>(c, ui, uo, bb, 0, 1, nz, s);
        // in place: even planes, then odd planes (which read the new even planes)
        int rc = plane_pass<T>(c, ui, uo, bb, 0, 2, (nz + 1) / 2, s);
        if (rc == BRS_OK && nz > 1)
            rc = plane_pass<T>(c, ui, uo, bb, 1, 2, nz / 2, s);
        return rc;
    };
    if (c->p.dtype == BRS_F64)
        return run(double{});
    const int math = ps(c)->math;
    if (math == BRS_PLANE_TF32 || math == BRS_PLANE_3XTF32) {
        const float* ui = static_cast<const float*>(uin);
        float* uo = static_cast<float*>(uout);
        const float* bb = static_cast<const float*>(b);
        const bool xdst = ps(c)->form == 1;
        auto pass = [&](int k0, int kstep, int nb) {
            if (xdst)
                return math == BRS_PLANE_3XTF32
                           ? plane_pass_tc_xdst<3>(c, ui, uo, bb, k0, kstep, nb, s)
                           : plane_pass_tc_xdst<1>(c, ui, uo, bb, k0, kstep, nb, s);
            return math == BRS_PLANE_3XTF32 ? plane_pass_tc<3>(c, ui, uo, bb, k0, kstep, nb, s)
                                            : plane_pass_tc<1>(c, ui, uo, bb, k0, kstep, nb, s);
        };
        if (!gs)
            return pass(0, 1, nz);
        int rc = pass(0, 2, (nz + 1) / 2);
        if (rc == BRS_OK && nz > 1)
            rc = pass(1, 2, nz / 2);
        return rc;
    }
    return run(float{});
}

int plane_modes_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s,
                      bool u_zero)
{
    PlaneState* P = ps(c);
    if (!P || !P->modes || nsweeps < P->modes_min)
        return BRS_ERR_UNSUPPORTED;
    const bool gs = c->p.method == BRS_CHAOTIC_GS;
    if (!gs && !c->scratch)
        return BRS_ERR_UNSUPPORTED;
    if (P->twist)
        return twist_sweep(c, u, b, nsweeps, s, u_zero);
    const ModeCfg& m = P->mcfg;
    const bool two_pass = gs && !P->gs_fused;
    if (!gs && P->mm_v_ptr != c->scratch) {
        // the Jacobi second vector is the context's scratch array (allocated after set-up)
        int rc = mode_encode_map(m, &P->mm_v, c->scratch);
        if (rc != BRS_OK)
            return rc;
        P->mm_v_ptr = c->scratch;
    }
    int rc = modes_forward(c, b, P->mb, s);
    if (rc == BRS_OK)
        rc = u_zero ? brs_cuda_status(cudaMemsetAsync(P->mu, 0, (size_t)c->cells * c->esize, s))
                    : modes_forward(c, u, P->mu, s);
    const double az = c->p.az, om = c->omega;
    void* cur = P->mu;
    void* nxt = gs ? P->mv : c->scratch;
    const CUtensorMap* mcur = &P->mm_u;
    const CUtensorMap* mnxt = &P->mm_v;
    for (int it = 0; it < nsweeps && rc == BRS_OK; ++it) {
        if (two_pass) {
            // even planes, then odd planes, in place
            rc = mode_sweep_launch(m, &P->mm_u, &P->mm_b, P->mu, P->mtab, az, om, 0, c->dev_status, s);
            if (rc == BRS_OK && c->p.nz > 1)
                rc = mode_sweep_launch(m, &P->mm_u, &P->mm_b, P->mu, P->mtab, az, om, 1,
                                       c->dev_status, s);
        } else {
            // Jacobi, or both colours in one launch (zebra order), into the second vector
            rc = mode_sweep_launch(m, mcur, &P->mm_b, nxt, P->mtab, az, om, gs ? 2 : -1,
                                   c->dev_status, s);
            std::swap(cur, nxt);
            std::swap(mcur, mnxt);
        }
    }
    if (rc == BRS_OK)
        rc = modes_inverse(c, cur, u, s);
    return rc;
}
