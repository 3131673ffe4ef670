// Tensor-core (tcgen05, TF32 / split-TF32) batched products for the xy-plane solve.
//
// The plane solve X = Sy [ (Sy R Sx) ./ L ] Sx runs as four batched "TN" products
// C = A B^T (both operands K-major, one plane per batch index), see plane.cu.  Here each
// product is one kernel:
//   * 128 x BN output tile per CTA, K consumed in blocks of 32 FP32 values (one 128-byte
//     swizzle atom), staged by TMA (SWIZZLE_128B) through an NST-stage shared-memory ring;
//   * one thread issues tcgen05.mma.kind::tf32 (M=128, N=BN, K=8 per instruction) with
//     the FP32 accumulator in tensor memory; tcgen05.commit releases ring slots;
//   * 128 threads read the accumulator back with tcgen05.ld (one TMEM lane = one output
//     row per thread) and apply the epilogue.
// Split-TF32 ("3xTF32", the published technique of representing x = hi + lo with both
// parts TF32 and dropping lo*lo): operands are stored as separate hi and lo arrays,
// hi = rn_tf32(x), lo = rn_tf32(x - hi); every K-step accumulates hi*hi + hi*lo + lo*hi.
// With SPLIT = 1 only the hi parts are used (single TF32 pass).
#pragma once

#include "brs_internal.cuh"

namespace brs_tc {

constexpr int BM = 128;  // MMA M (one TMEM lane per output row)
constexpr int BK = 32;   // K per ring stage: 32 FP32 = one 128-byte swizzle row

enum Epi {
    EPI_SPLIT = 0,
    EPI_SCALE_SPLIT = 1,
    EPI_UPDATE = 2,
    EPI_BOX = 3,
    EPI_YTHOMAS = 4,
    EPI_YGATHER = 5  // EPI_YTHOMAS with B = R_k formed from u and b in shared memory
};

struct TcArgs {
    int M, N, K;        // per-plane product sizes
    int a_batched;      // A is per plane (3D map) or shared (2D map)
    int b_batched;
    int k0, kstep;      // blockIdx.z -> plane k0 + blockIdx.z * kstep
    long long plane;    // elements per plane of the outputs (M * N)
    float* out_hi;      // EPI_SPLIT / EPI_SCALE_SPLIT outputs, [plane][M][N]
    float* out_lo;
    int out_plain;      // EPI_SPLIT / EPI_SCALE_SPLIT: store the FP32 result in out_hi, unsplit
    const float* scale; // EPI_SCALE_SPLIT: [M][N]
    const float* u;     // EPI_UPDATE: old plane values [plane][M][N]
    float* uout;        // EPI_UPDATE: updated planes
    float omega;
    int* status;
    // EPI_BOX (persistent kernel only): output row m is one box block whose packed block
    // coordinates bi | bj << 21 | bk << 42 are box_rows[m]; column l is local cell l, at grid
    // offset box_off[l] from the block's first cell.  u / uout are whole grids.
    const long long* box_rows;
    const int* box_off;
    int box_bx, box_by, box_bz, box_nx, box_ny;
    int box_vec4;  // bx and nx multiples of 4: 4 consecutive local cells are 16 aligned bytes
    // EPI_YTHOMAS (persistent kernel only): row m of the tile is x-mode p = m, its columns
    // are y = 0 .. N-1, and the epilogue solves tridiag(-ay, d_p, -ay) w = row along the
    // columns.  ym[y * M + p] = 1 / (d_p + ay c_{y-1}) are the elimination's reciprocal
    // pivots; w is written to out_hi (/ out_lo) as [plane][y][p], split for the next product.
    const float* ym;
    float ay;
    // EPI_YGATHER: the B maps are u (mB_hi) and b (mB_lo) as [k][y][x]; each stage loads the
    // boxes of u_{k-1}, u_{k+1} and b_k (planes outside the grid read as zeros) and converter
    // warps form R = b_k + az (u_{k-1} + u_{k+1}) and its TF32 split in place.
    float az;
};

#ifdef __CUDACC__

__device__ __forceinline__ uint32_t tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with SWIZZLE_128B:
// rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* tile)
{
    const uint64_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;          // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                  // fixed constant 0b001
    d |= (uint64_t)2 << 61;                  // swizzle: 128-byte
    return d;
}

// Descriptor of a K-major tile written by TMA with a swizzle as wide as its rows: BKT = 32
// FP32 (128-byte rows, SWIZZLE_128B, 8-row groups 1024 bytes apart) or BKT = 16 (64-byte
// rows, SWIZZLE_64B, 8-row groups 512 bytes apart).
template <int BKT>
__device__ __forceinline__ uint64_t smem_desc_kmajor(const void* tile)
{
    static_assert(BKT == 32 || BKT == 16, "K block of 16 or 32 FP32");
    if constexpr (BKT == 32)
        return smem_desc_sw128(tile);
    const uint64_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;          // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;         // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                  // fixed constant 0b001
    d |= (uint64_t)4 << 61;                  // swizzle: 64-byte
    return d;
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
        "%27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
        "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
        "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}

template <int SPLIT, int EPI, int BN, int NST>
__global__ void __launch_bounds__(128, 2) tc_gemm_kernel(
    const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
    const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
    TcArgs g)
{
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "MMA N for M = 128");
    constexpr uint32_t A_BYTES = BM * BK * 4;   // 16 KB
    constexpr uint32_t B_BYTES = BN * BK * 4;
    constexpr uint32_t STAGE = (SPLIT == 3 ? 2 : 1) * (A_BYTES + B_BYTES);
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // align the ring to 1024 bytes (swizzle atom)
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base + NST * STAGE);
    uint64_t* empty = full + NST;
    uint64_t* done = empty + NST;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int plane = g.k0 + (int)blockIdx.z * g.kstep;
    const int nkb = (g.K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_d = *tmem_slot;
    pdl_wait();  // operands and u come from the previous kernel

    int issued = 0;  // producer: stages issued (thread 0 only)
    if (warp == 0 && lane == 0) {
        // producer: TMA loads of A and B K-blocks
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % NST;
            if (kb >= NST) {
                if (!mbar_wait_bounded(&empty[s], ((kb / NST) - 1) & 1)) {
                    *abort_flag = 1;
                    break;
                }
            }
            unsigned char* st = base + s * STAGE;
            mbar_arrive_expect_tx(&full[s], STAGE);
            const int kx = kb * BK;
            if (g.a_batched)
                tma_load_3d(st, &mA_hi, &full[s], kx, m0, plane);
            else
                tma_load_2d(st, &mA_hi, &full[s], kx, m0);
            if (SPLIT == 3) {
                if (g.a_batched)
                    tma_load_3d(st + A_BYTES, &mA_lo, &full[s], kx, m0, plane);
                else
                    tma_load_2d(st + A_BYTES, &mA_lo, &full[s], kx, m0);
            }
            unsigned char* sb = st + (SPLIT == 3 ? 2 : 1) * A_BYTES;
            if (g.b_batched)
                tma_load_3d(sb, &mB_hi, &full[s], kx, n0, plane);
            else
                tma_load_2d(sb, &mB_hi, &full[s], kx, n0);
            if (SPLIT == 3) {
                if (g.b_batched)
                    tma_load_3d(sb + B_BYTES, &mB_lo, &full[s], kx, n0, plane);
                else
                    tma_load_2d(sb + B_BYTES, &mB_lo, &full[s], kx, n0);
            }
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_tf32(BN);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % NST;
            if (*abort_flag || !mbar_wait_bounded(&full[s], (kb / NST) & 1)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            unsigned char* st = base + s * STAGE;
            unsigned char* sa_hi = st;
            unsigned char* sa_lo = st + A_BYTES;
            unsigned char* sb_hi = st + (SPLIT == 3 ? 2 : 1) * A_BYTES;
            unsigned char* sb_lo = sb_hi + B_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 8; ++k) {
                // K = 8 TF32 per instruction = 32 bytes along the swizzled row
                const uint64_t ah = smem_desc_sw128(sa_hi) + (uint64_t)((k * 32) >> 4);
                const uint64_t bh = smem_desc_sw128(sb_hi) + (uint64_t)((k * 32) >> 4);
                mma_tf32(tmem_d, ah, bh, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                if (SPLIT == 3) {
                    const uint64_t al = smem_desc_sw128(sa_lo) + (uint64_t)((k * 32) >> 4);
                    const uint64_t bl = smem_desc_sw128(sb_lo) + (uint64_t)((k * 32) >> 4);
                    mma_tf32(tmem_d, ah, bl, idesc, 1u);
                    mma_tf32(tmem_d, al, bh, idesc, 1u);
                }
            }
            mma_commit(&empty[s]);  // slot free once these MMAs have read it
        }
        mma_commit(done);  // accumulator complete (covers every MMA issued above)
    }
    __syncwarp();

    // epilogue: thread t owns output row m0 + t (TMEM lane t)
    const bool ok = mbar_wait_bounded(done, 0);
    tc_fence_after();
    const bool good = __syncthreads_and(ok && !*abort_flag) != 0;
    if (good) {
        // TMEM lane = output row: thread t holds row m0 + t.  Each warp stages its 32 x 32
        // chunk through the (now idle) ring memory so that a warp store covers 32
        // consecutive columns of one row.
        float* tile = reinterpret_cast<float*>(base) + warp * (32 * 33);
        const uint32_t trow = tmem_d + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t r[32];
            tmem_ld32(trow + (uint32_t)(c * 32), r);
#pragma unroll
            for (int q = 0; q < 32; ++q)
                tile[lane * 33 + q] = __uint_as_float(r[q]);
            __syncwarp();
            const int n = n0 + c * 32 + lane;
            const bool nok = n < g.N;
            const int mrow = m0 + warp * 32;
            const long long obase = (long long)plane * g.plane + (long long)mrow * g.N + n;
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                v[i] = tile[i * 33 + lane];
            // issue every row's load before using any, so their latencies overlap
            if (EPI == EPI_SCALE_SPLIT) {
                float sc[32];
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    sc[i] = (nok && mrow + i < g.M)
                                ? __ldg(g.scale + (long long)(mrow + i) * g.N + n)
                                : 0.0f;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    v[i] *= sc[i];
            }
            if (EPI == EPI_UPDATE) {
                float uo[32];
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    uo[i] = (nok && mrow + i < g.M) ? g.u[obase + (long long)i * g.N] : 0.0f;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (nok && mrow + i < g.M)
                        g.uout[obase + (long long)i * g.N] =
                            fmaf(g.omega, v[i], (1.0f - g.omega) * uo[i]);
            } else if (g.out_plain) {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (nok && mrow + i < g.M)
                        g.out_hi[obase + (long long)i * g.N] = v[i];
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (nok && mrow + i < g.M) {
                        const uint32_t hi = tf32_rn(v[i]);
                        g.out_hi[obase + (long long)i * g.N] = __uint_as_float(hi);
                        if (SPLIT == 3)
                            g.out_lo[obase + (long long)i * g.N] =
                                __uint_as_float(tf32_rn(v[i] - __uint_as_float(hi)));
                    }
            }
            __syncwarp();
        }
    } else if (threadIdx.x == 0) {
        set_status(g.status, BRS_ERR_TIMEOUT);
    }
    if (!good && warp == 0 && lane == 0) {
        // drain TMA copies still in flight into this CTA's shared memory
        for (int kb = (issued > NST ? issued - NST : 0); kb < issued; ++kb)
            mbar_wait_bounded(&full[kb % NST], (kb / NST) & 1, 200000000ull);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// EPI_BOX epilogue of one accumulator tile, run by one warp for its 32 TMEM lanes: lane =
// block (row m), each 32-column chunk = 32 consecutive local cells of that block.
//   uout[cell] = (1 - omega) u[cell] + omega D[m][l]
// Lanes are consecutive blocks, so a warp's stores cover whole runs of grid rows.
template <int BN>
__device__ __forceinline__ void box_epilogue(const TcArgs& g, uint32_t trow, int m, int n0)
{
    const bool mok = m < g.M;
    long long base = 0;
    if (mok) {
        const long long pk = g.box_rows[m];
        const long long bi = pk & 0x1FFFFF, bj = (pk >> 21) & 0x1FFFFF, bk = pk >> 42;
        base = bi * g.box_bx + (long long)g.box_nx * (bj * g.box_by + (long long)g.box_ny * bk * g.box_bz);
    }
    const float om = g.omega, om1 = 1.0f - g.omega;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        tmem_ld32(trow + (uint32_t)(c * 32), r);
        const int l0 = n0 + c * 32;
        if (mok && g.box_vec4) {
            long long cell[8];
            float4 uo[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int l = l0 + 4 * v;
                cell[v] = l < g.N ? base + __ldg(g.box_off + l) : -1;
                if (cell[v] >= 0)
                    uo[v] = *reinterpret_cast<const float4*>(g.u + cell[v]);
            }
#pragma unroll
            for (int v = 0; v < 8; ++v)
                if (cell[v] >= 0) {
                    float4 o;
                    o.x = fmaf(om, __uint_as_float(r[4 * v + 0]), om1 * uo[v].x);
                    o.y = fmaf(om, __uint_as_float(r[4 * v + 1]), om1 * uo[v].y);
                    o.z = fmaf(om, __uint_as_float(r[4 * v + 2]), om1 * uo[v].z);
                    o.w = fmaf(om, __uint_as_float(r[4 * v + 3]), om1 * uo[v].w);
                    *reinterpret_cast<float4*>(g.uout + cell[v]) = o;
                }
        } else if (mok) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int l = l0 + i;
                if (l < g.N) {
                    const long long cell = base + __ldg(g.box_off + l);
                    g.uout[cell] = fmaf(om, __uint_as_float(r[i]), om1 * g.u[cell]);
                }
            }
        }
        __syncwarp();  // the next tcgen05.ld is warp-collective
    }
}

// EPI_YTHOMAS epilogue of one accumulator tile: TMEM lane = x-mode p, its N = n columns =
// the right-hand side r along y of tridiag(-ay, d_p, -ay) w = r.  Two warps share each lane
// quarter and split the line at k = n / 2 (twisted elimination):
//   top    (half 0), y = 0 .. k-1 :  z_y = m_y (r_y + ay z_{y-1})
//   bottom (half 1), y = n-1 .. k :  z_y = m_{n-1-y} (r_y + ay z_{y+1})
// with the reciprocal pivots m_j of the elimination from one end (by symmetry the same from
// either end), g.ym[j * M + p].  z is written back to the TMEM columns.  The halves swap
// z_{k-1} and z_k through shared memory; with m = m_{k-1} (= m_{n-1-k}) the interface is
//   w_{k-1} = (z_{k-1} + ay m z_k) / (1 - ay^2 m^2),   w_k = z_k + ay m w_{k-1},
// and each half back-substitutes its own rows:
//   top    y = k-1 .. 0 :  w_y = z_y + ay m_y w_{y+1}
//   bottom y = k .. n-1 :  w_y = z_y + ay m_{n-1-y} w_{y-1}.
// w is stored split (hi, lo) at [plane][y][p]: a warp's store of one y covers 32 consecutive
// modes.  tcgen05.ld / st are warp-collective, so every lane runs the loops; lanes past the
// last mode read mode 0's pivots and store nothing.  xch holds this pair's two 32-value
// exchange slots; pbar (64 arrivals: both warps' lanes) orders them, waited with a bound.
template <int SPLIT>
__device__ __forceinline__ bool ythomas_twist_epilogue(const TcArgs& g, uint32_t trow, int p,
                                                       int plane, int half, float* xch,
                                                       uint64_t* pbar, uint32_t parity)
{
    const int lane = threadIdx.x & 31;
    const bool pok = p < g.M;
    const int n = g.N, k = n >> 1, nck = k >> 4;  // N a multiple of 32: k a multiple of 16
    const float ay = g.ay;
    const long long M = g.M;
    const float* tab = g.ym + (pok ? p : 0);
    auto load_piv = [&](int blk, float (&dst)[16]) {  // m_j, j = 16 blk .. 16 blk + 15
#pragma unroll
        for (int j = 0; j < 16; ++j)
            dst[j] = __ldg(tab + (long long)(blk * 16 + j) * M);
    };
    float mn[16];
    load_piv(0, mn);
    float z = 0.0f;
#pragma unroll 1
    for (int c = 0; c < nck; ++c) {
        float m[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            m[j] = mn[j];
        if (c + 1 < nck)
            load_piv(c + 1, mn);
        uint32_t r[16];
        if (half == 0) {
            const uint32_t col = (uint32_t)(c * 16);
            tmem_ld16(trow + col, r);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                z = m[j] * fmaf(ay, z, __uint_as_float(r[j]));
                r[j] = __float_as_uint(z);
            }
            tmem_st16(trow + col, r);
        } else {
            // columns n - 16(c+1) .. n - 16c - 1, from the highest; column y uses m_{n-1-y}
            const uint32_t col = (uint32_t)(n - 16 * (c + 1));
            tmem_ld16(trow + col, r);
#pragma unroll
            for (int j = 15; j >= 0; --j) {
                z = m[15 - j] * fmaf(ay, z, __uint_as_float(r[j]));
                r[j] = __float_as_uint(z);
            }
            tmem_st16(trow + col, r);
        }
    }
    tmem_wait_st();
    // interface: top publishes z_{k-1}, bottom z_k
    xch[half * 32 + lane] = z;
    mbar_arrive(pbar);
    const bool ok = mbar_wait_bounded(pbar, parity);
    const float zt = xch[lane], zb = xch[32 + lane];
    const float mk = __ldg(tab + (long long)(k - 1) * M);
    const float wk1 = (zt + ay * mk * zb) / (1.0f - ay * ay * mk * mk);
    const float wk = fmaf(ay * mk, wk1, zb);
    float w = half == 0 ? wk : wk1;
    float* oh = g.out_hi + (long long)plane * g.plane + p;
    float* ol = g.out_lo + (long long)plane * g.plane + p;
    // back substitution: chunk order reversed for the top half, pivot blocks reversed for both
    load_piv(nck - 1, mn);
#pragma unroll 1
    for (int c = 0; c < nck; ++c) {
        float m[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            m[j] = mn[j];
        if (c + 1 < nck)
            load_piv(nck - 2 - c, mn);
        uint32_t r[16];
        if (half == 0) {
            // columns 16 b .. 16 b + 15, b = nck-1-c, from the highest; column y uses m_y
            const int y0 = 16 * (nck - 1 - c);
            tmem_ld16(trow + (uint32_t)y0, r);
            float* ph = oh + (long long)y0 * M;
            float* pl = ol + (long long)y0 * M;
#pragma unroll
            for (int j = 15; j >= 0; --j) {
                w = fmaf(ay * m[j], w, __uint_as_float(r[j]));
                if (pok) {
                    const uint32_t hb = tf32_rn(w);
                    ph[j * M] = __uint_as_float(hb);
                    if (SPLIT == 3)
                        pl[j * M] = __uint_as_float(tf32_rn(w - __uint_as_float(hb)));
                }
            }
        } else {
            // columns k + 16 c .. k + 16 c + 15, from the lowest; column y uses m_{n-1-y}, the
            // block b = nck-1-c reversed
            const int y0 = k + 16 * c;
            tmem_ld16(trow + (uint32_t)y0, r);
            float* ph = oh + (long long)y0 * M;
            float* pl = ol + (long long)y0 * M;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                w = fmaf(ay * m[15 - j], w, __uint_as_float(r[j]));
                if (pok) {
                    const uint32_t hb = tf32_rn(w);
                    ph[j * M] = __uint_as_float(hb);
                    if (SPLIT == 3)
                        pl[j * M] = __uint_as_float(tf32_rn(w - __uint_as_float(hb)));
                }
            }
        }
        __syncwarp();  // the next tcgen05.ld is warp-collective
    }
    return ok;
}

// Persistent variant: one CTA per SM walks tiles t = blockIdx.x, +gridDim.x, ... of the
// (n-tile, m-tile, plane) space.  Warp 0 streams K-blocks of every tile through the TMA
// ring, warp 1 issues the MMAs into one of two TMEM accumulators, warps 2-5 drain the other
// accumulator (epilogue of the previous tile) at the same time.  The y elimination epilogue
// has eight epilogue warps (warps 2-9): two per TMEM lane quarter, one per half of the line.
template <int EPI>
__host__ __device__ constexpr int pers_threads()
{
    return EPI == EPI_YGATHER ? 448 : EPI == EPI_YTHOMAS ? 320 : 192;
}

// Ring stage of the gather form: A hi (/ lo) and three B boxes (u_{k-1}, u_{k+1}, b_k), K blocks
// of 16; the stage count fills 192 KB (at most 8).
__host__ __device__ constexpr int gather_stage(int split, int bn)
{
    return ((split == 3 ? 2 : 1) * BM + 3 * bn) * 16 * 4;
}

__host__ __device__ constexpr int gather_nst(int split, int bn)
{
    return 196608 / gather_stage(split, bn) < 8 ? 196608 / gather_stage(split, bn) : 8;
}

// Shared memory past the ring of the y elimination epilogue: four pair barriers, and a
// double-buffered exchange area of 4 pairs x 2 halves x 32 values.
constexpr int kTwistExtra = 4 * 8 + 2 * 4 * 64 * 4;

template <int SPLIT, int EPI, int BN, int NST, int BKT = BK>
__global__ void __launch_bounds__(pers_threads<EPI>(), 1) tc_gemm_persistent(
    const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
    const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
    TcArgs g, int tiles_n, int tiles_m, int nbatch)
{
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "MMA N for M = 128");
    constexpr bool GATHER = EPI == EPI_YGATHER;
    constexpr bool YT = EPI == EPI_YTHOMAS || GATHER;
    static_assert(!GATHER || BKT == 16, "gather form: K blocks of 16");
    constexpr uint32_t A_PARTS = SPLIT == 3 ? 2 : 1;
    constexpr uint32_t A_BYTES = BM * BKT * 4;
    constexpr uint32_t B_BYTES = BN * BKT * 4;
    constexpr uint32_t STAGE =
        GATHER ? A_PARTS * A_BYTES + 3 * B_BYTES : A_PARTS * (A_BYTES + B_BYTES);
    constexpr int EPI_END = YT ? 10 : 6;  // epilogue warps 2 .. EPI_END-1; then converters
    constexpr uint32_t TMEM_COLS = 2 * BN;  // two accumulators
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base + NST * STAGE);
    uint64_t* empty = full + NST;
    uint64_t* accf = empty + NST;  // accumulator a holds a finished tile
    uint64_t* acce = accf + 2;     // accumulator a has been read out
    uint64_t* done = acce + 2;     // every MMA issued by this CTA has completed
    constexpr int NPB = YT ? 4 : 0;
    constexpr int NCV = GATHER ? NST : 0;
    uint64_t* pairb = done + 1;    // y elimination: the two warps of lane quarter q meet here
    uint64_t* conv = pairb + NPB;  // gather form: stage s holds R's split (128 arrivals)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(conv + NCV);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* xbase = reinterpret_cast<float*>(conv + NCV + 1);  // [2][4][2][32]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = (g.K + BKT - 1) / BKT;
    const long long ntiles = (long long)tiles_n * tiles_m * nbatch;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], YT ? 8 : 4);
        }
        for (int q = 0; q < NPB; ++q)
            mbar_init(&pairb[q], 64);
        for (int q = 0; q < NCV; ++q)
            mbar_init(&conv[q], 128);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    pdl_wait();  // operands and u come from the previous kernel

    auto decode = [&](long long t, int* m0, int* n0, int* plane) {
        const int tn = (int)(t % tiles_n);
        const long long r = t / tiles_n;
        const int tm = (int)(r % tiles_m);
        const int b = (int)(r / tiles_m);
        *n0 = tn * BN;
        *m0 = tm * BM;
        *plane = g.k0 + b * g.kstep;
    };

    long long issued = 0;  // producer: K-blocks issued (thread 0)
    if (warp == 0 && lane == 0) {
        long long kg = 0;
        for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
            int m0, n0, plane;
            decode(t, &m0, &n0, &plane);
            for (int kb = 0; kb < nkb; ++kb, ++kg) {
                const int s = (int)(kg % NST);
                if (kg >= NST && !mbar_wait_bounded(&empty[s], (uint32_t)(((kg / NST) - 1) & 1))) {
                    *abort_flag = 1;
                    break;
                }
                unsigned char* st = base + s * STAGE;
                mbar_arrive_expect_tx(&full[s], STAGE);
                const int kx = kb * BKT;
                if (g.a_batched)
                    tma_load_3d(st, &mA_hi, &full[s], kx, m0, plane);
                else
                    tma_load_2d(st, &mA_hi, &full[s], kx, m0);
                if (SPLIT == 3) {
                    if (g.a_batched)
                        tma_load_3d(st + A_BYTES, &mA_lo, &full[s], kx, m0, plane);
                    else
                        tma_load_2d(st + A_BYTES, &mA_lo, &full[s], kx, m0);
                }
                unsigned char* sb = st + A_PARTS * A_BYTES;
                if constexpr (GATHER) {
                    tma_load_3d(sb, &mB_hi, &full[s], kx, n0, plane - 1);
                    tma_load_3d(sb + B_BYTES, &mB_hi, &full[s], kx, n0, plane + 1);
                    tma_load_3d(sb + 2 * B_BYTES, &mB_lo, &full[s], kx, n0, plane);
                } else if (g.b_batched)
                    tma_load_3d(sb, &mB_hi, &full[s], kx, n0, plane);
                else
                    tma_load_2d(sb, &mB_hi, &full[s], kx, n0);
                if (SPLIT == 3 && !GATHER) {
                    if (g.b_batched)
                        tma_load_3d(sb + B_BYTES, &mB_lo, &full[s], kx, n0, plane);
                    else
                        tma_load_2d(sb + B_BYTES, &mB_lo, &full[s], kx, n0);
                }
                issued = kg + 1;
            }
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_tf32(BN);
        long long kg = 0;
        int ti = 0;
        for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++ti) {
            const int a = ti & 1;
            if (ti >= 2 && !mbar_wait_bounded(&acce[a], (uint32_t)(((ti >> 1) - 1) & 1))) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t tacc = tmem_base + (uint32_t)(a * BN);
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb, ++kg) {
                const int s = (int)(kg % NST);
                uint64_t* ready = GATHER ? &conv[s] : &full[s];
                if (*abort_flag || !mbar_wait_bounded(ready, (uint32_t)((kg / NST) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                unsigned char* st = base + s * STAGE;
                unsigned char* sa_hi = st;
                unsigned char* sa_lo = st + A_BYTES;
                // gather form: the split of R is in the b_k (hi) and u_{k-1} (lo) boxes
                unsigned char* sb_hi = st + A_PARTS * A_BYTES + (GATHER ? 2 * B_BYTES : 0);
                unsigned char* sb_lo = GATHER ? st + A_PARTS * A_BYTES : sb_hi + B_BYTES;
#pragma unroll
                for (int k = 0; k < BKT / 8; ++k) {
                    const uint64_t ah = smem_desc_kmajor<BKT>(sa_hi) + (uint64_t)((k * 32) >> 4);
                    const uint64_t bh = smem_desc_kmajor<BKT>(sb_hi) + (uint64_t)((k * 32) >> 4);
                    mma_tf32(tacc, ah, bh, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    if (SPLIT == 3) {
                        const uint64_t al = smem_desc_kmajor<BKT>(sa_lo) + (uint64_t)((k * 32) >> 4);
                        const uint64_t bl = smem_desc_kmajor<BKT>(sb_lo) + (uint64_t)((k * 32) >> 4);
                        mma_tf32(tacc, ah, bl, idesc, 1u);
                        mma_tf32(tacc, al, bh, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
            }
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            mma_commit(&accf[a]);
        }
        mma_commit(done);
    } else if (GATHER && warp >= EPI_END) {
        // converters: R = b_k + az (u_{k-1} + u_{k+1}) element by element (the three boxes
        // share one swizzled layout), hi = rn_tf32(R) over b_k's box, lo = rn_tf32(R - hi) over
        // u_{k-1}'s; the async-proxy fence makes the writes visible to the MMAs
        const int ct = threadIdx.x - 32 * EPI_END;
        const float az = g.az;
        long long kg = 0;
        bool run = true;
        for (long long t = blockIdx.x; t < ntiles && run; t += gridDim.x) {
            for (int kb = 0; kb < nkb; ++kb, ++kg) {
                const int s = (int)(kg % NST);
                if (!mbar_wait_bounded(&full[s], (uint32_t)((kg / NST) & 1)) || *abort_flag) {
                    *abort_flag = 1;
                    run = false;
                    break;
                }
                unsigned char* sb = base + s * STAGE + A_PARTS * A_BYTES;
                float4* um = reinterpret_cast<float4*>(sb);
                const float4* up = reinterpret_cast<const float4*>(sb + B_BYTES);
                float4* bb = reinterpret_cast<float4*>(sb + 2 * B_BYTES);
#pragma unroll 2
                for (int i = ct; i < (int)(B_BYTES / 16); i += 128) {
                    const float4 x = um[i], y = up[i], b4 = bb[i];
                    float r[4] = {fmaf(az, x.x + y.x, b4.x), fmaf(az, x.y + y.y, b4.y),
                                  fmaf(az, x.z + y.z, b4.z), fmaf(az, x.w + y.w, b4.w)};
                    float h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        h[e] = __uint_as_float(tf32_rn(r[e]));
                        l[e] = __uint_as_float(tf32_rn(r[e] - h[e]));
                    }
                    bb[i] = make_float4(h[0], h[1], h[2], h[3]);
                    if (SPLIT == 3)
                        um[i] = make_float4(l[0], l[1], l[2], l[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&conv[s]);
            }
        }
    } else if (warp >= 2 && warp < EPI_END) {
        // epilogue: this warp reads TMEM lanes 32*(warp % 4) .. +31 = tile rows
        const int q = warp & 3;
        int ti = 0;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++ti) {
            const int a = ti & 1;
            const bool ok = mbar_wait_bounded(&accf[a], (uint32_t)((ti >> 1) & 1));
            if (__any_sync(0xffffffffu, !ok || *abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            int m0, n0, plane;
            decode(t, &m0, &n0, &plane);
            const uint32_t trow = tmem_base + (uint32_t)(a * BN) + ((uint32_t)(q * 32) << 16);
            if constexpr (EPI == EPI_BOX) {
                box_epilogue<BN>(g, trow, m0 + q * 32 + lane, n0);
            } else if constexpr (YT) {
                const int half = (warp - 2) >> 2;
                float* xch = xbase + ((ti & 1) * 4 + q) * 64;
                if (!ythomas_twist_epilogue<SPLIT>(g, trow, m0 + q * 32 + lane, plane, half, xch,
                                                   &pairb[q], (uint32_t)(ti & 1)))
                    *abort_flag = 1;
            } else {
            // Row-direct epilogue: this thread's TMEM lane is output row mrow; a 32-column
            // chunk of it is 128 contiguous bytes, written (and, for the update, the old u
            // read) as eight 16-byte vectors.  N is a multiple of 32 on this path, so a chunk
            // lies inside the row or wholly past it.  The old u of the next chunk is loaded
            // while the current one is processed.
            const int mrow = m0 + q * 32 + lane;
            const bool mok = mrow < g.M;
            const long long rbase = (long long)plane * g.plane + (long long)mrow * g.N;
            float4 unext[8];
            auto load_u = [&](int c, float4 (&dst)[8]) {
                const int n = n0 + c * 32;
                if (mok && n < g.N) {
                    const float4* src = reinterpret_cast<const float4*>(g.u + rbase + n);
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        dst[v] = src[v];
                }
            };
            if (EPI == EPI_UPDATE)
                load_u(0, unext);
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                float4 ucur[8];
                if (EPI == EPI_UPDATE) {
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        ucur[v] = unext[v];
                    if (c + 1 < BN / 32)
                        load_u(c + 1, unext);
                }
                uint32_t r[32];
                tmem_ld32(trow + (uint32_t)(c * 32), r);  // warp-collective: every lane
                const int n = n0 + c * 32;
                if (mok && n < g.N) {
                    const long long o = rbase + n;
                    float v[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        v[i] = __uint_as_float(r[i]);
                    if (EPI == EPI_SCALE_SPLIT) {
                        const float4* sc4 =
                            reinterpret_cast<const float4*>(g.scale + (long long)mrow * g.N + n);
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            const float4 sc = __ldg(sc4 + w);
                            v[4 * w + 0] *= sc.x;
                            v[4 * w + 1] *= sc.y;
                            v[4 * w + 2] *= sc.z;
                            v[4 * w + 3] *= sc.w;
                        }
                    }
                    if (EPI == EPI_UPDATE) {
                        const float om = g.omega, om1 = 1.0f - g.omega;
                        float4* dst = reinterpret_cast<float4*>(g.uout + o);
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            float4 out;
                            out.x = fmaf(om, v[4 * w + 0], om1 * ucur[w].x);
                            out.y = fmaf(om, v[4 * w + 1], om1 * ucur[w].y);
                            out.z = fmaf(om, v[4 * w + 2], om1 * ucur[w].z);
                            out.w = fmaf(om, v[4 * w + 3], om1 * ucur[w].w);
                            dst[w] = out;
                        }
                    } else if (g.out_plain) {
                        float4* dst = reinterpret_cast<float4*>(g.out_hi + o);
#pragma unroll
                        for (int w = 0; w < 8; ++w)
                            dst[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2],
                                                 v[4 * w + 3]);
                    } else {
                        float hi[32], lo[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const uint32_t hb = tf32_rn(v[i]);
                            hi[i] = __uint_as_float(hb);
                            lo[i] = __uint_as_float(tf32_rn(v[i] - hi[i]));
                        }
                        float4* dh = reinterpret_cast<float4*>(g.out_hi + o);
#pragma unroll
                        for (int w = 0; w < 8; ++w)
                            dh[w] = make_float4(hi[4 * w], hi[4 * w + 1], hi[4 * w + 2],
                                                hi[4 * w + 3]);
                        if (SPLIT == 3) {
                            float4* dl = reinterpret_cast<float4*>(g.out_lo + o);
#pragma unroll
                            for (int w = 0; w < 8; ++w)
                                dl[w] = make_float4(lo[4 * w], lo[4 * w + 1], lo[4 * w + 2],
                                                    lo[4 * w + 3]);
                        }
                    }
                }
                __syncwarp();
            }
            }  // EPI != EPI_BOX
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&acce[a]);
        }
    }
    __syncwarp();
    // every MMA of this CTA has completed before TMEM is released; TMA copies still in
    // flight (abort only) are drained by the producer
    const bool fin = mbar_wait_bounded(done, 0);
    if (warp == 0 && lane == 0 && (*abort_flag || !fin)) {
        set_status(g.status, BRS_ERR_TIMEOUT);
        for (long long kg = (issued > NST ? issued - NST : 0); kg < issued; ++kg)
            mbar_wait_bounded(&full[kg % NST], (uint32_t)((kg / NST) & 1), 200000000ull);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

#endif  // __CUDACC__

}  // namespace brs_tc
