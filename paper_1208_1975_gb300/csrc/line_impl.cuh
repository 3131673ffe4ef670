// x-line block relaxation kernels (Sec. 2, Alg. 1 / Alg. 2 with full x-line blocks).
//
// For one line (j,k) the sweep gathers the off-block neighbours into the block
// right-hand side and solves the line block exactly:
//   rhs_i = b_ijk + ay (u_{i,j-1,k} + u_{i,j+1,k}) + az (u_{i,j,k-1} + u_{i,j,k+1})
//   M_line x = rhs,   M_line = tridiag(-ax, d, -ax),  d = 2(ax+ay+az)
//   new u = (1-omega) u + omega x
// which equals u + omega M^{-1}(b - A u) (Eq. blockiteration2) in exact arithmetic.
//
// Because the coefficients are constant, the LU pivots of M_line are the same for every
// line; the host computes them once (Sec. 2 / Sec. 4.3: factor once, reuse) in FP64:
//   p_0 = 1/d,  p_i = 1/(d - ax^2 p_{i-1})
// With z_i = rhs_i + c_i z_{i-1}  (c_i = ax p_{i-1}),      forward elimination
//      w_i = z_i + e_i w_{i+1}    (e_i = ax p_{i+1}),      back substitution
//      x_i = p_i w_i
// every step is one FMA.  A line is spread over G lanes (E cells each); the forward and
// backward first-order recurrences are solved across lanes with an affine scan (each
// lane's chunk is the map z_end = A z_in + B with a constant A = product of its c_i).
//
// Two kernels:
//  * line_tma_kernel -- persistent CTAs march in +z over a tile of JT lines; planes of
//    u (JT+2 rows incl. the j-1 / j+JT halo) and b (JT rows) are staged in a shared
//    memory ring by 3D TMA loads whose out-of-range rows/planes read as zero, which is
//    exactly the homogeneous Dirichlet boundary.  u(j,k-1), u(j,k) stay in registers.
//  * line_plain_kernel -- one group per line, direct global loads; any nx.
#pragma once

#include "brs_internal.cuh"

namespace brs {

// Line factor tables (context dtype), padded to NP = G*E entries:
//   [0, NP)        c_i   forward multipliers (0 beyond nx)
//   [NP, 2NP)      e_i   backward multipliers (0 at nx-1 and beyond)
//   [2NP, 3NP)     omega * p_i (0 beyond nx)
//   [3NP, 3NP+G*LG)       forward scan multipliers, step t at [t*G + lane]
//   [3NP+G*LG, 3NP+2G*LG) backward scan multipliers
//   [3NP+2G*LG, 4NP+2G*LG) p_i (0 beyond nx)
template <int G>
struct Log2 {
    static constexpr int value = (G <= 1) ? 0 : 1 + Log2<G / 2>::value;
};

template <typename T, int E, int G>
struct LineTables {
    static constexpr int LG = Log2<G>::value;
    T c[E], e[E], wp[E];
    T af[LG > 0 ? LG : 1], ab[LG > 0 ? LG : 1];

    __device__ __forceinline__ void load(const T* __restrict__ tab, int lane)
    {
        constexpr int NP = G * E;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            c[q] = tab[lane * E + q];
            e[q] = tab[NP + lane * E + q];
            wp[q] = tab[2 * NP + lane * E + q];
        }
#pragma unroll
        for (int t = 0; t < LG; ++t) {
            af[t] = tab[3 * NP + t * G + lane];
            ab[t] = tab[3 * NP + LG * G + t * G + lane];
        }
    }
};

// Solve M_line x = rhs for one line held by G lanes (E cells each, in r[]).
// On return r[q] holds w_i (x_i = p_i w_i; the caller folds p_i into the update).
template <typename T, int E, int G>
__device__ __forceinline__ void line_solve(T (&r)[E], const LineTables<T, E, G>& tb, int lane)
{
    constexpr int LG = Log2<G>::value;
    // forward: chunk summary with zero carry-in
    T z = T(0);
#pragma unroll
    for (int q = 0; q < E; ++q)
        z = fma(tb.c[q], z, r[q]);
    T B = z;
#pragma unroll
    for (int t = 0; t < LG; ++t) {
        const int d = 1 << t;
        T Bp = __shfl_up_sync(0xffffffffu, B, d, G);
        if (lane >= d)
            B = fma(tb.af[t], Bp, B);
    }
    T carry = __shfl_up_sync(0xffffffffu, B, 1, G);
    if (lane == 0)
        carry = T(0);
    z = carry;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        z = fma(tb.c[q], z, r[q]);
        r[q] = z;
    }
    // backward: chunk summary with zero carry-in from the right
    T w = T(0);
#pragma unroll
    for (int q = E - 1; q >= 0; --q)
        w = fma(tb.e[q], w, r[q]);
    B = w;
#pragma unroll
    for (int t = 0; t < LG; ++t) {
        const int d = 1 << t;
        T Bn = __shfl_down_sync(0xffffffffu, B, d, G);
        if (lane + d < G)
            B = fma(tb.ab[t], Bn, B);
    }
    carry = __shfl_down_sync(0xffffffffu, B, 1, G);
    if (lane == G - 1)
        carry = T(0);
    w = carry;
#pragma unroll
    for (int q = E - 1; q >= 0; --q) {
        w = fma(tb.e[q], w, r[q]);
        r[q] = w;
    }
}

// Two-warp form for lines of up to 512 cells (tables of scan_pair_fill): 64 lanes of 8
// cells, the line's first 256 cells in lanes 0-31 of one warp and the rest in lanes 32-63
// of the next.  Each warp scans its half as line_solve does; the forward carry of the lower
// half's last cell and the backward carry of the upper half's first cell cross through
// shared memory (xch, two values per line) at a barrier of the line's 64 threads.  Every
// other lane's carry is its half-local scan value plus the crossing carry times the product
// of the multipliers in between (pf, pb): 5 scan steps per direction instead of the 4 cells
// x 32 lanes form's 16-cell chunks, at 8 cells per lane.
template <typename T>
struct PairTables {
    static constexpr int E = 8, NP = 512, L = 64, LG = 5;
    T c[E], e[E], wp[E];
    T af[LG], ab[LG];
    T pf, pb;

    __device__ __forceinline__ void load(const T* __restrict__ tab, int lane64)
    {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            c[q] = tab[lane64 * E + q];
            e[q] = tab[NP + lane64 * E + q];
            wp[q] = tab[2 * NP + lane64 * E + q];
        }
#pragma unroll
        for (int t = 0; t < LG; ++t) {
            af[t] = tab[3 * NP + t * L + lane64];
            ab[t] = tab[3 * NP + LG * L + t * L + lane64];
        }
        pf = tab[3 * NP + 2 * LG * L + lane64];
        pb = tab[3 * NP + 2 * LG * L + L + lane64];
    }
};

// the factor tables a line group of G lanes with E cells each reads
template <typename T, int E, int G>
struct SolveTables {
    using type = LineTables<T, E, G>;
};
template <typename T>
struct SolveTables<T, 8, 64> {
    using type = PairTables<T>;
};

// Named barrier `id` (1-4: the lines of a two-warp tile) of 64 threads; the immediate ids
// let ptxas reserve only the barriers in use.
__device__ __forceinline__ void bar_sync_64(int id)
{
    switch (id) {
    case 1: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
    case 3: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    }
}

// Solve M_line x = rhs for one line held by the 64 lanes of two warps (lane64 = 0..63);
// on return r[q] holds w_i as for line_solve.  bar: the named barrier of this line's
// 64 threads (1..4); xch: this line's two exchange slots.
template <typename T>
__device__ __forceinline__ void line_solve_pair(T (&r)[8], const PairTables<T>& tb, int lane64,
                                                T* xch, int bar)
{
    constexpr int E = 8, LG = 5;
    const int half = lane64 >> 5, lane = lane64 & 31;
    // forward: half-local inclusive scan of the chunk summaries
    T z = T(0);
#pragma unroll
    for (int q = 0; q < E; ++q)
        z = fma(tb.c[q], z, r[q]);
    T B = z;
#pragma unroll
    for (int t = 0; t < LG; ++t) {
        const int d = 1 << t;
        const T Bp = __shfl_up_sync(0xffffffffu, B, d);
        if (lane >= d)
            B = fma(tb.af[t], Bp, B);
    }
    if (half == 0 && lane == 31)
        xch[0] = B;
    bar_sync_64(bar);
    const T C = half ? xch[0] : T(0);  // z of the lower half's last cell
    T carry = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0)
        carry = T(0);
    z = fma(tb.pf, C, carry);
#pragma unroll
    for (int q = 0; q < E; ++q) {
        z = fma(tb.c[q], z, r[q]);
        r[q] = z;
    }
    // backward, mirrored
    T w = T(0);
#pragma unroll
    for (int q = E - 1; q >= 0; --q)
        w = fma(tb.e[q], w, r[q]);
    B = w;
#pragma unroll
    for (int t = 0; t < LG; ++t) {
        const int d = 1 << t;
        const T Bn = __shfl_down_sync(0xffffffffu, B, d);
        if (lane + d < 32)
            B = fma(tb.ab[t], Bn, B);
    }
    if (half == 1 && lane == 0)
        xch[1] = B;
    bar_sync_64(bar);
    const T D = half ? T(0) : xch[1];  // w of the upper half's first cell
    carry = __shfl_down_sync(0xffffffffu, B, 1);
    if (lane == 31)
        carry = T(0);
    w = fma(tb.pb, D, carry);
#pragma unroll
    for (int q = E - 1; q >= 0; --q) {
        w = fma(tb.e[q], w, r[q]);
        r[q] = w;
    }
}

// 16-byte vector with the element type T (loads and stores through it keep T arrays in
// registers; a vector of another element type would force them into local memory).
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
};
template <>
struct Vec16<double> {
    using type = double2;
};

// Vector helpers: E consecutive elements, 16-byte chunks.
template <typename T, int E>
__device__ __forceinline__ void ld_shared_vec(T (&v)[E], const T* p)
{
    static_assert((E * sizeof(T)) % 16 == 0, "chunk must be whole 16-byte vectors");
    using V = typename Vec16<T>::type;  // same element type: v stays in registers
    const V* s = reinterpret_cast<const V*>(p);
#pragma unroll
    for (int m = 0; m < (int)(E * sizeof(T) / 16); ++m) {
        V f = s[m];
        reinterpret_cast<V*>(v)[m] = f;
    }
}

// Same as ld_shared_vec, but conflict-free when the lanes of a quarter-warp read adjacent
// 32-byte chunks of one row: lane l starts at 16-byte half (l >> 2) & 1 of its chunk, so the
// 8 lanes of each 128-bit access phase cover all 32 banks.
template <typename T, int E>
__device__ __forceinline__ void ld_shared_vec_rot(T (&v)[E], const T* p, int lane)
{
    constexpr int C = (int)(E * sizeof(T) / 16);
    if constexpr (C == 2) {
        using V = typename Vec16<T>::type;
        const V* s = reinterpret_cast<const V*>(p);
        const int h = (lane >> 2) & 1;
        const V f0 = s[h], f1 = s[h ^ 1];
        reinterpret_cast<V*>(v)[0] = h ? f1 : f0;
        reinterpret_cast<V*>(v)[1] = h ? f0 : f1;
    } else {
        ld_shared_vec<T, E>(v, p);
    }
}

// Measured on the 256^3 FP32 workload (same-box A/B): conflict-free row reads with two
// CTAs per SM (128 registers, 6-stage ring) are fastest; three CTAs per SM cap registers
// at 80 and spill, and a one-CTA minimum lets ptxas grow past 128 registers.
#ifndef BRS_LINE_ROT
#define BRS_LINE_ROT 1
#endif
#ifndef BRS_LINE_MINB
#define BRS_LINE_MINB 2
#endif

template <typename T, int E>
__device__ __forceinline__ void ld_row(T (&v)[E], const T* p, int lane)
{
    if (BRS_LINE_ROT)
        ld_shared_vec_rot<T, E>(v, p, lane);
    else
        ld_shared_vec<T, E>(v, p);
}

template <typename T, int E>
__device__ __forceinline__ void st_global_vec(T* p, const T (&v)[E])
{
    using V = typename Vec16<T>::type;
    V* d = reinterpret_cast<V*>(p);
#pragma unroll
    for (int m = 0; m < (int)(E * sizeof(T) / 16); ++m)
        d[m] = reinterpret_cast<const V*>(v)[m];
}

// ---------------------------------------------------------------------------------------
// TMA ring kernel.
//
// Work split: plane-steps are numbered L = jt * nz + k (jt = y tile); CTA c owns the
// contiguous range [c*total/grid, (c+1)*total/grid), i.e. one or a few "segments"
// (jt, k_begin, k_end) that it marches through in +z.  For a segment of n planes the
// ring receives n+2 stages: stage t holds the u rows j0-1..j0+JT of plane k_begin-1+t
// and (t >= 2) the b rows j0..j0+JT-1 of plane k_begin-2+t.  Step s (plane k_begin+s)
// reads stage s+1 (u(k) and its y neighbours) and stage s+2 (u(k+1), b(k)); u(k-1) and
// u(k) come from registers after the first step.
struct SegIter {
    long long L, L1;
    long long nz;
    int jt, kb, n;  // current segment
    __device__ __forceinline__ bool next()
    {
        if (L >= L1)
            return false;
        jt = (int)(L / nz);
        kb = (int)(L - (long long)jt * nz);
        long long rem = L1 - L;
        long long room = nz - kb;
        n = (int)(rem < room ? rem : room);
        L += n;
        return true;
    }
};

template <typename T, int E, int G, bool GS>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && E <= 8) ? BRS_LINE_MINB : 1) line_tma_kernel(const __grid_constant__ CUtensorMap tm_u,
                                                       const __grid_constant__ CUtensorMap tm_b,
                                                       T* __restrict__ out,
                                                       const T* __restrict__ tab, LineArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int JT = a.JT, NS = a.NS, bx = a.bx, pieces = a.pieces;
    const int urows = JT + 2;
    // every TMA box lands on a 128-byte boundary
    const size_t ubox = (((size_t)urows * bx * sizeof(T) + 127) & ~size_t(127)) / sizeof(T);
    const size_t bbox = (((size_t)JT * bx * sizeof(T) + 127) & ~size_t(127)) / sizeof(T);
    const size_t u_elems = (size_t)pieces * ubox;  // u part of a slot (elements)
    const size_t slot_bytes = (u_elems + (size_t)pieces * bbox) * sizeof(T);
    const uint32_t ubytes = (uint32_t)((size_t)pieces * urows * bx * sizeof(T));
    const uint32_t bbytes = (uint32_t)((size_t)pieces * JT * bx * sizeof(T));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NS * slot_bytes);

    const int tid = threadIdx.x;
    const int g = tid / G;      // line within the tile
    const int lane = tid % G;   // lane within the line group
    const int x0 = lane * E;    // first cell of this lane
    const bool xin = x0 < a.nx; // nx % E == 0 on this path: chunks are full or empty
    const int piece = xin ? x0 / bx : 0;
    const int xo = x0 - piece * bx;

    typename SolveTables<T, E, G>::type tb;
    tb.load(tab, lane);
    // two-warp lines: this line's exchange slots after the ring barriers, its named barrier
    T* xch = reinterpret_cast<T*>(full + NS) + 2 * g;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s)
            mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const long long L0 = (long long)blockIdx.x * a.total / gridDim.x;
    const long long L1 = (long long)(blockIdx.x + 1) * a.total / gridDim.x;
    auto slot_ptr = [&](int slot) -> T* {
        return reinterpret_cast<T*>(smem_raw + (uint32_t)slot * (uint32_t)slot_bytes);
    };
    auto inc = [&](int slot) { return slot + 1 == NS ? 0 : slot + 1; };

    // Producer state (thread 0).  Stage indices are per CTA and fit in 32 bits; ring
    // slots advance incrementally (no division on the hot path).
    SegIter pit{L0, L1, a.nz, 0, 0, 0};
    int p_next = 0, p_slot = 0;   // next stage to issue and its slot
    int p_seg_base = 0, p_end = 0;
    bool p_has = false;
    int b_pre = 0;                // stages [0, b_pre) had their b rows requested early
    auto issue = [&](int limit) {
        while (true) {
            if (!p_has || p_next >= p_end) {
                if (p_has)
                    p_seg_base = p_end;
                p_has = pit.next();
                if (!p_has)
                    return;
                p_end = p_seg_base + pit.n + 2;
            }
            if (p_next >= limit)
                return;
            const int t = p_next - p_seg_base;
            T* dst = slot_ptr(p_slot);
            uint64_t* bar = &full[p_slot];
            const bool with_b = t >= 2;
            const bool pre = p_next < b_pre;  // b rows already requested (see below)
            if (!pre)
                mbar_arrive_expect_tx(bar, ubytes + (with_b ? bbytes : 0u));
            const int j0 = pit.jt * JT;
            const int ku = pit.kb - 1 + t;
            for (int pc = 0; pc < pieces; ++pc)
                tma_load_3d(dst + (size_t)pc * ubox, &tm_u, bar, pc * bx, j0 - 1, ku);
            if (with_b && !pre) {
                T* bdst = dst + u_elems;
                for (int pc = 0; pc < pieces; ++pc)
                    tma_load_3d(bdst + (size_t)pc * bbox, &tm_b, bar, pc * bx, j0, ku - 1);
            }
            ++p_next;
            p_slot = inc(p_slot);
        }
    };
    // Launched as a programmatic dependent of the previous sweep: everything above (the
    // constant factor tables, barrier set-up) overlaps that sweep's tail, and so do the
    // b rows of the first ring stages (b is read only, for every sweep).  The previous grid
    // must have completed before this one reads u or writes the output buffer; a stage's
    // barrier expects its u and b bytes together, so no step starts before its u arrives.
    // The next sweep may be scheduled as soon as this grid's CTAs begin to retire.
    if (tid == 0) {
        SegIter it = pit;
        int seg_base = 0, end = 0, slot = 0;
        bool has = false;
        while (b_pre < NS) {
            if (!has || b_pre >= end) {
                if (has)
                    seg_base = end;
                has = it.next();
                if (!has)
                    break;
                end = seg_base + it.n + 2;
            }
            const int t = b_pre - seg_base;
            uint64_t* bar = &full[slot];
            const bool with_b = t >= 2;
            mbar_arrive_expect_tx(bar, ubytes + (with_b ? bbytes : 0u));
            if (with_b) {
                T* bdst = slot_ptr(slot) + u_elems;
                for (int pc = 0; pc < pieces; ++pc)
                    tma_load_3d(bdst + (size_t)pc * bbox, &tm_b, bar, pc * bx, it.jt * JT,
                                it.kb - 2 + t);
            }
            ++b_pre;
            slot = inc(slot);
        }
    }
    pdl_wait_trigger();
    if (tid == 0)
        issue(NS);

    SegIter cit{L0, L1, a.nz, 0, 0, 0};
    int c_base = 0;               // stage 0 of the consumer's segment
    int cs_slot = 0;              // slot of stage c_base + s
    int waited = 0, w_slot = 0;   // stages [0, waited) have completed; slot of `waited`
    uint32_t w_phase = 0;         // parity of the ring pass `waited` is in
    bool failed = false;

    const T ay = (T)a.ay, az = (T)a.az, om1 = (T)a.om1;
    T um[E], uc[E], up[E], r[E];
    const uint32_t urow_off = (uint32_t)(piece * ubox + xo);
    const uint32_t brow_off = (uint32_t)(u_elems + piece * bbox + g * bx + xo);

    while (cit.next()) {
        const int j = cit.jt * JT + g;
        const bool jin = j < a.ny;
        T* outp = out + ((size_t)cit.kb * a.ny + j) * a.nx + x0;
        const size_t plane = (size_t)a.ny * a.nx;
        for (int s = 0; s < cit.n; ++s) {
            // wait for stages up to c_base + s + 2
            const int need = c_base + s + 3;
            bool ok = true;
            while (waited < need && ok) {
                ok = mbar_wait_bounded(&full[w_slot], w_phase);
                if (ok) {
                    ++waited;
                    w_slot = inc(w_slot);
                    if (w_slot == 0)
                        w_phase ^= 1u;
                }
            }
            // the solve shuffles across the warp: skip it warp-uniformly on a timeout (and,
            // for two-warp lines, whose halves meet at a barrier, CTA-uniformly)
            if constexpr (G == 64)
                ok = __syncthreads_and(ok) != 0;
            else
                ok = __all_sync(0xffffffffu, ok);
            const int s1 = inc(cs_slot), s2 = inc(s1);
            if (ok) {
                const T* st1 = slot_ptr(s1);
                const T* st2 = slot_ptr(s2);
                if (xin) {
                    if (s == 0) {
                        ld_row<T, E>(um, slot_ptr(cs_slot) + urow_off + (g + 1) * bx, lane);
                        ld_row<T, E>(uc, st1 + urow_off + (g + 1) * bx, lane);
                    }
                    ld_row<T, E>(up, st2 + urow_off + (g + 1) * bx, lane);
                    T un[E], us[E], bb[E];
                    ld_row<T, E>(un, st1 + urow_off + g * bx, lane);
                    ld_row<T, E>(us, st1 + urow_off + (g + 2) * bx, lane);
                    ld_row<T, E>(bb, st2 + brow_off, lane);
#pragma unroll
                    for (int q = 0; q < E; ++q)
                        r[q] = fma(az, um[q] + up[q], fma(ay, un[q] + us[q], bb[q]));
                } else {
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        r[q] = T(0);
                        um[q] = uc[q] = up[q] = T(0);
                    }
                }
                if constexpr (G == 64)
                    line_solve_pair<T>(r, tb, lane, xch, 1 + g);
                else
                    line_solve<T, E, G>(r, tb, lane);
                T v[E];
#pragma unroll
                for (int q = 0; q < E; ++q)
                    v[q] = fma(tb.wp[q], r[q], om1 * uc[q]);
                if (xin && jin)
                    st_global_vec<T, E>(outp, v);
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    um[q] = GS ? v[q] : uc[q];
                    uc[q] = up[q];
                }
            }
            outp += plane;
            cs_slot = s1;
            failed = __syncthreads_or(!ok) != 0;
            if (failed)
                break;
            if (tid == 0) {
                // stages below the first one the next step needs are free
                const int next_first = (s + 1 < cit.n) ? c_base + s + 1 : c_base + cit.n + 2;
                issue(next_first + NS);
            }
        }
        if (failed)
            break;
        c_base += cit.n + 2;
        cs_slot = inc(inc(cs_slot));  // skip the segment's last two stages
    }
    if (failed && tid == 0) {
        set_status(a.status, BRS_ERR_TIMEOUT);
        // drain copies still in flight before the CTA's shared memory is released
        for (int q = waited; q < p_next; ++q) {
            mbar_wait_bounded(&full[w_slot], w_phase, 200000000ull);
            w_slot = inc(w_slot);
            if (w_slot == 0)
                w_phase ^= 1u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Plain kernel: one line group per (j,k), direct global loads, any nx <= G*E.
template <typename T, int E, int G, bool GS>
__global__ void __launch_bounds__(256) line_plain_kernel(const T* uin, T* out,
                                                         const T* __restrict__ b,
                                                         const T* __restrict__ tab, LineArgs a)
{
    const int groups = blockDim.x / G;
    const long long line = (long long)blockIdx.x * groups + threadIdx.x / G;
    const int lane = threadIdx.x % G;
    const long long nlines = (long long)a.ny * a.nz;
    const bool active = line < nlines;  // whole groups share this flag
    const int j = active ? (int)(line % a.ny) : 0;
    const int k = active ? (int)(line / a.ny) : 0;
    LineTables<T, E, G> tb;
    tb.load(tab, lane);
    const T ay = (T)a.ay, az = (T)a.az, om1 = (T)a.om1;
    const size_t plane = (size_t)a.nx * a.ny;
    const size_t base = ((size_t)k * a.ny + j) * a.nx;
    T r[E], uc[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int x = lane * E + q;
        T acc = T(0), ucq = T(0);
        if (active && x < a.nx) {
            const size_t o = base + x;
            T s1 = (j > 0 ? uin[o - a.nx] : T(0)) + (j + 1 < a.ny ? uin[o + a.nx] : T(0));
            T s2 = (k > 0 ? uin[o - plane] : T(0)) + (k + 1 < a.nz ? uin[o + plane] : T(0));
            acc = fma(az, s2, fma(ay, s1, b[o]));
            ucq = uin[o];
        }
        r[q] = acc;
        uc[q] = ucq;
    }
    line_solve<T, E, G>(r, tb, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int x = lane * E + q;
        if (active && x < a.nx)
            out[base + x] = fma(tb.wp[q], r[q], om1 * uc[q]);
    }
}

}  // namespace brs
