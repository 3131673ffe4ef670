// xy-plane block sweeps carried out in the x-sine basis (Sec. 2 with one block per xy-plane).
//
// The orthonormal DST-I matrix S (S = S^T = S^{-1}) diagonalises T_x, S T_x S = diag(s_p),
// and commutes with everything else a plane sweep applies along the other axes: T_y inside
// the block, the z coupling az (u_{k-1} + u_{k+1}) and the damping.  With
//   u^_k[p][y] = sum_x S[p][x] u_k[y][x]        (and b^_k the same way)
// one plane sweep (Jacobi or the two-colour Gauss-Seidel order) is, for every x-mode p on
// its own,
//   u^_k[p][:] <- (1 - omega) u^_k[p][:] + omega M_p^{-1} (b^_k[p][:] + az (u^_{k-1}[p][:] + u^_{k+1}[p][:]))
//   M_p = tridiag(-ay, ax s_p + 2 ay + 2 az, -ay)  along y,
// i.e. the iterates of the plane sweep itself in exact arithmetic.  A call of several sweeps
// therefore transforms b and u once, runs its sweeps as these mode-line sweeps, and
// transforms u back once (plane.cu).  The mode-line sweep is an x-line-style sweep of the
// array u^[k][p][y]: lines along y (contiguous), one row per mode p, planes k, but with
// per-row factor tables (the pivots depend on s_p) and no neighbour rows: the coupling
// between modes is gone.  Like the x-line sweep it is HBM-bound, 3 words per cell.
//
// mode_tma_kernel: persistent CTAs march in +z over a tile of JT consecutive mode rows.
// Ring stage t of a segment (jt, kb, n) holds the u^ rows of plane kb-1+t and, for t >= 2,
// the b^ rows of plane kb-2+t; step s (plane kb+s) reads stage s+1 (u^_k) and s+2
// (u^_{k+1}, b^_k); u^_{k-1} and u^_k come from registers after the first step.  Boxes
// outside the grid (plane -1, plane nz, rows past the last mode) read as zeros: the
// homogeneous Dirichlet boundary in z.
//  * MODE 0: Jacobi, from the input array into another one.
//  * MODE 1: the planes with k % 2 == colour are updated in place; every value they read
//    belongs to the other colour, which this launch does not write, so the result does not
//    depend on the CTAs' order.  Two launches (colour 0, then 1) make one sweep in the order
//    even planes, then odd planes.
//  * MODE 2: the same sweep (even planes, then odd planes from the new even ones) in one
//    launch, from the input array into another one.  A CTA marches over its planes
//    [kb, ke) extended by one plane at each end; at an even plane j it forms the new even
//    plane from the old odd neighbours and then the new odd plane j-1 from the new even
//    planes j-2 and j (the odd plane's b^ + az u^_{j-2} is formed at step j-1 and kept in
//    registers, in the place of the new even plane j-2).  The even planes kb-1 and ke just outside the
//    segment are recomputed from the same old values their owners use, so every CTA sees
//    the same new even planes and the result does not depend on the CTAs' order; 3 words
//    per cell, as for Jacobi.
#include <cstdlib>

#include "line_impl.cuh"
#include "plane.cuh"
#include "thomas_tables.h"

namespace {

struct ModeArgs {
    int ny, nm, nz;        // line length (y), mode rows (p), planes
    int JT, NS, pieces, bx;
    long long total;       // tiles * nz plane-steps
    double az, om1;        // z coefficient, 1 - omega
    int colour;            // MODE 1: the colour updated by this launch
    int tab_len;           // table entries per mode
    int* status;
};

template <typename T, int E, int G, int MODE>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && E <= 8) ? 2 : 1)
    mode_tma_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_b,
                    T* __restrict__ out, const T* __restrict__ tab, ModeArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int JT = a.JT, NS = a.NS, bx = a.bx, pieces = a.pieces;
    // every TMA box lands on a 128-byte boundary
    const size_t box = (((size_t)JT * bx * sizeof(T) + 127) & ~size_t(127)) / sizeof(T);
    const size_t u_elems = (size_t)pieces * box;  // u^ part of a slot; the b^ part follows
    const size_t slot_bytes = 2 * u_elems * sizeof(T);
    const uint32_t rbytes = (uint32_t)((size_t)pieces * JT * bx * sizeof(T));  // one array's rows
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NS * slot_bytes);

    const int tid = threadIdx.x;
    const int g = tid / G;     // row within the tile
    const int lane = tid % G;  // lane within the line group
    const int y0 = lane * E;   // first cell of this lane
    const bool yin = y0 < a.ny;  // ny % E == 0 on this path: chunks are full or empty
    const int piece = yin ? y0 / bx : 0;
    const int yo = y0 - piece * bx;

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
    constexpr bool COLOUR = MODE == 1;
    // stage t of a segment starting at plane kb carries b^ rows (plane kb-2+t) if it is a
    // step's last stage and, for a colour launch, that step's plane is updated
    auto has_b = [&](int t, int kb) {
        return t >= 2 && (!COLOUR || ((kb - 2 + t) & 1) == a.colour);
    };
    // MODE 2 marches over each segment extended by one plane at both ends
    auto next_seg = [&](brs::SegIter& it) {
        const bool ok = it.next();
        if (MODE == 2 && ok) {
            it.kb -= 1;
            it.n += 2;
        }
        return ok;
    };

    // producer state (thread 0); stage indices are per CTA
    brs::SegIter pit{L0, L1, a.nz, 0, 0, 0};
    int p_next = 0, p_slot = 0, p_seg_base = 0, p_end = 0;
    bool p_has = false;
    int b_pre = 0;  // stages [0, b_pre) had their barrier armed and b^ rows requested early
    auto issue = [&](int limit) {
        while (true) {
            if (!p_has || p_next >= p_end) {
                if (p_has)
                    p_seg_base = p_end;
                p_has = next_seg(pit);
                if (!p_has)
                    return;
                p_end = p_seg_base + pit.n + 2;
            }
            if (p_next >= limit)
                return;
            const int t = p_next - p_seg_base;
            T* dst = slot_ptr(p_slot);
            uint64_t* bar = &full[p_slot];
            const bool wb = has_b(t, pit.kb);
            const bool pre = p_next < b_pre;
            if (!pre)
                mbar_arrive_expect_tx(bar, rbytes + (wb ? rbytes : 0u));
            const int j0 = pit.jt * JT;
            const int ku = pit.kb - 1 + t;
            for (int pc = 0; pc < pieces; ++pc)
                tma_load_3d(dst + (size_t)pc * box, &tm_u, bar, pc * bx, j0, ku);
            if (wb && !pre)
                for (int pc = 0; pc < pieces; ++pc)
                    tma_load_3d(dst + u_elems + (size_t)pc * box, &tm_b, bar, pc * bx, j0, ku - 1);
            ++p_next;
            p_slot = inc(p_slot);
        }
    };
    // b^ is read only and was written before the launch that precedes the first sweep of a
    // call, so the first stages' b^ rows are requested before the dependency wait (as in
    // the x-line sweep); u^ is loaded only after it.
    if (tid == 0) {
        brs::SegIter it = pit;
        int seg_base = 0, end = 0, slot = 0;
        bool has = false;
        while (b_pre < NS) {
            if (!has || b_pre >= end) {
                if (has)
                    seg_base = end;
                has = next_seg(it);
                if (!has)
                    break;
                end = seg_base + it.n + 2;
            }
            const int t = b_pre - seg_base;
            const bool wb = has_b(t, it.kb);
            mbar_arrive_expect_tx(&full[slot], rbytes + (wb ? rbytes : 0u));
            if (wb)
                for (int pc = 0; pc < pieces; ++pc)
                    tma_load_3d(slot_ptr(slot) + u_elems + (size_t)pc * box, &tm_b, &full[slot],
                                pc * bx, it.jt * JT, it.kb - 2 + t);
            ++b_pre;
            slot = inc(slot);
        }
    }
    pdl_wait_trigger();
    if (tid == 0)
        issue(NS);

    brs::SegIter cit{L0, L1, a.nz, 0, 0, 0};
    int c_base = 0, cs_slot = 0;
    int waited = 0, w_slot = 0;
    uint32_t w_phase = 0;
    bool failed = false;

    const T az = (T)a.az, om1 = (T)a.om1;
    T um[E], uc[E], up[E], r[E];
    const uint32_t row_off = (uint32_t)(piece * box + g * bx + yo);
    const size_t plane = (size_t)a.nm * a.ny;

    while (next_seg(cit)) {
        const int p = cit.jt * JT + g;
        const bool pin = p < a.nm;
        brs::LineTables<T, E, G> tb;  // this mode's factor tables (omega folded in)
        tb.load(tab + (size_t)(pin ? p : 0) * a.tab_len, lane);
        // planes this CTA writes: the segment (without MODE 2's extension)
        const int kw0 = MODE == 2 ? cit.kb + 1 : cit.kb;
        const int kw1 = MODE == 2 ? cit.kb + cit.n - 1 : cit.kb + cit.n;
        T* const out_row = out + (size_t)p * a.ny + y0;  // plane 0 of this lane's row
        // MODE 2: after an even step the new even plane, after an odd step k the odd plane's
        // right-hand side so far, b^_k + az (new u^_{k-1})
        T carry[E];
#pragma unroll
        for (int q = 0; q < E; ++q)
            carry[q] = T(0);
        for (int s = 0; s < cit.n; ++s) {
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
            ok = __all_sync(0xffffffffu, ok);  // the solve shuffles across the warp
            const int s1 = inc(cs_slot), s2 = inc(s1);
            const int k = cit.kb + s;
            // steps that solve: every plane (Jacobi), this launch's colour (MODE 1), the even
            // planes (MODE 2); uniform over the CTA
            const bool act = MODE == 0 || (MODE == 1 ? (k & 1) == a.colour : (k & 1) == 0);
            if (ok) {
                const T* st2 = slot_ptr(s2);
                T bb[E];
                if (yin) {
                    if (s == 0) {
                        brs::ld_row<T, E>(um, slot_ptr(cs_slot) + row_off, lane);
                        brs::ld_row<T, E>(uc, slot_ptr(s1) + row_off, lane);
                    }
                    brs::ld_row<T, E>(up, st2 + row_off, lane);
                    if (act || MODE == 2)
                        brs::ld_row<T, E>(bb, st2 + u_elems + row_off, lane);
                } else {
#pragma unroll
                    for (int q = 0; q < E; ++q)
                        um[q] = uc[q] = up[q] = bb[q] = T(0);
                }
                if (act) {
                    T v[E];
                    if (MODE == 2 && k >= a.nz) {
                        // the even plane past the grid: the Dirichlet zeros
#pragma unroll
                        for (int q = 0; q < E; ++q)
                            v[q] = T(0);
                    } else {
#pragma unroll
                        for (int q = 0; q < E; ++q)
                            r[q] = fma(az, um[q] + up[q], bb[q]);
                        brs::line_solve<T, E, G>(r, tb, lane);
#pragma unroll
                        for (int q = 0; q < E; ++q)
                            v[q] = fma(tb.wp[q], r[q], om1 * uc[q]);
                    }
                    if (yin && pin && k >= kw0 && k < kw1)
                        brs::st_global_vec<T, E>(out_row + (size_t)k * plane, v);
                    if (MODE == 2) {
                        // the odd plane below, now that both its new even neighbours exist
                        if (k - 1 >= kw0 && k - 1 < kw1) {
#pragma unroll
                            for (int q = 0; q < E; ++q)
                                r[q] = fma(az, v[q], carry[q]);
                            brs::line_solve<T, E, G>(r, tb, lane);
#pragma unroll
                            for (int q = 0; q < E; ++q)
                                r[q] = fma(tb.wp[q], r[q], om1 * um[q]);
                            if (yin && pin)
                                brs::st_global_vec<T, E>(out_row + (size_t)(k - 1) * plane, r);
                        }
#pragma unroll
                        for (int q = 0; q < E; ++q)
                            carry[q] = v[q];
                    }
                } else if (MODE == 2) {
#pragma unroll
                    for (int q = 0; q < E; ++q)
                        carry[q] = fma(az, carry[q], bb[q]);
                }
                // the neighbours of the next steps are old values: Jacobi and MODE 2 read the
                // input array, a colour launch reads only planes of the other colour
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    um[q] = uc[q];
                    uc[q] = up[q];
                }
            }
            cs_slot = s1;
            failed = __syncthreads_or(!ok) != 0;
            if (failed)
                break;
            if (tid == 0) {
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

template <typename T, int MODE>
const void* mode_kernel_for(int E, int G)
{
#define BRS_MODE_CASE(EE, GG)                                                  \
    if (E == EE && G == GG)                                                    \
        return (const void*)mode_tma_kernel<T, EE, GG, MODE>;
    BRS_MODE_CASE(4, 4)
    BRS_MODE_CASE(4, 8)
    BRS_MODE_CASE(4, 16)
    BRS_MODE_CASE(4, 32)
    BRS_MODE_CASE(8, 32)
    BRS_MODE_CASE(12, 32)
    BRS_MODE_CASE(16, 32)
#undef BRS_MODE_CASE
    return nullptr;
}

const void* mode_kernel(int dtype, int mode, int E, int G)
{
    if (dtype == BRS_F64)
        return mode == 0 ? mode_kernel_for<double, 0>(E, G)
             : mode == 1 ? mode_kernel_for<double, 1>(E, G) : mode_kernel_for<double, 2>(E, G);
    return mode == 0 ? mode_kernel_for<float, 0>(E, G)
         : mode == 1 ? mode_kernel_for<float, 1>(E, G) : mode_kernel_for<float, 2>(E, G);
}

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

size_t slot_bytes(const ModeCfg& m, size_t es)
{
    return 2 * (size_t)m.pieces * (((size_t)m.JT * m.bx * es + 127) & ~size_t(127));
}

}  // namespace

int mode_config(int ny, int nm, int nz, int dtype, int device, ModeCfg* out)
{
    ModeCfg m;
    if (!scan_lanes(ny, &m.E, &m.G))
        return BRS_ERR_UNSUPPORTED;
    const size_t es = dtype == BRS_F64 ? 8 : 4;
    m.pieces = (ny + 255) / 256;
    m.bx = ny / m.pieces;
    // TMA rows: 16-byte aligned, whole lane chunks, boxes of <= 256 elements
    if ((ny * es) % 16 != 0 || ny % m.E != 0 || ny % m.pieces != 0 || (m.bx * es) % 16 != 0 ||
        m.bx % m.E != 0 || m.bx > 256)
        return BRS_ERR_UNSUPPORTED;
    const int gpw = 32 / m.G;  // rows per warp
    const bool wide = dtype == BRS_F32 && m.E >= 12;
    int jt = env_int("BRSMOOTH_MODE_JT",
                     (dtype == BRS_F64 && m.E >= 8) ? 4 : wide ? 128 / m.G : 256 / m.G);
    const int nm_round = ((nm + gpw - 1) / gpw) * gpw;
    if (jt > nm_round)
        jt = nm_round;
    jt = ((jt + gpw - 1) / gpw) * gpw;
    if (jt * m.G > 256)
        jt = 256 / m.G;
    m.JT = jt;
    m.NS = env_int("BRSMOOTH_MODE_NS", (dtype == BRS_F64 || wide) ? 4 : 6);
    if (m.NS < 3)
        m.NS = 3;
    while (m.NS > 3 && (size_t)m.NS * (slot_bytes(m, es) + 8) > 227u * 1024u)
        --m.NS;
    m.smem = (size_t)m.NS * slot_bytes(m, es) + (size_t)m.NS * 8;
    m.tab_len = scan_table_len(m.E, m.G, false);
    int occ = 1 << 30;
    for (int mode = 0; mode < 3; ++mode) {
        const void* k = mode_kernel(dtype, mode, m.E, m.G);
        if (!k)
            return BRS_ERR_UNSUPPORTED;
        // the attribute belongs to the kernel, shared by every context: only ever raise it
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < m.smem)
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m.smem);
        int o = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, m.JT * m.G, m.smem);
        if (e != cudaSuccess)
            return brs_cuda_status(e);
        if (o < occ)
            occ = o;
    }
    if (occ < 1)
        return BRS_ERR_UNSUPPORTED;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    m.grid = sms * occ;
    const long long tiles = (nm + m.JT - 1) / m.JT;
    if (m.grid > tiles * nz)
        m.grid = (int)(tiles * nz);
    m.total = tiles * nz;
    m.ny = ny;
    m.nm = nm;
    m.nz = nz;
    m.dtype = dtype;
    *out = m;
    return BRS_OK;
}

int mode_encode_map(const ModeCfg& m, CUtensorMap* map, const void* ptr)
{
    PFN_encode_tiled enc = brs_encoder();
    if (!enc)
        return BRS_ERR_CUDA;
    const size_t es = m.dtype == BRS_F64 ? 8 : 4;
    cuuint64_t gdim[3] = {(cuuint64_t)m.ny, (cuuint64_t)m.nm, (cuuint64_t)m.nz};
    cuuint64_t gstride[2] = {(cuuint64_t)m.ny * es, (cuuint64_t)m.ny * m.nm * es};
    cuuint32_t box[3] = {(cuuint32_t)m.bx, (cuuint32_t)m.JT, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(map,
                     m.dtype == BRS_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     3, const_cast<void*>(ptr), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BRS_OK : BRS_ERR_CUDA;
}

int mode_sweep_launch(const ModeCfg& m, const CUtensorMap* mu, const CUtensorMap* mb, void* out,
                      const void* tab, double az, double omega, int colour, int* status,
                      cudaStream_t s)
{
    // colour: -1 Jacobi, 0 / 1 one colour in place, 2 both colours (zebra order) into out
    const void* k = mode_kernel(m.dtype, colour < 0 ? 0 : colour == 2 ? 2 : 1, m.E, m.G);
    if (!k)
        return BRS_ERR_UNSUPPORTED;
    ModeArgs a{};
    a.ny = m.ny;
    a.nm = m.nm;
    a.nz = m.nz;
    a.JT = m.JT;
    a.NS = m.NS;
    a.pieces = m.pieces;
    a.bx = m.bx;
    a.total = m.total;
    a.az = az;
    a.om1 = 1.0 - omega;
    a.colour = colour == 0 || colour == 1 ? colour : 0;
    a.tab_len = m.tab_len;
    a.status = status;
    CUtensorMap tu = *mu, tbm = *mb;
    void* o = out;
    const void* t = tab;
    void* args[] = {&tu, &tbm, &o, (void*)&t, &a};
    return brs_cuda_status(launch_pdl_c(k, dim3(m.grid), dim3(m.JT * m.G), m.smem, s, args));
}
