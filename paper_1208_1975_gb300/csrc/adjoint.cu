// Reverse-mode sweep of damped x-line block Jacobi (the transpose of Eq. blockiteration2).
//
// A forward sweep is u_{k+1} = u_k + omega z_k with z_k = M^{-1}(b - A u_k), i.e.
// u_{k+1} = G u_k + omega M^{-1} b with G = I - omega M^{-1} A.  A and the line block
// diagonal M are symmetric, so for a loss L(u_K) with lambda_{k+1} = dL/du_{k+1}:
//   mu_k       = M^{-1} lambda_{k+1}
//   lambda_k   = G^T lambda_{k+1} = lambda_{k+1} - omega A mu_k
//   dL/db     += omega mu_k
//   dL/da_d   += -omega mu_k . ( (dM/da_d) z_k + (dA/da_d) u_k )
// with dA/da_d = T_d (second difference along axis d, zero outside), and for x-line
// blocks dM/dax = Tx, dM/day = dM/daz = 2 I.
// One call performs these updates for one sweep; the caller supplies u_k (checkpointed
// or recomputed) and runs the calls from the last sweep to the first.
// The gradient terms only need z_k through x_k = u_k + z_k = M^{-1}(b + N u_k), the
// undamped line-Jacobi iterate (A = M - N), which the x-line sweep kernel produces in one
// pass: Tx (z + u) = Tx x, 2 z + Ty u = 2 x - Sy u, 2 z + Tz u = 2 x - Sz u, with S_d the
// sum of the two neighbours along d (T_d = 2 I - S_d).
#include <cstdlib>

#include "brs_internal.cuh"
#include "line_impl.cuh"

namespace {

constexpr int kThreads = 256;

// out = M_line^{-1} in, one line group per (j,k) at a time; in-place safe (a group reads
// its whole line, and its next one, before writing it).
template <typename T, int E, int G>
__global__ void __launch_bounds__(kThreads) line_minv_kernel(const T* in, T* out,
                                                             const T* __restrict__ tab, int nx,
                                                             int ny, int nz, bool vec)
{
    // Grid-stride over lines, the next line's cells loaded before the current one is solved
    // (the load latency overlaps the solve).  Every group of a warp runs the same number of
    // iterations, because the solve shuffles across the warp; groups past the last line
    // solve zeros.
    const int groups = blockDim.x / G;
    const long long nlines = (long long)ny * nz;
    const long long stride = (long long)gridDim.x * groups;
    const int lane = threadIdx.x % G;
    const long long warp_line0 = (long long)blockIdx.x * groups + (threadIdx.x & ~31) / G;
    const long long iters = warp_line0 < nlines ? (nlines - warp_line0 + stride - 1) / stride : 0;
    brs::LineTables<T, E, G> tb;
    tb.load(tab, lane);
    constexpr int NP = G * E;
    constexpr int LG = brs::Log2<G>::value;
    const T* ptab = tab + 3 * NP + 2 * LG * G;
    // VEC: full lines (nx = E G) with 16-byte aligned rows and E a whole number of 16-byte
    // vectors: each lane moves its E cells as vectors of the element type
    using V = typename brs::Vec16<T>::type;
    constexpr int NV = (int)(E * sizeof(T) / 16);
    constexpr bool CAN_VEC = (E * sizeof(T)) % 16 == 0;
    auto load = [&](long long line, T (&r)[E]) {
        const bool active = line < nlines;
        const size_t base = (size_t)(active ? line : 0) * nx;
        if (CAN_VEC && vec) {
            const V* src = reinterpret_cast<const V*>(in + base + lane * E);
#pragma unroll
            for (int m = 0; m < NV; ++m)
                reinterpret_cast<V*>(r)[m] = active ? src[m] : V{};
        } else {
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const int x = lane * E + q;
                r[q] = (active && x < nx) ? in[base + x] : T(0);
            }
        }
    };
    long long line = (long long)blockIdx.x * groups + threadIdx.x / G;
    T nxt[E];
    load(line, nxt);
    for (long long it = 0; it < iters; ++it, line += stride) {
        T r[E];
#pragma unroll
        for (int q = 0; q < E; ++q)
            r[q] = nxt[q];
        if (it + 1 < iters)
            load(line + stride, nxt);
        brs::line_solve<T, E, G>(r, tb, lane);
#pragma unroll
        for (int q = 0; q < E; ++q)
            r[q] = ptab[lane * E + q] * r[q];
        if (line < nlines) {
            const size_t base = (size_t)line * nx;
            if (CAN_VEC && vec) {
                V* dst = reinterpret_cast<V*>(out + base + lane * E);
#pragma unroll
                for (int m = 0; m < NV; ++m)
                    dst[m] = reinterpret_cast<const V*>(r)[m];
            } else {
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    const int x = lane * E + q;
                    if (x < nx)
                        out[base + x] = r[q];
                }
            }
        }
    }
}

// Four consecutive cells of a row (rem = cells left in the row); VEC: 16-byte vectors.
template <typename T>
__device__ __forceinline__ void ld4(T (&v)[4], const T* p, int rem, bool vec)
{
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            const float4 f = *reinterpret_cast<const float4*>(p);
            v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
        } else {
            const double2 f0 = reinterpret_cast<const double2*>(p)[0];
            const double2 f1 = reinterpret_cast<const double2*>(p)[1];
            v[0] = f0.x, v[1] = f0.y, v[2] = f1.x, v[3] = f1.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            v[q] = q < rem ? p[q] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4], int rem, bool vec)
{
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
            reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < rem)
                p[q] = v[q];
    }
}

// Second-difference neighbour sums of four cells of row `row` (at p, j, k): x (within the
// row), y and z.
template <typename T>
struct Nb4 {
    T c[4], sx[4], sy[4], sz[4];
};

template <typename T>
__device__ __forceinline__ void neighbours4(Nb4<T>& o, const T* p, int i0, int rem, int j,
                                            int k, int nx, int ny, int nz, long long plane,
                                            bool vec, bool xs, bool yz)
{
    ld4(o.c, p, rem, vec);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        o.sx[q] = o.sy[q] = o.sz[q] = T(0);
    if (xs) {
        const T left = i0 > 0 ? p[-1] : T(0);
        const T right = rem > 4 ? p[4] : T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            o.sx[q] = (q == 0 ? left : o.c[q - 1]) +
                      (q == 3 ? right : (q + 1 < rem ? o.c[q + 1] : T(0)));
    }
    if (!yz)
        return;
    T a[4];
    if (j > 0) {
        ld4(a, p - nx, rem, vec);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            o.sy[q] += a[q];
    }
    if (j + 1 < ny) {
        ld4(a, p + nx, rem, vec);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            o.sy[q] += a[q];
    }
    if (k > 0) {
        ld4(a, p - plane, rem, vec);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            o.sz[q] += a[q];
    }
    if (k + 1 < nz) {
        ld4(a, p + plane, rem, vec);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            o.sz[q] += a[q];
    }
}

// lambda <- lambda - omega A mu; gb += omega mu; per-CTA partial sums of the three
// coefficient-gradient terms mu.(Tx x), mu.(2x - Sy u), mu.(2x - Sz u) with x = M^{-1}(b +
// N u_k), u = u_k.  One warp per grid row at a time (grid-stride over rows with a fixed
// grid, so the partial sums are reproducible), four cells per lane.  FP32 contexts sum a
// lane's products over a row in FP32 before the FP64 sums (the FP64 pipe is the narrow one).
// Latency bound (ncu: long-scoreboard stalls, 16 resident warps at 120 registers): the FP32
// build is held to 3 CTAs per SM (78 registers, no spills); FP64 would spill, so it keeps 2.
template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) adjoint_update_kernel(
    T* __restrict__ lam, const T* __restrict__ mu, const T* __restrict__ x,
    const T* __restrict__ u, T* __restrict__ gb, int nx, int ny, int nz, double ax, double ay,
    double az, double omega, double* partials, bool vec)
{
    const long long plane = (long long)nx * ny;
    const long long nrows = (long long)ny * nz;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const T cx = (T)ax, cy = (T)ay, cz = (T)az, dg = (T)(2.0 * (ax + ay + az)), om = (T)omega;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (long long row = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); row < nrows;
         row += (long long)gridDim.x * wpb) {
        const int k = (int)(row / ny), j = (int)(row - (long long)k * ny);
        const long long base = row * nx;
        T h0 = T(0), h1 = T(0), h2 = T(0);
        for (int i0 = 4 * lane; i0 < nx; i0 += 128) {
            const int rem = nx - i0;
            const long long t = base + i0;
            Nb4<T> m, xx, uu;
            neighbours4(m, mu + t, i0, rem, j, k, nx, ny, nz, plane, vec, true, true);
            neighbours4(xx, x + t, i0, rem, j, k, nx, ny, nz, plane, vec, true, false);
            neighbours4(uu, u + t, i0, rem, j, k, nx, ny, nz, plane, vec, false, true);
            T lv[4], gv[4];
            ld4(lv, lam + t, rem, vec);
            ld4(gv, gb + t, rem, vec);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T mq = m.c[q];
                const T Amu = dg * mq - cx * m.sx[q] - cy * m.sy[q] - cz * m.sz[q];
                lv[q] = lv[q] - om * Amu;
                gv[q] += om * mq;
                const T x2 = T(2) * xx.c[q];
                if (q < rem) {
                    if constexpr (sizeof(T) == 4) {
                        h0 = fma(mq, x2 - xx.sx[q], h0);
                        h1 = fma(mq, x2 - uu.sy[q], h1);
                        h2 = fma(mq, x2 - uu.sz[q], h2);
                    } else {
                        g0 = fma(mq, x2 - xx.sx[q], g0);
                        g1 = fma(mq, x2 - uu.sy[q], g1);
                        g2 = fma(mq, x2 - uu.sz[q], g2);
                    }
                }
            }
            st4(lam + t, lv, rem, vec);
            st4(gb + t, gv, rem, vec);
        }
        if constexpr (sizeof(T) == 4) {
            g0 += (double)h0;
            g1 += (double)h1;
            g2 += (double)h2;
        }
    }
    __shared__ double red[3][kThreads / 32];
    double v[3] = {g0, g1, g2};
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1)
            v[d] += __shfl_down_sync(0xffffffffu, v[d], o);
        if ((threadIdx.x & 31) == 0)
            red[d][threadIdx.x >> 5] = v[d];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int d = 0; d < 3; ++d) {
            double w = threadIdx.x < kThreads / 32 ? red[d][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                w += __shfl_down_sync(0xffffffffu, w, o);
            if (threadIdx.x == 0)
                partials[3 * blockIdx.x + d] = w;
        }
    }
}

// FP32 form of the same update as a z-march: a warp owns 128 cells of row j (four per lane)
// over a chunk of kMarchKC planes, keeps mu and u of planes k-1, k, k+1 in registers, and
// loads the next plane's inputs before computing the current one (more loads in flight per
// warp, and the z neighbours are not loaded twice).  Items (j, x-chunk, z-chunk) go to warps
// in a fixed grid-stride order, so the partial sums are reproducible.
constexpr int kMarchKC = 16;

template <int N>
__device__ __forceinline__ void zero4(float (&v)[N])
{
#pragma unroll
    for (int q = 0; q < N; ++q)
        v[q] = 0.0f;
}

struct MarchIn {  // one plane's loads for the lanes' four cells
    float mup[4], up[4], muym[4], muyp[4], uym[4], uyp[4], xc[4], lam[4], gb[4];
    float mul, mur, xl, xr;
};

__global__ void __launch_bounds__(kThreads, 2) adjoint_update_march(
    float* __restrict__ lam, const float* __restrict__ mu, const float* __restrict__ x,
    const float* __restrict__ u, float* __restrict__ gb, int nx, int ny, int nz, double ax,
    double ay, double az, double omega, double* partials, bool vec)
{
    const long long plane = (long long)nx * ny;
    const int ncx = (nx + 127) / 128, nkc = (nz + kMarchKC - 1) / kMarchKC;
    const long long nitems = (long long)ny * ncx * nkc;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const float cx = (float)ax, cy = (float)ay, cz = (float)az;
    const float dg = (float)(2.0 * (ax + ay + az)), om = (float)omega;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (long long it = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); it < nitems;
         it += (long long)gridDim.x * wpb) {
        const int kc = (int)(it % nkc);
        const long long rest = it / nkc;
        const int xc = (int)(rest % ncx), j = (int)(rest / ncx);
        const int i0 = xc * 128 + 4 * lane, rem = nx - i0;
        const bool act = rem > 0;
        const int k0 = kc * kMarchKC, k1 = min(nz, k0 + kMarchKC);
        const long long row = (long long)j * nx + i0;
        auto at = [&](const float* a, int k) { return a + (long long)k * plane + row; };
        // plane k's loads (zeros outside the grid or for lanes past the row)
        auto load = [&](MarchIn& P, int k) {
            zero4(P.mup), zero4(P.up), zero4(P.muym), zero4(P.muyp), zero4(P.uym), zero4(P.uyp);
            zero4(P.xc), zero4(P.lam), zero4(P.gb);
            P.mul = P.mur = P.xl = P.xr = 0.0f;
            if (!act)
                return;
            if (k + 1 < nz) {
                ld4(P.mup, at(mu, k + 1), rem, vec);
                ld4(P.up, at(u, k + 1), rem, vec);
            }
            if (j > 0) {
                ld4(P.muym, at(mu, k) - nx, rem, vec);
                ld4(P.uym, at(u, k) - nx, rem, vec);
            }
            if (j + 1 < ny) {
                ld4(P.muyp, at(mu, k) + nx, rem, vec);
                ld4(P.uyp, at(u, k) + nx, rem, vec);
            }
            const float* px = at(x, k);
            const float* pm = at(mu, k);
            ld4(P.xc, px, rem, vec);
            ld4(P.lam, at(lam, k), rem, vec);
            ld4(P.gb, at(gb, k), rem, vec);
            if (i0 > 0) {
                P.mul = pm[-1];
                P.xl = px[-1];
            }
            if (rem > 4) {
                P.mur = pm[4];
                P.xr = px[4];
            }
        };
        float mum[4], muc[4], um[4], uc[4];
        zero4(mum), zero4(muc), zero4(um), zero4(uc);
        if (act) {
            if (k0 > 0) {
                ld4(mum, at(mu, k0 - 1), rem, vec);
                ld4(um, at(u, k0 - 1), rem, vec);
            }
            ld4(muc, at(mu, k0), rem, vec);
            ld4(uc, at(u, k0), rem, vec);
        }
        MarchIn nxt;
        load(nxt, k0);
        float h0 = 0.0f, h1 = 0.0f, h2 = 0.0f;
        for (int k = k0; k < k1; ++k) {
            const MarchIn cur = nxt;
            if (k + 1 < k1)
                load(nxt, k + 1);
            float lv[4], gv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float mq = muc[q];
                const float sxm = (q == 0 ? cur.mul : muc[q - 1]) +
                                  (q == 3 ? cur.mur : (q + 1 < rem ? muc[q + 1] : 0.0f));
                const float sym = cur.muym[q] + cur.muyp[q], szm = mum[q] + cur.mup[q];
                const float Amu = dg * mq - cx * sxm - cy * sym - cz * szm;
                lv[q] = cur.lam[q] - om * Amu;
                gv[q] = cur.gb[q] + om * mq;
                const float x2 = 2.0f * cur.xc[q];
                const float sxx = (q == 0 ? cur.xl : cur.xc[q - 1]) +
                                  (q == 3 ? cur.xr : (q + 1 < rem ? cur.xc[q + 1] : 0.0f));
                if (q < rem) {
                    h0 = fmaf(mq, x2 - sxx, h0);
                    h1 = fmaf(mq, x2 - (cur.uym[q] + cur.uyp[q]), h1);
                    h2 = fmaf(mq, x2 - (um[q] + cur.up[q]), h2);
                }
            }
            if (act) {
                st4(lam + (long long)k * plane + row, lv, rem, vec);
                st4(gb + (long long)k * plane + row, gv, rem, vec);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                mum[q] = muc[q], muc[q] = cur.mup[q];
                um[q] = uc[q], uc[q] = cur.up[q];
            }
        }
        g0 += (double)h0;
        g1 += (double)h1;
        g2 += (double)h2;
    }
    __shared__ double red[3][kThreads / 32];
    double v[3] = {g0, g1, g2};
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1)
            v[d] += __shfl_down_sync(0xffffffffu, v[d], o);
        if ((threadIdx.x & 31) == 0)
            red[d][threadIdx.x >> 5] = v[d];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int d = 0; d < 3; ++d) {
            double w = threadIdx.x < kThreads / 32 ? red[d][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                w += __shfl_down_sync(0xffffffffu, w, o);
            if (threadIdx.x == 0)
                partials[3 * blockIdx.x + d] = w;
        }
    }
}

// grad_a[d] += -omega * sum of the partials, in a fixed order.
__global__ void adjoint_reduce_kernel(const double* partials, int nblocks, double omega,
                                      double* grad_a)
{
    __shared__ double red[3][kThreads / 32];
    for (int d = 0; d < 3; ++d) {
        double acc = 0.0;
        for (int t = threadIdx.x; t < nblocks; t += blockDim.x)
            acc += partials[3 * t + d];
        for (int o = 16; o > 0; o >>= 1)
            acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0)
            red[d][threadIdx.x >> 5] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int d = 0; d < 3; ++d) {
            double w = threadIdx.x < kThreads / 32 ? red[d][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                w += __shfl_down_sync(0xffffffffu, w, o);
            if (threadIdx.x == 0)
                grad_a[d] += -omega * w;
        }
    }
}

template <typename T>
cudaError_t launch_minv(const brs_ctx* c, const T* in, T* out, cudaStream_t s)
{
    const LineCfg& L = c->lcfg;
    const int groups = kThreads / L.G;
    const long long nlines = (long long)c->p.ny * c->p.nz;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const long long need = (nlines + groups - 1) / groups;
    const T* tab = static_cast<const T*>(c->line_tab);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    const bool vec = nx == L.E * L.G && (nx * sizeof(T)) % 16 == 0 && a16(in) && a16(out);
#define BRS_MINV_CASE(EE, GG)                                                          \
    if (L.E == EE && L.G == GG) {                                                      \
        int per_sm = 1; /* one resident wave: the kernel strides over the lines */      \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, line_minv_kernel<T, EE, GG>, \
                                                      kThreads, 0);                    \
        const long long cap = (long long)sms * (per_sm > 0 ? per_sm : 1);               \
        const unsigned blocks = (unsigned)(need < cap ? need : cap);                    \
        line_minv_kernel<T, EE, GG><<<blocks, kThreads, 0, s>>>(in, out, tab, nx, ny, nz, vec); \
        return cudaGetLastError();                                                     \
    }
    BRS_MINV_CASE(4, 4)
    BRS_MINV_CASE(4, 8)
    BRS_MINV_CASE(4, 16)
    BRS_MINV_CASE(4, 32)
    BRS_MINV_CASE(8, 32)
    BRS_MINV_CASE(12, 32)
    BRS_MINV_CASE(16, 32)
#undef BRS_MINV_CASE
    return cudaErrorInvalidConfiguration;
}

// BRSMOOTH_ADJ_MARCH=0 selects the row form of the FP32 update (A/B measurements)
bool env_march()
{
    const char* v = std::getenv("BRSMOOTH_ADJ_MARCH");
    return !(v && v[0] == '0');
}

struct AdjState {
    void* mu = nullptr;
    double* partials = nullptr;
    int nblocks = 0;
    brs_ctx* xctx = nullptr;  // x-line Jacobi with omega = 1: x = M^{-1}(b + N u) in one pass
    int* xstatus = nullptr;   // xctx's own status word (its kernels report to the owner's)
};

template <typename T>
int adjoint_run(brs_ctx* c, T* lam, const T* u, const T* b, T* gb, double* ga, cudaStream_t s)
{
    AdjState* A = static_cast<AdjState*>(c->adjoint);
    T* x = static_cast<T*>(c->scratch);
    T* mu = static_cast<T*>(A->mu);
    // x = M^{-1}(b + N u_k): one undamped x-line Jacobi sweep from u_k
    int rc = line_sweep_launch(A->xctx, u, x, b, s);
    if (rc != BRS_OK)
        return rc;
    cudaError_t e = launch_minv<T>(c, lam, mu, s);  // mu = M^{-1} lambda
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    const bool vec = c->p.nx % 4 == 0 && a16(lam) && a16(mu) && a16(x) && a16(u) && a16(gb);
    if constexpr (sizeof(T) == 4) {
        if (env_march())
            adjoint_update_march<<<A->nblocks, kThreads, 0, s>>>(
                lam, mu, x, u, gb, c->p.nx, c->p.ny, c->p.nz, c->p.ax, c->p.ay, c->p.az,
                c->omega, A->partials, vec);
        else
            adjoint_update_kernel<T><<<A->nblocks, kThreads, 0, s>>>(
                lam, mu, x, u, gb, c->p.nx, c->p.ny, c->p.nz, c->p.ax, c->p.ay, c->p.az,
                c->omega, A->partials, vec);
    } else
    adjoint_update_kernel<T><<<A->nblocks, kThreads, 0, s>>>(lam, mu, x, u, gb, c->p.nx, c->p.ny,
                                                             c->p.nz, c->p.ax, c->p.ay, c->p.az,
                                                             c->omega, A->partials, vec);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return brs_cuda_status(e);
    adjoint_reduce_kernel<<<1, kThreads, 0, s>>>(A->partials, A->nblocks, c->omega, ga);
    return brs_cuda_status(cudaGetLastError());
}

}  // namespace

void adjoint_teardown(brs_ctx* c)
{
    AdjState* A = static_cast<AdjState*>(c->adjoint);
    if (!A)
        return;
    if (A->mu)
        cudaFree(A->mu);
    if (A->partials)
        cudaFree(A->partials);
    if (A->xctx) {
        A->xctx->dev_status = A->xstatus;
        brsmooth_destroy(A->xctx);
    }
    delete A;
    c->adjoint = nullptr;
}

extern "C" int brsmooth_adjoint_sweep(brs_ctx* c, void* lam, const void* u_k, const void* b,
                                      void* grad_b, double* grad_a, void* stream)
{
    cudaGetLastError();  // start from a clean launch-error state
    if (!c || !lam || !u_k || !b || !grad_b || !grad_a)
        return BRS_ERR_ARG;
    if (c->batch || c->p.block != BRS_XLINE || c->p.method != BRS_JACOBI)
        return BRS_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!c->adjoint) {
        AdjState* A = new AdjState();
        c->adjoint = A;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const long long need = ((long long)c->p.ny * c->p.nz + kThreads / 32 - 1) / (kThreads / 32);
        A->nblocks = (int)(need < (long long)sms * 8 ? need : (long long)sms * 8);
        if (A->nblocks < 1)
            A->nblocks = 1;
        cudaError_t e = cudaMalloc(&A->mu, (size_t)c->cells * c->esize);
        if (e == cudaSuccess)
            e = cudaMalloc(&A->partials, sizeof(double) * 3 * A->nblocks);
        int rc = brs_cuda_status(e);
        if (rc == BRS_OK) {
            brs_params q = c->p;
            q.omega = 1.0;
            rc = brsmooth_create(&q, &A->xctx);
        }
        if (rc != BRS_OK) {
            adjoint_teardown(c);
            return rc;
        }
        // only its line kernel is used: no Jacobi buffer or line-major copies, and faults
        // land in this context
        cudaFree(A->xctx->scratch);
        A->xctx->scratch = nullptr;
        line_seq_teardown(A->xctx);
        A->xstatus = A->xctx->dev_status;
        A->xctx->dev_status = c->dev_status;
    }
    c->last_stream = s;
    if (c->p.dtype == BRS_F64)
        return adjoint_run<double>(c, (double*)lam, (const double*)u_k, (const double*)b,
                                   (double*)grad_b, grad_a, s);
    return adjoint_run<float>(c, (float*)lam, (const float*)u_k, (const float*)b, (float*)grad_b,
                              grad_a, s);
}
