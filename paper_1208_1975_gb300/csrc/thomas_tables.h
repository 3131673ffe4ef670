// Construction of the factor tables used by the cross-lane scan Thomas solve
// (line_solve in line_impl.cuh) for a constant symmetric tridiagonal block
//   M = tridiag(-off, diag, -off) of size n.
// The LU pivots are the same for every system with this (n, off, diag), so they are
// computed once in FP64:  p_0 = 1/diag,  p_i = 1/(diag - off^2 p_{i-1}).
// Layout for G lanes x E cells per lane (NP = G E, LG = log2 G), rounded to T:
//   [0, NP)                c_i = off p_{i-1}   (forward multipliers; 0 at i = 0 and i >= n)
//   [NP, 2NP)              e_i = off p_{i+1}   (backward multipliers; 0 at i >= n-1)
//   [2NP, 3NP)             omega p_i           (0 beyond n)
//   [3NP, 3NP+G LG)        forward scan multipliers, step t at [t G + lane]
//   [3NP+G LG, 3NP+2G LG)  backward scan multipliers
//   [3NP+2G LG, 4NP+2G LG) p_i (only when with_p)
// One routine serves the host (context set-up) and the device (the allocation-free entry
// point builds its tables in a one-thread kernel), so both paths use the same arithmetic.
#pragma once

#include <vector>

#ifdef __CUDACC__
#define BRS_HD __host__ __device__
#else
#define BRS_HD
#endif

// Largest G*E of any lane layout (32 lanes x 16 cells).
constexpr int kScanMaxNP = 512;

// Lanes per line G and cells per lane E for a line of n cells (G E >= n; E a whole number
// of 16-byte vectors for both FP32 and FP64).  False beyond 512 cells.
BRS_HD inline bool scan_lanes(int n, int* E, int* G)
{
    if (n <= 16) { *G = 4; *E = 4; }
    else if (n <= 32) { *G = 8; *E = 4; }
    else if (n <= 64) { *G = 16; *E = 4; }
    else if (n <= 128) { *G = 32; *E = 4; }
    else if (n <= 256) { *G = 32; *E = 8; }
    else if (n <= 384) { *G = 32; *E = 12; }
    else if (n <= 512) { *G = 32; *E = 16; }
    else return false;
    return true;
}

// Number of table entries for the layout (E, G).
BRS_HD inline int scan_table_len(int E, int G, bool with_p)
{
    int LG = 0;
    while ((1 << LG) < G)
        ++LG;
    return (with_p ? 4 : 3) * G * E + 2 * LG * G;
}

// Write the tables into tab[0 .. scan_table_len) (caller storage); -1 if the layout is
// larger than kScanMaxNP cells or cap entries, else the entry count.
template <typename T>
BRS_HD int scan_thomas_fill(T* tab, int cap, int n, double off, double diag, double omega, int E,
                            int G, bool with_p)
{
    const int NP = G * E;
    int LG = 0;
    while ((1 << LG) < G)
        ++LG;
    const int len = scan_table_len(E, G, with_p);
    if (NP > kScanMaxNP || G > 32 || len > cap)
        return -1;
    // one pass over the cells with the pivots p_{i-1}, p_i, p_{i+1} live: the only arrays
    // are the per-lane products (a few hundred bytes of stack, so a one-thread device
    // launch needs no larger stack than the default)
    double Af[32], Ab[32];
    for (int l = 0; l < G; ++l)
        Af[l] = Ab[l] = 1.0;
    double pprev = 0.0, pcur = 1.0 / diag;  // p_{i-1}, p_i (p_0 = 1/diag)
    for (int i = 0; i < NP; ++i) {
        const double pi = i < n ? pcur : 0.0;
        const double pnext = i + 1 < n ? 1.0 / (diag - off * off * pi) : 0.0;
        const double ci = (i >= 1 && i < n) ? off * pprev : 0.0;  // c_i = off p_{i-1}
        const double ei = i + 1 < n ? off * pnext : 0.0;          // e_i = off p_{i+1}
        tab[i] = (T)ci;
        tab[NP + i] = (T)ei;
        tab[2 * NP + i] = (T)(omega * pi);
        if (with_p)
            tab[3 * NP + 2 * LG * G + i] = (T)pi;
        Af[i / E] *= ci;
        Ab[i / E] *= ei;
        pprev = pi;
        pcur = pnext;
    }
    for (int t = 0; t < LG; ++t)
        for (int l = 0; l < G; ++l) {
            double f = 1.0, b = 1.0;
            const int m0 = l - (1 << t) + 1;
            for (int m = m0 > 0 ? m0 : 0; m <= l; ++m)
                f *= Af[m];
            for (int m = l; m < G && m < l + (1 << t); ++m)
                b *= Ab[m];
            tab[3 * NP + t * G + l] = (T)f;
            tab[3 * NP + LG * G + t * G + l] = (T)b;
        }
    return len;
}

// Tables of the two-warp line solve (line_solve_pair in line_impl.cuh) for lines of up to
// 512 cells: 64 lanes of kPairE = 8 cells, lanes 0-31 (cells 0-255) in one warp and lanes
// 32-63 (cells 256-511) in the other.  Each warp scans its half on its own; the halves'
// carries cross through shared memory.  Layout (NP = 512):
//   [0, NP)                  c_i   (as for scan_thomas_fill)
//   [NP, 2NP)                e_i
//   [2NP, 3NP)               omega p_i
//   [3NP, 3NP+5*64)          forward scan multipliers within a half, step t at [t*64 + lane]
//   [3NP+5*64, 3NP+10*64)    backward scan multipliers within a half
//   [3NP+640, 3NP+704)       pf: product of the half's lane products before the lane
//   [3NP+704, 3NP+768)       pb: product of the half's lane products after the lane
constexpr int kPairE = 8;
constexpr int kPairLen = 3 * 512 + 768;

template <typename T>
BRS_HD int scan_pair_fill(T* tab, int cap, int n, double off, double diag, double omega)
{
    constexpr int NP = 512, L = 64, H = 32, LG = 5;
    if (n > NP || cap < kPairLen)
        return -1;
    double Af[L], Ab[L];
    for (int l = 0; l < L; ++l)
        Af[l] = Ab[l] = 1.0;
    double pprev = 0.0, pcur = 1.0 / diag;
    for (int i = 0; i < NP; ++i) {
        const double pi = i < n ? pcur : 0.0;
        const double pnext = i + 1 < n ? 1.0 / (diag - off * off * pi) : 0.0;
        const double ci = (i >= 1 && i < n) ? off * pprev : 0.0;
        const double ei = i + 1 < n ? off * pnext : 0.0;
        tab[i] = (T)ci;
        tab[NP + i] = (T)ei;
        tab[2 * NP + i] = (T)(omega * pi);
        Af[i / kPairE] *= ci;
        Ab[i / kPairE] *= ei;
        pprev = pi;
        pcur = pnext;
    }
    for (int m = 0; m < L; ++m) {
        const int h0 = (m / H) * H, h1 = h0 + H - 1;  // the lanes of m's half
        for (int t = 0; t < LG; ++t) {
            double f = 1.0, b = 1.0;
            for (int q = m - (1 << t) + 1 < h0 ? h0 : m - (1 << t) + 1; q <= m; ++q)
                f *= Af[q];
            for (int q = m; q <= h1 && q < m + (1 << t); ++q)
                b *= Ab[q];
            tab[3 * NP + t * L + m] = (T)f;
            tab[3 * NP + LG * L + t * L + m] = (T)b;
        }
        double pf = 1.0, pb = 1.0;
        for (int q = h0; q < m; ++q)
            pf *= Af[q];
        for (int q = m + 1; q <= h1; ++q)
            pb *= Ab[q];
        tab[3 * NP + 2 * LG * L + m] = (T)pf;
        tab[3 * NP + 2 * LG * L + L + m] = (T)pb;
    }
    return kPairLen;
}

// Pivots of the elimination from both ends (twisted factorisation) of tridiag(-off, diag,
// -off) of size n, FP64: pv_i = p_i left of the twist cell m = (n-1)/2 (p_0 = 1/diag,
// p_i = 1/(diag - off^2 p_{i-1})), g_m = 1/(diag - off^2 (p_{m-1} + q_{m+1})) at it, and
// q_i = p_{n-1-i} right of it (the same recurrence from the other end).
inline std::vector<double> twist_pivots(int n, double off, double diag)
{
    const int m = (n - 1) / 2;
    std::vector<double> pv(n, 0.0);
    double p = 0.0;
    for (int i = 0; i < n - 1 - m; ++i) {  // p_0 .. p_{n-2-m}: both sides' steps
        p = 1.0 / (diag - (i ? off * off * p : 0.0));
        if (i < m)
            pv[i] = p;
        pv[n - 1 - i] = p;
    }
    const double pl = m >= 1 ? pv[m - 1] : 0.0;
    const double qr = m + 1 <= n - 1 ? pv[m + 1] : 0.0;
    pv[m] = 1.0 / (diag - off * off * pl - off * off * qr);
    return pv;
}

// Host convenience: the tables as a vector (empty if the layout is too large).
template <typename T>
std::vector<T> scan_thomas_tables(int n, double off, double diag, double omega, int E, int G,
                                  bool with_p)
{
    std::vector<T> tab(scan_table_len(E, G, with_p));
    if (scan_thomas_fill<T>(tab.data(), (int)tab.size(), n, off, diag, omega, E, G, with_p) < 0)
        tab.clear();
    return tab;
}

template <typename T>
std::vector<T> scan_pair_tables(int n, double off, double diag, double omega)
{
    std::vector<T> tab(kPairLen);
    if (scan_pair_fill<T>(tab.data(), (int)tab.size(), n, off, diag, omega) < 0)
        tab.clear();
    return tab;
}
