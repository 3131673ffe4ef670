// Host construction of the factor tables used by the cross-lane scan Thomas solve
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
#pragma once

#include <algorithm>
#include <vector>

template <typename T>
std::vector<T> scan_thomas_tables(int n, double off, double diag, double omega, int E, int G,
                                  bool with_p)
{
    const int NP = G * E;
    int LG = 0;
    while ((1 << LG) < G)
        ++LG;
    std::vector<double> p(NP, 0.0), c(NP, 0.0), e(NP, 0.0);
    p[0] = 1.0 / diag;
    for (int i = 1; i < n; ++i)
        p[i] = 1.0 / (diag - off * off * p[i - 1]);
    for (int i = 1; i < n; ++i)
        c[i] = off * p[i - 1];
    for (int i = 0; i + 1 < n; ++i)
        e[i] = off * p[i + 1];
    std::vector<double> Af(G, 1.0), Ab(G, 1.0);
    for (int l = 0; l < G; ++l)
        for (int q = 0; q < E; ++q) {
            Af[l] *= c[l * E + q];
            Ab[l] *= e[l * E + q];
        }
    std::vector<T> tab((with_p ? 4 : 3) * NP + 2 * LG * G);
    for (int i = 0; i < NP; ++i) {
        tab[i] = (T)c[i];
        tab[NP + i] = (T)e[i];
        tab[2 * NP + i] = (T)(i < n ? omega * p[i] : 0.0);
    }
    for (int t = 0; t < LG; ++t)
        for (int l = 0; l < G; ++l) {
            double f = 1.0, b = 1.0;
            for (int m = std::max(0, l - (1 << t) + 1); m <= l; ++m)
                f *= Af[m];
            for (int m = l; m < G && m < l + (1 << t); ++m)
                b *= Ab[m];
            tab[3 * NP + t * G + l] = (T)f;
            tab[3 * NP + LG * G + t * G + l] = (T)b;
        }
    if (with_p)
        for (int i = 0; i < NP; ++i)
            tab[3 * NP + 2 * LG * G + i] = (T)(i < n ? p[i] : 0.0);
    return tab;
}
