// Command-line driver for the library's host-side table builders (thomas_tables.h,
// box_parity.h), so that the CPU tests can check the tables against direct solves in numpy.
// Output: whitespace-separated numbers on stdout.
//   scan   n off diag omega E G with_p   -> len, then the scan Thomas tables (FP64)
//   pair   n off diag omega              -> len, then the two-warp tables (FP64)
//   twist  n off diag                    -> the n pivots of the elimination from both ends
//   parity bx by bz  (stdin: the n*n block inverse, row-major)
//                                        -> use, cls_n[8], cls_off[8], pc_off[8],
//                                           |pc| and pc, |ftab| and ftab, |utab| and utab
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "box_parity.h"
#include "thomas_tables.h"

static void put(const std::vector<double>& v)
{
    std::printf("%zu\n", v.size());
    for (double x : v)
        std::printf("%.17g\n", x);
}

static void put(const std::vector<int>& v)
{
    std::printf("%zu\n", v.size());
    for (int x : v)
        std::printf("%d\n", x);
}

int main(int argc, char** argv)
{
    if (argc < 2)
        return 2;
    const char* mode = argv[1];
    if (!std::strcmp(mode, "scan") && argc == 9) {
        const int n = std::atoi(argv[2]), E = std::atoi(argv[6]), G = std::atoi(argv[7]);
        put(scan_thomas_tables<double>(n, std::atof(argv[3]), std::atof(argv[4]),
                                       std::atof(argv[5]), E, G, std::atoi(argv[8]) != 0));
        return 0;
    }
    if (!std::strcmp(mode, "pair") && argc == 6) {
        put(scan_pair_tables<double>(std::atoi(argv[2]), std::atof(argv[3]), std::atof(argv[4]),
                                     std::atof(argv[5])));
        return 0;
    }
    if (!std::strcmp(mode, "twist") && argc == 5) {
        put(twist_pivots(std::atoi(argv[2]), std::atof(argv[3]), std::atof(argv[4])));
        return 0;
    }
    if (!std::strcmp(mode, "parity") && argc == 5) {
        const int bx = std::atoi(argv[2]), by = std::atoi(argv[3]), bz = std::atoi(argv[4]);
        const size_t n = (size_t)bx * by * bz;
        std::vector<double> inv(n * n);
        for (size_t i = 0; i < n * n; ++i)
            if (std::scanf("%lf", &inv[i]) != 1)
                return 3;
        const ParityTables pt = parity_tables(bx, by, bz, inv);
        std::printf("%d\n", pt.use ? 1 : 0);
        for (int c = 0; c < 8; ++c)
            std::printf("%d\n", pt.cls_n[c]);
        for (int c = 0; c < 8; ++c)
            std::printf("%d\n", pt.cls_off[c]);
        for (int c = 0; c < 8; ++c)
            std::printf("%lld\n", pt.pc_off[c]);
        put(pt.pc);
        put(pt.ftab);
        put(pt.utab);
        return 0;
    }
    return 2;
}
