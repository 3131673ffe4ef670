// Parity classes of a box block (host side, plain C++): the tables with which box.cu applies
// the block inverse by its 8 parity-class blocks, and which the host tests check on CPU.
//
// With constant coefficients the block matrix of a bx x by x bz box, and so its inverse
// Ahat, is unchanged by the reflections of the box along x, y and z.  G maps a block's cells
// to sums and differences of mirrored cells along each axis; in that basis Ahat is block
// diagonal with one dense block per parity class, and
//   Ahat r = G^T P (G r),   P = W G Ahat G^T W,   W = diag(1/2 per mirrored pair and axis).
#pragma once

#include <vector>

struct ParityTables {
    bool use = false;        // the classes save half the multiply-adds and one has 16+ cells
    int cls_n[8] = {0};      // class sizes (class c: sums / differences along x, y, z by its bits)
    int cls_off[8] = {0};    // offsets in the class-major folded row
    long long pc_off[8] = {0};
    std::vector<double> pc;  // class blocks of P, class c at pc_off[c], cls_n[c] x cls_n[c]
    // [3][n] pairs (a, b): out[o] = in[a] + sign(b) in[|b| - 1] (b = 0: in[a]); the fold's
    // passes x, y, z (the last writes class order) and the unfold's z, y, x (the first reads it)
    std::vector<int> ftab, utab;
};

// Parity classes of a bx x by x bz box (see the file comment).  Along an axis of extent b the
// folded coordinates are the sums j < ceil(b/2) (pair (j, b-1-j), or the middle cell of an
// odd b) and the differences j < floor(b/2); a class picks sums or differences per axis.
// Builds the class sizes and offsets, the butterflies of G (fmap) and G^T (umap), and the
// class blocks of P = W G Ahat G^T W from the FP64 inverse.
inline ParityTables parity_tables(int bx, int by, int bz, const std::vector<double>& inv)
{
    ParityTables pt;
    const int b[3] = {bx, by, bz}, n = bx * by * bz;
    int hs[3], ha[3];
    for (int d = 0; d < 3; ++d) {
        ha[d] = b[d] / 2;
        hs[d] = b[d] - ha[d];
    }
    long long work = 0;
    int off = 0;
    for (int cl = 0; cl < 8; ++cl) {
        int nc = 1;
        for (int d = 0; d < 3; ++d)
            nc *= ((cl >> d) & 1) ? ha[d] : hs[d];
        pt.cls_n[cl] = nc;
        pt.cls_off[cl] = off;
        off += nc;
        work += (long long)nc * nc;
    }
    // only where it saves at least half of the multiply-adds and the class products are not
    // tiny: 4^3 boxes (classes of 8 cells) measured 8.27 -> 7.64 Gcell/s (FP64 GS, 256^3),
    // 8^3 (classes of 64) 1.15 -> 3.81
    int big = 0;
    for (int cl = 0; cl < 8; ++cl)
        big = pt.cls_n[cl] > big ? pt.cls_n[cl] : big;
    if (off != n || 2 * work > (long long)n * n || big < 16)
        return pt;
    // folded index f -> its cells with signs, and the weight W[f]
    std::vector<int> fmap((size_t)n * 8, 0), umap((size_t)n * 8, 0);
    std::vector<double> W(n);
    std::vector<int> ucount(n, 0);
    for (int cl = 0; cl < 8; ++cl) {
        const int c3[3] = {cl & 1, (cl >> 1) & 1, (cl >> 2) & 1};
        const int sz[3] = {c3[0] ? ha[0] : hs[0], c3[1] ? ha[1] : hs[1], c3[2] ? ha[2] : hs[2]};
        for (int i = 0; i < pt.cls_n[cl]; ++i) {
            const int j[3] = {i % sz[0], (i / sz[0]) % sz[1], i / (sz[0] * sz[1])};
            const int f = pt.cls_off[cl] + i;
            double w = 1.0;
            int q = 0;
            for (int e = 0; e < 8; ++e) {
                int x[3], sign = 1;
                bool ok = true;
                for (int d = 0; d < 3; ++d) {
                    const bool mir = (e >> d) & 1;
                    const bool pair = j[d] < ha[d];  // a mirrored pair (not the middle cell)
                    if (mir && !pair) {
                        ok = false;
                        break;
                    }
                    x[d] = mir ? b[d] - 1 - j[d] : j[d];
                    if (mir && c3[d])
                        sign = -sign;
                }
                if (!ok)
                    continue;
                const int l = x[0] + b[0] * (x[1] + b[1] * x[2]);
                fmap[(size_t)(q++) * n + f] = sign * (l + 1);
                umap[(size_t)(ucount[l]++) * n + l] = sign * (f + 1);
            }
            for (int d = 0; d < 3; ++d)
                if (j[d] < ha[d])
                    w *= 0.5;
            W[f] = w;
        }
    }
    // class blocks of P: P[f][g] = W[f] W[g] sum over their cells of s s' Ahat[l][l']
    std::vector<double>& pc = pt.pc;
    for (int cl = 0; cl < 8; ++cl) {
        const int nc = pt.cls_n[cl], o = pt.cls_off[cl];
        pt.pc_off[cl] = (long long)pc.size();
        for (int f = o; f < o + nc; ++f)
            for (int g = o; g < o + nc; ++g) {
                double acc = 0.0;
                for (int q = 0; q < 8 && fmap[(size_t)q * n + f]; ++q) {
                    const int ef = fmap[(size_t)q * n + f];
                    const int l = (ef > 0 ? ef : -ef) - 1;
                    for (int r = 0; r < 8 && fmap[(size_t)r * n + g]; ++r) {
                        const int eg = fmap[(size_t)r * n + g];
                        const int l2 = (eg > 0 ? eg : -eg) - 1;
                        const double v = inv[(size_t)l * n + l2];
                        acc += ((ef > 0) == (eg > 0)) ? v : -v;
                    }
                }
                pc.push_back(W[f] * W[g] * acc);
            }
    }
    // the separable passes: layouts are (c0, c1, c2) lexicographic with each coordinate a
    // cell or, once its axis is folded, a folded coordinate (sums first, then differences)
    auto lex = [&](const int c[3]) { return c[0] + b[0] * (c[1] + b[1] * c[2]); };
    std::vector<int> perm(n);  // lexicographic folded index -> class-major index
    for (int cl = 0; cl < 8; ++cl) {
        const int c3[3] = {cl & 1, (cl >> 1) & 1, (cl >> 2) & 1};
        const int sz[3] = {c3[0] ? ha[0] : hs[0], c3[1] ? ha[1] : hs[1], c3[2] ? ha[2] : hs[2]};
        for (int i = 0; i < pt.cls_n[cl]; ++i) {
            const int j[3] = {i % sz[0], (i / sz[0]) % sz[1], i / (sz[0] * sz[1])};
            const int f[3] = {j[0] + c3[0] * hs[0], j[1] + c3[1] * hs[1], j[2] + c3[2] * hs[2]};
            perm[lex(f)] = pt.cls_off[cl] + i;
        }
    }
    std::vector<int>& ftab = pt.ftab;
    std::vector<int>& utab = pt.utab;
    ftab.assign((size_t)6 * n, 0);
    utab.assign((size_t)6 * n, 0);
    for (int d = 0; d < 3; ++d)
        for (int o = 0; o < n; ++o) {
            int c[3] = {o % b[0], (o / b[0]) % b[1], o / (b[0] * b[1])};
            // fold pass d: output folded coordinate c[d] from the cells along d
            {
                int ca[3] = {c[0], c[1], c[2]}, cb[3] = {c[0], c[1], c[2]};
                const bool anti = c[d] >= hs[d];
                const int jj = anti ? c[d] - hs[d] : c[d];
                ca[d] = jj;
                cb[d] = b[d] - 1 - jj;
                const size_t at = 2 * ((size_t)d * n + (d == 2 ? perm[o] : o));
                ftab[at] = lex(ca);
                ftab[at + 1] = jj < ha[d] ? (anti ? -(lex(cb) + 1) : lex(cb) + 1) : 0;  // cb valid for pairs
                // (the last pass, z, writes class order: its table is indexed by the output's
                // class-major position)
            }
            // unfold pass (z, y, x): output cell coordinate c[ax] from the folded ones
            {
                const int ax = 2 - d;
                int ca[3] = {c[0], c[1], c[2]}, cb[3] = {c[0], c[1], c[2]};
                const int x = c[ax], jj = x < b[ax] - 1 - x ? x : b[ax] - 1 - x;
                ca[ax] = jj;
                cb[ax] = hs[ax] + jj;
                const bool pair = jj < ha[ax];  // else the middle cell: no difference term
                const size_t at = 2 * ((size_t)d * n + o);
                utab[at] = d == 0 ? perm[lex(ca)] : lex(ca);
                utab[at + 1] = 0;
                if (pair) {
                    const int ib = d == 0 ? perm[lex(cb)] : lex(cb);
                    utab[at + 1] = x == jj ? ib + 1 : -(ib + 1);
                }
            }
        }
    pt.use = true;
    return pt;
}
