/*
 * Plain, slow, FP64 reference of block relaxation on a 3D constant-coefficient
 * 7-point stencil.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it; the CUDA library never calls it.
 *
 * Shares no code, header, table or helper with the CUDA path.  Every routine is the
 * textbook definition written out; no blocking, fusion or reordering beyond it.
 *
 * Grid layout: interior unknowns only, x fastest: idx = i + nx*(j + ny*k).
 * Values outside the interior are Dirichlet values equal to zero (a caller with
 * non-zero boundary data folds it into b).  Every cell therefore uses the interior
 * stencil, as the ghost-cell layer of Sec. 1.1 makes it do.
 *
 * Operator (Eq. stencil3d7 of Sec. 1.1, generalised to per-axis coefficients):
 *   (A u)_ijk = 2(ax+ay+az) u_ijk - ax(u_{i-1}+u_{i+1}) - ay(u_{j-1}+u_{j+1}) - az(u_{k-1}+u_{k+1})
 * With ax=ay=az=1 this is the paper's 6u - sum(neighbours) = h^2 f.
 *
 * Block iteration (Sec. 2, Eq. blockiteration2):  u <- u + omega * M^{-1} (b - A u)
 * where M is the block diagonal of A for a partition into full x-lines (one block per
 * (j,k)), full xy-planes (one block per k) or bx*by*bz boxes (the spatial blocks of the
 * paper, one precomputed inverse applied as a dense product).  Block Jacobi evaluates every block from
 * the same old iterate into a second vector (Sec. 2, Alg. 2 step 4); block
 * Gauss-Seidel (Eq. sm:blockm) visits the blocks one after another, always reading the
 * newest values.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC brs_oracle.c -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, k) ((long)(i) + (long)nx * ((long)(j) + (long)ny * (long)(k)))

/* Value of u at (i,j,k), zero outside the interior (homogeneous Dirichlet). */
static double at(const double *u, int nx, int ny, int nz, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz)
        return 0.0;
    return u[IDX(i, j, k)];
}

/* (A u) at one cell: the 7-point stencil of Eq. stencil3d7 with coefficients ax, ay, az. */
static double stencil_at(const double *u, int nx, int ny, int nz, double ax, double ay,
                         double az, int i, int j, int k)
{
    double c = 2.0 * (ax + ay + az) * at(u, nx, ny, nz, i, j, k);
    c -= ax * (at(u, nx, ny, nz, i - 1, j, k) + at(u, nx, ny, nz, i + 1, j, k));
    c -= ay * (at(u, nx, ny, nz, i, j - 1, k) + at(u, nx, ny, nz, i, j + 1, k));
    c -= az * (at(u, nx, ny, nz, i, j, k - 1) + at(u, nx, ny, nz, i, j, k + 1));
    return c;
}

/* out = A u over the whole grid (Sec. 1.1). */
void orc_apply_A(int nx, int ny, int nz, double ax, double ay, double az, const double *u,
                 double *out)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                out[IDX(i, j, k)] = stencil_at(u, nx, ny, nz, ax, ay, az, i, j, k);
}

/* r = b - A u (the residual of Eq. blockiteration2). */
void orc_residual(int nx, int ny, int nz, double ax, double ay, double az, const double *u,
                  const double *b, double *r)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                r[IDX(i, j, k)] = b[IDX(i, j, k)] - stencil_at(u, nx, ny, nz, ax, ay, az, i, j, k);
}

/* Sum of squares in FP64, sequential order. */
double orc_sumsq(long n, const double *r)
{
    double s = 0.0;
    for (long t = 0; t < n; ++t)
        s += r[t] * r[t];
    return s;
}

/*
 * Textbook Thomas algorithm for the symmetric tridiagonal system
 *   diag*x_i + off*(x_{i-1} + x_{i+1}) = rhs_i,  i = 0..n-1,
 * forward elimination followed by back substitution.  The elimination is re-derived
 * for every call.  `cp` and `dp` are caller scratch of length n.
 */
void orc_thomas(int n, double off, double diag, const double *rhs, double *x, double *cp,
                double *dp)
{
    if (n <= 0)
        return;
    cp[0] = off / diag;
    dp[0] = rhs[0] / diag;
    for (int i = 1; i < n; ++i) {
        double m = diag - off * cp[i - 1];
        cp[i] = off / m;
        dp[i] = (rhs[i] - off * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i)
        x[i] = dp[i] - cp[i] * x[i + 1];
}

/*
 * x-line block of A: for fixed (j,k) the rows of A restricted to the line's unknowns,
 * M_line = tridiag(-ax, 2(ax+ay+az), -ax) of size nx.  Solve M_line d = r for the
 * line (j,k) of r, writing d into the same line of `out`.
 */
static void line_block_solve(int nx, int ny, double ax, double ay, double az, int j, int k,
                             const double *r, double *out, double *scratch)
{
    double *rhs = scratch, *x = scratch + nx, *cp = scratch + 2 * nx, *dp = scratch + 3 * nx;
    for (int i = 0; i < nx; ++i)
        rhs[i] = r[IDX(i, j, k)];
    orc_thomas(nx, -ax, 2.0 * (ax + ay + az), rhs, x, cp, dp);
    for (int i = 0; i < nx; ++i)
        out[IDX(i, j, k)] = x[i];
}

/* out = M^{-1} r for the x-line partition (every line solved independently). */
void orc_line_minv(int nx, int ny, int nz, double ax, double ay, double az, const double *r,
                   double *out)
{
#pragma omp parallel
    {
        double *scratch = (double *)malloc(sizeof(double) * 4 * (size_t)nx);
#pragma omp for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                line_block_solve(nx, ny, ax, ay, az, j, k, r, out, scratch);
        free(scratch);
    }
}

/*
 * Damped block Jacobi with x-line blocks (Alg. 2 with full-line blocks):
 *   step 1: r = b - A u        step 2: d = M_line^{-1} r per line
 *   step 3: v = u + omega d    (step 4, the pointer swap, is the caller's)
 * `work` is caller scratch of nx*ny*nz doubles.
 */
void orc_line_jacobi(int nx, int ny, int nz, double ax, double ay, double az, double omega,
                     const double *u, const double *b, double *v, double *work)
{
    long n = (long)nx * ny * nz;
    orc_residual(nx, ny, nz, ax, ay, az, u, b, work);
    orc_line_minv(nx, ny, nz, ax, ay, az, work, work);
#pragma omp parallel for schedule(static)
    for (long t = 0; t < n; ++t)
        v[t] = u[t] + omega * work[t];
}

/*
 * Block Gauss-Seidel with x-line blocks (Eq. sm:blockm): the lines are visited one at a
 * time in the order given, each reading the newest values:
 *   r_b = b_b - (A u)_b,  u_b <- u_b + omega * M_line^{-1} r_b.
 * order 0: lexicographic (k outer, j inner); 1: reverse lexicographic;
 * 2: zebra (lines with j+k even first, then odd, each colour lexicographic).
 */
void orc_line_gs(int nx, int ny, int nz, double ax, double ay, double az, double omega,
                 int order, double *u, const double *b)
{
    double *scratch = (double *)malloc(sizeof(double) * 6 * (size_t)nx);
    double *r = scratch + 4 * nx, *d = scratch + 5 * nx;
    long nlines = (long)ny * nz;
    long *seq = (long *)malloc(sizeof(long) * (size_t)nlines);
    long cnt = 0;
    if (order == 2) {
        for (int colour = 0; colour < 2; ++colour)
            for (long q = 0; q < nlines; ++q)
                if ((int)(((q % ny) + (q / ny)) & 1) == colour)
                    seq[cnt++] = q;
    } else {
        for (long q = 0; q < nlines; ++q)
            seq[q] = (order == 1) ? nlines - 1 - q : q;
    }
    for (long s = 0; s < nlines; ++s) {
        int j = (int)(seq[s] % ny), k = (int)(seq[s] / ny);
        for (int i = 0; i < nx; ++i)
            r[i] = b[IDX(i, j, k)] - stencil_at(u, nx, ny, nz, ax, ay, az, i, j, k);
        orc_thomas(nx, -ax, 2.0 * (ax + ay + az), r, d, scratch, scratch + nx);
        for (int i = 0; i < nx; ++i)
            u[IDX(i, j, k)] += omega * d[i];
    }
    free(seq);
    free(scratch);
}

/*
 * xy-plane block of A: for fixed k the rows of A restricted to the plane's unknowns,
 *   M_plane = ax*Tx (x) I + ay*I (x) Ty + 2az*I,  size m = nx*ny, plane index i + nx*j.
 * It is symmetric positive definite with half-bandwidth nx.  It is factored once by a
 * banded Cholesky M = L L^T and the factor is reused for every plane and sweep (the
 * "invert once" of Sec. 4.3).  Band storage: row q holds L[q][q-nx .. q] at
 * L[q*(nx+1) + (c - q + nx)].
 * Returns 0 on success, -1 if a pivot is not positive.
 */
int orc_plane_factor(int nx, int ny, double ax, double ay, double az, double *L)
{
    long m = (long)nx * ny;
    int w = nx;
    for (long q = 0; q < m; ++q) {
        int iq = (int)(q % nx);
        long c0 = q - w < 0 ? 0 : q - w;
        for (long c = c0; c <= q; ++c) {
            /* entry M[q][c] of the plane block */
            double a = 0.0;
            if (c == q)
                a = 2.0 * (ax + ay + az);
            else if (c == q - 1 && iq > 0)
                a = -ax;
            else if (c == q - nx)
                a = -ay;
            double s = a;
            long t0 = c - w < c0 ? c0 : c - w;
            for (long t = t0; t < c; ++t)
                s -= L[q * (w + 1) + (t - q + w)] * L[c * (w + 1) + (t - c + w)];
            if (c < q) {
                L[q * (w + 1) + (c - q + w)] = s / L[c * (w + 1) + w];
            } else {
                if (!(s > 0.0))
                    return -1;
                L[q * (w + 1) + w] = sqrt(s);
            }
        }
    }
    return 0;
}

/* Solve M_plane x = rhs in place with the banded Cholesky factor (L y = rhs, L^T x = y). */
void orc_plane_solve(int nx, int ny, const double *L, double *x)
{
    long m = (long)nx * ny;
    int w = nx;
    for (long q = 0; q < m; ++q) {
        double s = x[q];
        long t0 = q - w < 0 ? 0 : q - w;
        for (long t = t0; t < q; ++t)
            s -= L[q * (w + 1) + (t - q + w)] * x[t];
        x[q] = s / L[q * (w + 1) + w];
    }
    for (long q = m - 1; q >= 0; --q) {
        double s = x[q];
        long t1 = q + w >= m ? m - 1 : q + w;
        for (long t = q + 1; t <= t1; ++t)
            s -= L[t * (w + 1) + (q - t + w)] * x[t];
        x[q] = s / L[q * (w + 1) + w];
    }
}

/* out = M^{-1} r for the xy-plane partition. */
void orc_plane_minv(int nx, int ny, int nz, const double *L, const double *r, double *out)
{
    long m = (long)nx * ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        if (out != r)
            memcpy(out + k * m, r + k * m, sizeof(double) * (size_t)m);
        orc_plane_solve(nx, ny, L, out + k * m);
    }
}

/* Damped block Jacobi with xy-plane blocks: r = b - A u, d = M_plane^{-1} r, v = u + omega d. */
void orc_plane_jacobi(int nx, int ny, int nz, double ax, double ay, double az, double omega,
                      const double *L, const double *u, const double *b, double *v,
                      double *work)
{
    long n = (long)nx * ny * nz;
    orc_residual(nx, ny, nz, ax, ay, az, u, b, work);
    orc_plane_minv(nx, ny, nz, L, work, work);
#pragma omp parallel for schedule(static)
    for (long t = 0; t < n; ++t)
        v[t] = u[t] + omega * work[t];
}

/*
 * Block Gauss-Seidel with xy-plane blocks, planes visited one at a time reading the
 * newest values.  order 0: k ascending; 1: k descending; 2: zebra (even k, then odd k).
 * `work` is caller scratch of nx*ny doubles.
 */
void orc_plane_gs(int nx, int ny, int nz, double ax, double ay, double az, double omega,
                  int order, const double *L, double *u, const double *b, double *work)
{
    long m = (long)nx * ny;
    for (int s = 0; s < nz; ++s) {
        int k;
        if (order == 1)
            k = nz - 1 - s;
        else if (order == 2)
            k = (s < (nz + 1) / 2) ? 2 * s : 2 * (s - (nz + 1) / 2) + 1;
        else
            k = s;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                work[i + (long)nx * j] =
                    b[IDX(i, j, k)] - stencil_at(u, nx, ny, nz, ax, ay, az, i, j, k);
        orc_plane_solve(nx, ny, L, work);
        for (long q = 0; q < m; ++q)
            u[(long)k * m + q] += omega * work[q];
    }
}

/*
 * Box blocks (Sec. 2; block sizes of Sec. 3; inversion of Sec. 4.3).  The grid is cut
 * into spatial blocks of bx*by*bz cells, every grid dimension a multiple of the block
 * dimension (the case in which one inverse serves every block, Sec. 4.3).  Inside a block
 * the cells are numbered x fastest, l = lx + bx*(ly + by*lz), n = bx*by*bz.
 *
 * The diagonal block A_b of A is the same for every block: the 7-point stencil restricted
 * to the block's cells (couplings leaving the block dropped).  Its inverse Ahat_b is
 * computed once (Sec. 4.3), here by a dense Cholesky factorisation A_b = L L^T followed by
 * the two triangular solves for every unit vector.  Ainv is n*n, row major.
 * `work` is caller scratch of n*n doubles.  Returns 0, or -1 if a pivot is not positive.
 */
int orc_box_inverse(int bx, int by, int bz, double ax, double ay, double az, double *Ainv,
                    double *work)
{
    int n = bx * by * bz;
    double *L = work;
    /* assemble A_b into L (lower part is overwritten by the factor) */
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            int rx = r % bx, ry = (r / bx) % by, rz = r / (bx * by);
            int cx = c % bx, cy = (c / bx) % by, cz = c / (bx * by);
            double a = 0.0;
            if (r == c)
                a = 2.0 * (ax + ay + az);
            else if (ry == cy && rz == cz && (rx - cx == 1 || cx - rx == 1))
                a = -ax;
            else if (rx == cx && rz == cz && (ry - cy == 1 || cy - ry == 1))
                a = -ay;
            else if (rx == cx && ry == cy && (rz - cz == 1 || cz - rz == 1))
                a = -az;
            L[(long)r * n + c] = a;
        }
    /* Cholesky, column by column (Cholesky-Banachiewicz) */
    for (int r = 0; r < n; ++r)
        for (int c = 0; c <= r; ++c) {
            double s = L[(long)r * n + c];
            for (int t = 0; t < c; ++t)
                s -= L[(long)r * n + t] * L[(long)c * n + t];
            if (c < r) {
                L[(long)r * n + c] = s / L[(long)c * n + c];
            } else {
                if (!(s > 0.0))
                    return -1;
                L[(long)r * n + r] = sqrt(s);
            }
        }
    /* column c of the inverse: L y = e_c, then L^T x = y */
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int c = 0; c < n; ++c) {
        for (int r = 0; r < n; ++r) {
            double s = (r == c) ? 1.0 : 0.0;
            for (int t = 0; t < r; ++t)
                s -= L[(long)r * n + t] * y[t];
            y[r] = s / L[(long)r * n + r];
        }
        for (int r = n - 1; r >= 0; --r) {
            double s = y[r];
            for (int t = r + 1; t < n; ++t)
                s -= L[(long)t * n + r] * Ainv[(long)t * n + c];
            Ainv[(long)r * n + c] = s / L[(long)r * n + r];
        }
    }
    free(y);
    return 0;
}

/* Grid index of local cell l of the block with block coordinates (bi, bj, bk). */
static long box_cell(int nx, int ny, int bx, int by, int bz, int bi, int bj, int bk, int l)
{
    int lx = l % bx, ly = (l / bx) % by, lz = l / (bx * by);
    return IDX(bi * bx + lx, bj * by + ly, bk * bz + lz);
}

/* out = M^{-1} r for the box partition: for every block d_b = Ahat_b r_b (the dense
 * matrix-vector product of Alg. 2 step 2).  out may equal r. */
void orc_box_minv(int nx, int ny, int nz, int bx, int by, int bz, const double *Ainv,
                  const double *r, double *out)
{
    int n = bx * by * bz;
    int nbx = nx / bx, nby = ny / by, nbz = nz / bz;
    long nblk = (long)nbx * nby * nbz;
#pragma omp parallel
    {
        double *rb = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        double *db = rb + n;
#pragma omp for schedule(static)
        for (long q = 0; q < nblk; ++q) {
            int bi = (int)(q % nbx), bj = (int)((q / nbx) % nby), bk = (int)(q / ((long)nbx * nby));
            for (int l = 0; l < n; ++l)
                rb[l] = r[box_cell(nx, ny, bx, by, bz, bi, bj, bk, l)];
            for (int l = 0; l < n; ++l) {
                double s = 0.0;
                for (int m = 0; m < n; ++m)
                    s += Ainv[(long)l * n + m] * rb[m];
                db[l] = s;
            }
            for (int l = 0; l < n; ++l)
                out[box_cell(nx, ny, bx, by, bz, bi, bj, bk, l)] = db[l];
        }
        free(rb);
    }
}

/*
 * Damped block Jacobi with box blocks (Alg. 2): r = b - A u, d_b = Ahat_b r_b for every
 * block, v = u + omega d.  `work` is caller scratch of nx*ny*nz doubles.
 */
void orc_box_jacobi(int nx, int ny, int nz, int bx, int by, int bz, double ax, double ay,
                    double az, double omega, const double *Ainv, const double *u,
                    const double *b, double *v, double *work)
{
    long n = (long)nx * ny * nz;
    orc_residual(nx, ny, nz, ax, ay, az, u, b, work);
    orc_box_minv(nx, ny, nz, bx, by, bz, Ainv, work, work);
#pragma omp parallel for schedule(static)
    for (long t = 0; t < n; ++t)
        v[t] = u[t] + omega * work[t];
}

/*
 * Block Gauss-Seidel with box blocks (Eq. sm:blockm, Alg. 1 with a fixed visiting order):
 * the blocks are visited one at a time, each reading the newest values,
 *   r_b = b_b - (A u)_b,  u_b <- u_b + omega * Ahat_b r_b.
 * order 0: lexicographic in (bk, bj, bi) with bi fastest; 1: reverse lexicographic;
 * 2: two colours, blocks with bi+bj+bk even first, then odd, each colour lexicographic.
 */
void orc_box_gs(int nx, int ny, int nz, int bx, int by, int bz, double ax, double ay,
                double az, double omega, int order, const double *Ainv, double *u,
                const double *b)
{
    int n = bx * by * bz;
    int nbx = nx / bx, nby = ny / by, nbz = nz / bz;
    long nblk = (long)nbx * nby * nbz;
    long *seq = (long *)malloc(sizeof(long) * (size_t)nblk);
    long cnt = 0;
    if (order == 2) {
        for (int colour = 0; colour < 2; ++colour)
            for (long q = 0; q < nblk; ++q) {
                long s = q % nbx + (q / nbx) % nby + q / ((long)nbx * nby);
                if ((int)(s & 1) == colour)
                    seq[cnt++] = q;
            }
    } else {
        for (long q = 0; q < nblk; ++q)
            seq[q] = (order == 1) ? nblk - 1 - q : q;
    }
    double *rb = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    double *db = rb + n;
    for (long s = 0; s < nblk; ++s) {
        long q = seq[s];
        int bi = (int)(q % nbx), bj = (int)((q / nbx) % nby), bk = (int)(q / ((long)nbx * nby));
        for (int l = 0; l < n; ++l) {
            int i = bi * bx + l % bx, j = bj * by + (l / bx) % by, k = bk * bz + l / (bx * by);
            rb[l] = b[IDX(i, j, k)] - stencil_at(u, nx, ny, nz, ax, ay, az, i, j, k);
        }
        for (int l = 0; l < n; ++l) {
            double acc = 0.0;
            for (int m = 0; m < n; ++m)
                acc += Ainv[(long)l * n + m] * rb[m];
            db[l] = acc;
        }
        for (int l = 0; l < n; ++l)
            u[box_cell(nx, ny, bx, by, bz, bi, bj, bk, l)] += omega * db[l];
    }
    free(rb);
    free(seq);
}

/*
 * A level of patches (Sec. 2: "the ghost cells between patches are updated in a Jacobi
 * fashion at the end of a complete smoothing step over all patches").  Patch p has dims
 * (nx, ny, nz) = dims[3p..3p+2], its cells at off[p] in the packed arrays (x fastest), and
 * face neighbours nbr[6p + f] for f = -x, +x, -y, +y, -z, +z (a patch index, or -1 for the
 * physical boundary, whose ghost values are zero).  Two patches that share a face have the
 * same extent along the face.
 *
 * One smoothing step of the level: every patch is smoothed with its ghost layer fixed at
 * the neighbours' values from before the step; the ghost values enter the patch's
 * right-hand side, b_eff = b + a_d * ghost on the patch's boundary cells (the stencil's
 * coupling to a cell outside the patch moved to the right-hand side).  Each patch is then
 * one x-line block-Jacobi sweep (method 0) or one lexicographic x-line block Gauss-Seidel
 * sweep (method 1) with zero values outside it.  `u` is read, `v` receives the new level
 * iterate (u and v distinct); `work` holds max-patch-size * 2 doubles.
 */
static double ghost(const double *u, const long *off, const int *dims, int q, int i, int j,
                    int k)
{
    int qx = dims[3 * q], qy = dims[3 * q + 1];
    return u[off[q] + (long)i + (long)qx * ((long)j + (long)qy * k)];
}

void orc_level_sweep(int npatch, const int *dims, const int *nbr, const long *off, double ax,
                     double ay, double az, double omega, int method, const double *u,
                     const double *b, double *v, double *work)
{
    for (int p = 0; p < npatch; ++p) {
        int nx = dims[3 * p], ny = dims[3 * p + 1], nz = dims[3 * p + 2];
        long n = (long)nx * ny * nz;
        double *beff = work, *up = work + n;
        const int *nb = nbr + 6 * p;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double s = b[off[p] + IDX(i, j, k)];
                    if (i == 0 && nb[0] >= 0)
                        s += ax * ghost(u, off, dims, nb[0], dims[3 * nb[0]] - 1, j, k);
                    if (i == nx - 1 && nb[1] >= 0)
                        s += ax * ghost(u, off, dims, nb[1], 0, j, k);
                    if (j == 0 && nb[2] >= 0)
                        s += ay * ghost(u, off, dims, nb[2], i, dims[3 * nb[2] + 1] - 1, k);
                    if (j == ny - 1 && nb[3] >= 0)
                        s += ay * ghost(u, off, dims, nb[3], i, 0, k);
                    if (k == 0 && nb[4] >= 0)
                        s += az * ghost(u, off, dims, nb[4], i, j, dims[3 * nb[4] + 2] - 1);
                    if (k == nz - 1 && nb[5] >= 0)
                        s += az * ghost(u, off, dims, nb[5], i, j, 0);
                    beff[IDX(i, j, k)] = s;
                }
        if (method == 0) {
            double *res = (double *)malloc(sizeof(double) * (size_t)n);
            orc_line_jacobi(nx, ny, nz, ax, ay, az, omega, u + off[p], beff, v + off[p], res);
            free(res);
        } else {
            memcpy(up, u + off[p], sizeof(double) * (size_t)n);
            orc_line_gs(nx, ny, nz, ax, ay, az, omega, 0, up, beff);
            memcpy(v + off[p], up, sizeof(double) * (size_t)n);
        }
    }
}
