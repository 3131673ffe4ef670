// xy-plane block path (plane.cu): setup, teardown and one sweep launch.
#pragma once
#include "brs_internal.cuh"

int plane_setup(brs_ctx* c);
void plane_teardown(brs_ctx* c);
int plane_sweep_launch(brs_ctx* c, const void* uin, void* uout, const void* b, cudaStream_t s);
// nsweeps plane sweeps of u in place, carried out in the x-sine basis (transform in, mode-line
// sweeps, transform out).  BRS_ERR_UNSUPPORTED when the context has no such form; the caller
// then runs the per-sweep form.  u_zero: u holds zeros on entry (its transform is skipped).
int plane_modes_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, cudaStream_t s,
                      bool u_zero = false);

// FP64 mode-line sweep with the twisted elimination (plane_modes_f64.cu): arrays [k][y][p];
// one Jacobi sweep from uin into out (z in out), or (colour 0 / 1) the in-place update of
// the planes k % 2 == colour (z in the scratch array zs).  Tables per mode p: fm[s][p],
// fb[s][p] (s < ny - 1 - (ny-1)/2), gm[p], gb[p]; bs holds b^ scaled by omega pv.
int mode_twist_launch(const double* uin, double* out, double* zs, const double* bs,
                      const double* fm, const double* fb, const double* gm, const double* gb,
                      int nx, int ny, int nz, double omega, int colour, cudaStream_t s);

// FP64 x-DST along the rows of [nz][ny][nx] arrays by the sine basis's even/odd symmetry
// (plane_modes_f64.cu): out[k][y][p] = sum_x S[p][x] u[k][y][x] (times scale[y][p] if set),
// and the inverse out[k][y][x] = sum_p S[x][p] uh[k][y][p].  Se / So: S's even / odd rows on
// the first ceil(nx/2) / floor(nx/2) columns; SeT / SoT their transposes.  work arrays: grid
// sized.
int dst_fold_forward(const double* u, double* out, const double* scale, double* work,
                     const double* Se, const double* So, int nx, int ny, int nz, cudaStream_t s);
int dst_fold_inverse(const double* uh, double* out, double* work1, double* work2,
                     const double* SeT, const double* SoT, int nx, int ny, int nz, cudaStream_t s);

// Mode-line sweeps of the x-sine form (plane_modes.cu): lines of ny cells along y, one row per
// x-mode (nm rows), nz planes, array layout [k][p][y].
struct ModeCfg {
    int ny = 0, nm = 0, nz = 0, dtype = 0;
    int E = 0, G = 0;     // cells per lane, lanes per line
    int JT = 0, NS = 0;   // rows per CTA tile, ring stages
    int pieces = 1, bx = 0;
    long long total = 0;  // tiles * nz plane-steps
    int grid = 0;
    size_t smem = 0;
    int tab_len = 0;      // factor-table entries per mode (scan_table_len(E, G, false))
};
// Launch configuration for the TMA ring kernel; BRS_ERR_UNSUPPORTED when the rows cannot be
// staged by TMA (ny * element size not a multiple of 16 bytes, or ny not whole lane chunks).
int mode_config(int ny, int nm, int nz, int dtype, int device, ModeCfg* out);
// Tensor map of an [nz][nm][ny] array with the kernel's box (bx, JT, 1).
int mode_encode_map(const ModeCfg& m, CUtensorMap* map, const void* ptr);
// One sweep from the array of `mu`: Jacobi into `out` (colour < 0), the in-place update of the
// planes with k % 2 == colour (colour 0 or 1), or the whole two-colour sweep, even planes then
// odd planes, into `out` (colour 2).  tab: nm tables of tab_len entries (omega folded in).
int mode_sweep_launch(const ModeCfg& m, const CUtensorMap* mu, const CUtensorMap* mb, void* out,
                      const void* tab, double az, double omega, int colour, int* status,
                      cudaStream_t s);
