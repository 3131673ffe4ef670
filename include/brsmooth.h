/*
 * brsmooth -- block-relaxation sweeps for 3D constant-coefficient 7-point stencils on one
 * NVIDIA GB300 (sm_103a).  C ABI: plain pointers and sizes, no C++ or framework types.
 *
 * Problem (Sec. 1.1, Eq. stencil3d7, with per-axis coefficients):
 *   (A u)_ijk = 2(ax+ay+az) u_ijk - ax(u_{i-1,j,k}+u_{i+1,j,k})
 *               - ay(u_{i,j-1,k}+u_{i,j+1,k}) - az(u_{i,j,k-1}+u_{i,j,k+1}) = b_ijk
 * on an nx*ny*nz grid of interior unknowns with Dirichlet values at the ghost indices
 * -1 and n of each axis.  The library treats those values as zero; a caller with
 * non-zero boundary data adds a_d * g to b on the adjacent cells (b = h^2 f + boundary).
 *
 * One sweep (Sec. 2, Eq. blockiteration2):  u <- u + omega * M^{-1} (b - A u)
 * with M the block diagonal of A for full x-line blocks (M_line = tridiag(-ax,
 * 2(ax+ay+az), -ax), one block per (j,k)), full y-line or z-line blocks (the same with the
 * axes exchanged), full xy-plane blocks (M_plane = ax Tx (x) I
 * + ay I (x) Ty + 2 az I, one block per k) or bx*by*bz boxes (the spatial blocks of
 * Sec. 2 and Sec. 3: M_box = the stencil restricted to the box's cells, inverted once
 * (Sec. 4.3) and applied as a dense product, Alg. 2 step 2).  Every block is solved
 * exactly.  Box-block Gauss-Seidel visits the boxes in two colours (bi+bj+bk even, then
 * odd): each colour reads the other colour's newest values, one admissible order of
 * the chaotic scheme, and the result is deterministic.  Updates are
 * damped block Jacobi (Sec. 2, Alg. 2: new values into a second buffer, then swap) or
 * chaotic block Gauss-Seidel (Sec. 2, Alg. 1: in place, blocks processed concurrently
 * with no ordering; a block may read its neighbours' old or new values).
 *
 * Memory layout of every grid array: interior cells only, x fastest,
 *   idx = i + nx*(j + ny*k), dtype as selected (double or float), contiguous.
 * Arrays passed to the *_sweep / *_residual calls are DEVICE pointers (e.g. from
 * cudaMalloc or a torch CUDA tensor) aligned to 16 bytes, owned by the caller.
 * `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 * All work is enqueued on `stream` and returns before it completes, unless stated.
 *
 * Errors: every call returns 0 (BRS_OK) or a negative code; nothing aborts, exits or
 * throws.  Device-side faults detected by the kernels (a bounded wait that ran out)
 * set a sticky status read by brsmooth_last_error() and returned by the next call
 * on the same context.
 */
#ifndef BRSMOOTH_H
#define BRSMOOTH_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define BRS_OK 0
#define BRS_ERR_ARG (-1)         /* bad dims, coefficient, pointer, alignment or count */
#define BRS_ERR_UNSUPPORTED (-2) /* valid request this build does not implement */
#define BRS_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define BRS_ERR_NOMEM (-4)       /* device or host allocation failed */
#define BRS_ERR_TIMEOUT (-5)     /* a bounded device-side wait ran out */
#define BRS_ERR_BOUNDS (-6)      /* a device-side index check failed */

/* Block shape (Sec. 2, block partition of A): full lines along x, y or z, full xy-planes,
 * or bx*by*bz boxes. */
#define BRS_XLINE 0
#define BRS_XYPLANE 1
#define BRS_BOX 2 /* bx*by*bz spatial blocks with one precomputed inverse (Sec. 2, Sec. 4.3) */
#define BRS_YLINE 3 /* lines along y: the blocks for y-dominant coefficients */
#define BRS_ZLINE 4 /* lines along z: the blocks for z-dominant coefficients */

/* Update scheme between blocks. */
#define BRS_JACOBI 0     /* damped block Jacobi, paper default omega = 0.8 (Sec. 2.1) */
#define BRS_CHAOTIC_GS 1 /* chaotic block Gauss-Seidel, paper default omega = 1.0 (Sec. 2.1) */

/* Arithmetic type of u, b and the sweep. */
#define BRS_F64 0
#define BRS_F32 1

/* Plane-solve arithmetic (xy-plane blocks only). */
#define BRS_PLANE_AUTO 0   /* F64: FP64 SIMT;  F32: 3xTF32 tensor cores */
#define BRS_PLANE_SIMT 1   /* CUDA-core FMA in the context dtype */
#define BRS_PLANE_TF32 2   /* one TF32 tensor-core pass per contraction (F32 only) */
#define BRS_PLANE_3XTF32 3 /* split-TF32: hi*hi + hi*lo + lo*hi (F32 only) */

typedef struct brs_ctx brs_ctx; /* opaque; owned by the library */

typedef struct brs_params {
    int nx, ny, nz;     /* interior cells per axis, each >= 1 */
    double ax, ay, az;  /* stencil coefficients, each > 0 and finite */
    int block;          /* BRS_XLINE, BRS_XYPLANE, BRS_BOX, BRS_YLINE or BRS_ZLINE */
    int method;         /* BRS_JACOBI or BRS_CHAOTIC_GS */
    int dtype;          /* BRS_F64 or BRS_F32 */
    double omega;       /* relaxation weight in (0, 2); <= 0 selects the paper default */
    int plane_math;     /* BRS_PLANE_*: arithmetic of the plane and box block solves
                           (ignored for x-line blocks) */
    int bx, by, bz;     /* BRS_BOX only: block dims, each >= 1 and dividing nx, ny, nz;
                           bx*by*bz <= 512 (the paper's blocks run from 2x2x2 to 8x8x8) */
} brs_params;

/*
 * Create a context for one grid shape, coefficient set and method (Sec. 2: the block
 * factorisation is computed once, before the sweeps, and reused; Sec. 4.3).
 * Host-side: validates `p`, factors the block (FP64, rounded to dtype) and allocates the
 * device tables and, for block Jacobi, one grid-sized scratch buffer (the second vector
 * of Alg. 2).  Uses the current CUDA device.  On success *out owns those resources until
 * brsmooth_destroy.  Errors: BRS_ERR_ARG (null pointer, dims < 1, non-positive or
 * non-finite coefficient, omega >= 2, unknown enum), BRS_ERR_UNSUPPORTED
 * (e.g. TF32 plane math with BRS_F64, or a grid beyond the implemented maxima:
 * x-lines nx <= 512; xy-planes nx, ny <= 1024; boxes bx*by*bz <= 512, and TF32 box math
 * needs bx*by*bz a multiple of 4 and >= 32), BRS_ERR_NOMEM, BRS_ERR_CUDA.
 * Box blocks (BRS_BOX): bx, by, bz must divide nx, ny, nz (BRS_ERR_ARG otherwise; one
 * inverse then serves every box, Sec. 4.3).  BRS_PLANE_AUTO selects FP64 CUDA-core math
 * for BRS_F64 and, for BRS_F32, split-TF32 tensor cores when bx*by*bz is a multiple of 4
 * and >= 32, else FP32 CUDA cores.
 * y-line and z-line blocks (BRS_YLINE, BRS_ZLINE): the full-extent lines along y or z,
 * solved exactly.  A y-line (z-line) sweep is the x-line sweep of the grid with its axes
 * permuted to (y, x, z) ((z, x, y)) and the coefficients permuted with them, so the
 * context holds an x-line context of that grid and two permuted grid copies (u and b,
 * plus the inner context's Jacobi buffer).  Each brsmooth_sweep call permutes u and b in,
 * runs all its sweeps, and permutes u back: three grid passes per call, whatever nsweeps.
 * Chaotic GS visits the lines in the permuted order.  Limits: the line length (ny or nz)
 * as for x-lines, and nz <= 65535 (y-lines) or ny <= 65535 (z-lines).
 * FP64 x-line blocks: the sweeps run on line-major copies of u and b (cell index i
 * outermost, the lines of each row k split by colour (j+k) mod 2), so the context holds
 * three more buffers of nx*nz*2*ceil(ny/2) doubles and each brsmooth_sweep call copies u
 * and b in and u back (three grid passes per call).  Each line is eliminated from both ends
 * by two threads with pivots factored once (Sec. 2 / Sec. 4.3: invert once, reuse).
 * Chaotic GS on these contexts visits the lines in two colours, j+k even then odd, each
 * colour reading the other colour's newest values: the red-black line order, one
 * admissible order of the chaotic scheme, deterministic.  BRSMOOTH_LINE_SEQ=0 in the
 * environment at creation selects the lane-scan kernel of the FP32 path instead.
 * xy-plane blocks (BRS_XYPLANE): the plane block is diagonalised along x by the
 * orthonormal DST-I.  FP64 contexts, and FP32 contexts where TMA can stage rows of ny
 * elements (ny times 4 bytes a multiple of 16, ny a whole number of the lane chunks of the
 * line solve), also hold the x-sine form of calls of several sweeps: two more grids (b and
 * u transformed; FP32 [k][p][y], FP64 [k][y][p]) and, for chaotic GS, a third.  Such a call
 * transforms b
 * and u once, runs its sweeps as y-line solves per x-mode with the z coupling, and
 * transforms u back; the iterates are the plane sweeps' own in exact arithmetic (the
 * transform commutes with the sweep), rounded differently, so a call of n sweeps is not
 * bitwise equal to n one-sweep calls.  It is taken for calls of at least 3 sweeps on the
 * tensor-core path and at least 2 otherwise (BRSMOOTH_PLANE_MODES_MIN); BRSMOOTH_PLANE_MODES=0
 * in the environment at creation leaves it out.  FP64 solves each y-line by elimination from
 * both ends (BRSMOOTH_MODE_TWIST=0: the lane-scan solve, TMA rows only).  Chaotic GS on plane contexts visits the
 * planes in two colours, even k then odd k, each colour reading the other's newest values.
 */
int brsmooth_create(const brs_params* p, brs_ctx** out);

/*
 * Run `nsweeps` sweeps (Sec. 2, Alg. 1 / Alg. 2) of the context's method on device
 * grid `u` (in/out) with right-hand side `b` (read only), both nx*ny*nz elements of the
 * context dtype.  Block Jacobi ping-pongs between `u` and the context scratch buffer;
 * the final iterate is always left in `u`.  nsweeps == 0 is a no-op.
 * Errors: BRS_ERR_ARG (null ctx/u/b, nsweeps < 0, pointer not 16-byte aligned,
 * u == b), BRS_ERR_CUDA (launch failure), or a sticky device status.
 * Not thread-safe per context; distinct contexts may be used from distinct threads.
 */
int brsmooth_sweep(brs_ctx* c, void* u, const void* b, int nsweeps, void* stream);

/*
 * Residual r = b - A u (Sec. 2, the r^k of Eq. blockiteration2) and its 2-norm.
 * `r` (device, nullable) receives the residual in the context dtype.  `norm2` (host,
 * nullable) receives ||r||_2 accumulated in FP64 in a fixed order (deterministic);
 * when it is non-NULL the call synchronises `stream` before returning.
 * Errors: BRS_ERR_ARG (null ctx/u/b), BRS_ERR_CUDA.
 */
int brsmooth_residual(brs_ctx* c, const void* u, const void* b, void* r, double* norm2,
                      void* stream);

/*
 * Same sweeps as brsmooth_sweep, but `u` and `b` are HOST arrays: the call copies b and
 * u to context-owned device buffers, sweeps, copies u back and synchronises `stream`.
 * Host arrays may be pageable or pinned (pinned is faster).  The device buffers are
 * allocated on first use and kept until destroy.
 * Errors: as brsmooth_sweep, plus BRS_ERR_NOMEM.
 */
int brsmooth_sweep_host(brs_ctx* c, void* u_host, const void* b_host, int nsweeps,
                        void* stream);

/*
 * brsmooth_sweep_host without the final synchronisation: the copies in, the sweeps and the
 * copy of u back are enqueued on `stream` and the call returns.  u_host holds the result
 * once the stream has reached that point (synchronise the stream or an event first), and
 * neither host array may be touched before then.  With pinned host arrays the copies run
 * asynchronously, so a caller with independent problems can keep two contexts on two
 * streams and overlap one problem's copies with the other's sweeps.  Calls on one context
 * must stay on one stream (its device buffers are reused in stream order).
 * Errors: as brsmooth_sweep_host; a device status raised by the sweeps is reported by a
 * later call or brsmooth_last_error.
 */
int brsmooth_sweep_host_async(brs_ctx* c, void* u_host, const void* b_host, int nsweeps,
                              void* stream);

/*
 * Release the context and every device resource it owns.  NULL is accepted (BRS_OK).
 * Synchronises the device work the context enqueued.
 */
int brsmooth_destroy(brs_ctx* c);

/* Sticky device-side status of the context (BRS_OK, BRS_ERR_TIMEOUT, BRS_ERR_BOUNDS);
 * synchronises the context's last stream.  Reading it clears it. */
int brsmooth_last_error(brs_ctx* c);

/* Text of the CUDA runtime error behind the calling thread's most recent BRS_ERR_CUDA or
 * BRS_ERR_NOMEM (static storage; "no error" if there was none); never NULL. */
const char* brsmooth_cuda_error_string(void);

/* Static English text for a status code; never NULL. */
const char* brsmooth_strerror(int code);

/*
 * Many independent patches of one refinement level (Sec. 1.1 patches; Sec. 4.2 mixed patch
 * sizes), swept as one stream of work: every patch uses x-line blocks with the common
 * coefficients, method, dtype and omega of `common` (its nx/ny/nz are ignored).
 * `dims` (host) holds npatch triples (nx, ny, nz), each >= 1, nx <= 128.
 * Packed layout: patch q occupies cells [off_q, off_q + nx*ny*nz) of one array, x fastest
 * within the patch, off_q = sum of the earlier patches' cell counts (no padding).
 * Creation runs the built-in autotuner (z-chunk length, warps per CTA, CTAs per SM),
 * timing candidates on scratch arrays; results are cached per process.
 * Errors: BRS_ERR_ARG (null, npatch < 1, a dim < 1, bad common params),
 * BRS_ERR_UNSUPPORTED (xy-plane blocks, nx > 128), BRS_ERR_NOMEM, BRS_ERR_CUDA.
 */
int brsmooth_create_batched(int npatch, const int* dims, const brs_params* common,
                            brs_ctx** out);

/*
 * `nsweeps` sweeps over every patch of a batched context; u_packed (in/out) and b_packed
 * are DEVICE arrays in the packed layout, 16-byte aligned.  One persistent launch per
 * sweep pulls (patch, y-block, z-chunk) work items from an atomic queue, so uneven
 * patches balance across the GPU.  The sweep sequence of a call is captured into a CUDA
 * graph on the first call with a given (u, b, nsweeps) and replayed as one graph launch
 * on `stream` afterwards (the graph is keyed by the pointers: reuse the same buffers).
 * Block Jacobi ping-pongs with a context buffer and leaves the result in u_packed.
 * Errors: as brsmooth_sweep; BRS_ERR_ARG if `c` is not a batched context.
 */
int brsmooth_sweep_batched(brs_ctx* c, void* u_packed, const void* b_packed, int nsweeps,
                           void* stream);

/*
 * A level of patches (Sec. 2: the ghost cells between patches are updated in a Jacobi
 * fashion at the end of a complete smoothing step over all patches).  As
 * brsmooth_create_batched, plus nbr[6 * npatch] (host): for patch p, nbr[6p + f] is the
 * patch that shares its face f (f = 0..5 for -x, +x, -y, +y, -z, +z) or -1 where the face
 * is the physical boundary (ghost value zero; fold non-zero boundary data into b).  The
 * table must be symmetric (q = nbr[6p + f] >= 0 implies nbr[6q + (f ^ 1)] == p; q == p
 * makes that direction periodic), neighbours across an x face have equal ny and nz (and so
 * on for y and z faces), and every patch dim must be >= 2.  Every step of
 * brsmooth_sweep_batched on a level context smooths each patch with its ghost layer held
 * at the face neighbours' values from before the step (zero on the physical boundary).
 * The ghost layers live in context-owned ghost blocks (the six faces of every patch): the
 * first step of a call gathers them from the iterate, and each later step of the same call
 * reads the faces that the previous step wrote there as it computed them (two ghost
 * arrays, alternating), so a call of n steps equals n calls of one step.  The context
 * holds two ghost arrays, each of 2 (nx ny + nx nz + ny nz) elements per patch (faces
 * rounded up to multiples of 4).  Errors: as brsmooth_create_batched; BRS_ERR_ARG for a
 * null, out-of-range, asymmetric or face-mismatched table or a dim < 2.
 */
int brsmooth_create_level(int npatch, const int* dims, const int* nbr,
                          const brs_params* common, brs_ctx** out);

/*
 * Keep a level's ghost layers across calls of brsmooth_sweep_batched (on != 0) or gather
 * them at every call's first step (on == 0, the default).  Sec. 2 refreshes the ghosts from
 * the face neighbours after every complete step; when on, the last step of a call also
 * writes its faces into the ghost array that the next step reads, and the next call's first
 * step uses them instead of gathering from the iterate.  The caller promises that the
 * iterate the next call receives holds exactly the values the previous call left (nothing
 * else writes it in between); then n calls of m steps equal one call of n m steps.  The
 * first call after switching on gathers.  Errors: BRS_ERR_ARG if `c` is null or not a
 * level context.
 */
int brsmooth_level_keep_ghosts(brs_ctx* c, int on);

/* Launch shape the autotuner chose for a batched context (host outputs). */
int brsmooth_batched_config(const brs_ctx* c, int* kchunk, int* warps_per_cta, int* ctas,
                            int* work_items);

/*
 * Mixed-precision defect correction (iterative refinement around the sweeps of Sec. 2,
 * Eq. blockiteration2): starting from the device FP64 iterate `u` (in/out) and FP64
 * right-hand side `b`, repeat
 *   r = b - A u in FP64 (stored to FP32), stop if ||r||_2 / ||b||_2 <= rtol or after
 *   max_outer corrections; c = 0; `inner_sweeps` sweeps of `inner_f32` on A c = r;
 *   u = u + c in FP64.
 * `outer_f64` must be a BRS_F64 single-grid context and `inner_f32` a BRS_F32 one with
 * the same dims and coefficients (either block shape and method).  The inner context owns
 * two FP32 grid buffers allocated on first use.  Host outputs (each nullable):
 * *outer_done = corrections applied, *rel_residual = final ||r||/||b||, history[i] =
 * ||r||/||b|| before correction i (max_outer + 1 entries).  Synchronises `stream` once
 * per outer step (to read the norm).  Errors: BRS_ERR_ARG (mismatched or wrong-dtype
 * contexts, null or misaligned arrays, inner_sweeps < 1, max_outer < 0, rtol < 0),
 * BRS_ERR_NOMEM, BRS_ERR_CUDA.
 */
int brsmooth_defect_correction(brs_ctx* outer_f64, brs_ctx* inner_f32, double* u,
                               const double* b, double rtol, int inner_sweeps, int max_outer,
                               int* outer_done, double* rel_residual, double* history,
                               void* stream);

/*
 * One reverse-mode step of damped x-line block Jacobi (the transpose of one sweep of
 * Eq. blockiteration2; A and M are symmetric).  For a loss L of the final iterate, with
 * `lam` = dL/du_{k+1} on entry (device, in/out) and `u_k` the iterate the forward sweep
 * started from (device, read):
 *   mu = M^{-1} lam;   lam <- lam - omega A mu            (= dL/du_k on return)
 *   grad_b[i] += omega mu[i]                               (device array, context dtype)
 *   grad_a[d] += -omega mu . ((dM/da_d) z_k + T_d u_k)     (device double[3]: ax, ay, az)
 * with z_k = M^{-1}(b - A u_k), T_d the second difference along axis d and, for x-line
 * blocks, dM/dax = Tx, dM/day = dM/daz = 2I.  Calls for sweeps K-1 .. 0 in that order
 * give dL/du_0 in `lam`, dL/db in grad_b and dL/da in grad_a.  The context owns one more
 * grid buffer and reduction scratch, allocated on first use; the Jacobi scratch buffer
 * is reused.  Errors: BRS_ERR_ARG (null), BRS_ERR_UNSUPPORTED (not a single-grid x-line
 * block-Jacobi context), BRS_ERR_NOMEM, BRS_ERR_CUDA.
 */
int brsmooth_adjoint_sweep(brs_ctx* c, void* lam, const void* u_k, const void* b,
                           void* grad_b, double* grad_a, void* stream);

/*
 * Allocation-free x-line block-Jacobi sweeps (no counterpart in the paper; a deployment
 * convenience).  brsmooth_create allocates device memory, and some callers cannot: their
 * device memory belongs entirely to another allocator (a framework's caching pool or a
 * fixed budget), or they run latency-sensitive loops where cudaMalloc/cudaFree and the
 * device-wide synchronisation they imply are not acceptable.  This call needs no context
 * and allocates nothing: the second vector and the line factor tables live in fixed
 * file-scope device arrays of the library, sized for BRSMOOTH_NOALLOC_MAX_CELLS cells
 * (8 MiB plus 32 KiB, held by every GPU that loads the library until the process exits).
 * The factor tables are built on the device by a one-thread kernel from the coefficients,
 * so the call copies nothing from the host and only enqueues work on `stream`.
 * It computes what brsmooth_sweep computes for a BRS_XLINE / BRS_JACOBI context with the
 * same dims, coefficients, omega (<= 0 selects 0.8) and dtype, with the lane-scan line
 * kernel: `nsweeps` sweeps on device grid `u` (in/out) with right-hand side `b`, the
 * result left in `u`.
 * The first call on each device looks up the arrays' device addresses (with that device
 * current); make that first call before any stream capture.  Later calls may be captured
 * into a CUDA graph: a call enqueues only kernels and a device-to-device copy, and a
 * replay recomputes the tables from the captured coefficients.  All calls share the arrays
 * and each call rewrites what it uses (tables and second vector are fully overwritten, so
 * nothing carries over); calls whose GPU work overlaps (different streams or threads)
 * race on them.  Errors: BRS_ERR_ARG (dims < 1, null, misaligned or aliased arrays,
 * nsweeps < 0, non-positive or non-finite coefficients, non-finite omega or omega >= 2,
 * bad dtype), BRS_ERR_UNSUPPORTED (nx*ny*nz greater than BRSMOOTH_NOALLOC_MAX_CELLS, or
 * nx > 512), BRS_ERR_CUDA.
 */
#define BRSMOOTH_NOALLOC_MAX_CELLS (1 << 20)
int brsmooth_line_jacobi_noalloc(int nx, int ny, int nz, double ax, double ay, double az,
                                 double omega, int dtype, void* u, const void* b, int nsweeps,
                                 void* stream);

/*
 * Diagnostic for the failure-detection path: enqueues one CTA that waits on a device-side
 * barrier nothing ever signals, using the same bounded wait as the sweep kernels; after
 * `limit_ns` (0 .. 1e9) it records BRS_ERR_TIMEOUT in the context's sticky status and
 * returns normally (no trap, no fault).  The next call on the context then returns
 * BRS_ERR_TIMEOUT until brsmooth_last_error() reads and clears it.
 * Errors: BRS_ERR_ARG (null context or limit out of range), BRS_ERR_CUDA.
 */
int brsmooth_selftest_wait(brs_ctx* c, long long limit_ns, void* stream);

/*
 * Measurement helper (no counterpart in the paper): enqueues `blocks` CTAs of 256 threads,
 * each thread running `iters` iterations of 8 independent FP64 fused multiply-adds, and
 * writes one double per thread to the device array `out` (blocks * 256 elements, caller
 * owned).  blocks * 256 * iters * 8 FMAs in total: timed with events on `stream`, this is
 * the FP64 FMA rate of the GPU, the roof of the FP64 x-line sweeps.
 * Errors: BRS_ERR_ARG (null out, blocks < 1, iters < 1), BRS_ERR_CUDA.
 */
int brsmooth_probe_fp64_fma(double* out, int blocks, int iters, void* stream);

/* Number of cell updates one sweep performs (nx*ny*nz summed over patches). */
long long brsmooth_cells(const brs_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* BRSMOOTH_H */
