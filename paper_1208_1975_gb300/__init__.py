"""brsmooth: block-relaxation sweeps for 3D constant-coefficient 7-point stencils on GB300.

Thin Python binding over the C ABI in ``include/brsmooth.h`` (argument marshalling only:
every step of a sweep runs in the CUDA library ``_build/libbrsmooth.so``).  Functions
carry the C names; :class:`Context` wraps one ``brs_ctx``.  Grid arrays are torch CUDA
tensors of shape (nz, ny, nx) (x fastest), float64 or float32, contiguous.

The library is required: if it has not been built (``build()``) or cannot be loaded,
every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "libbrsmooth.so"

BRS_OK = 0
BRS_ERR_ARG = -1
BRS_ERR_UNSUPPORTED = -2
BRS_ERR_CUDA = -3
BRS_ERR_NOMEM = -4
BRS_ERR_TIMEOUT = -5
BRS_ERR_BOUNDS = -6

BRS_XLINE, BRS_XYPLANE, BRS_BOX, BRS_YLINE, BRS_ZLINE = 0, 1, 2, 3, 4
BRS_JACOBI, BRS_CHAOTIC_GS = 0, 1
BRS_F64, BRS_F32 = 0, 1
BRS_PLANE_AUTO, BRS_PLANE_SIMT, BRS_PLANE_TF32, BRS_PLANE_3XTF32 = 0, 1, 2, 3

BLOCKS = {"line": BRS_XLINE, "plane": BRS_XYPLANE, "box": BRS_BOX, "yline": BRS_YLINE,
          "zline": BRS_ZLINE}
METHODS = {"jacobi": BRS_JACOBI, "gs": BRS_CHAOTIC_GS, "chaotic_gs": BRS_CHAOTIC_GS}
DTYPES = {"f64": BRS_F64, "f32": BRS_F32}
PLANE_MATH = {"auto": BRS_PLANE_AUTO, "simt": BRS_PLANE_SIMT, "tf32": BRS_PLANE_TF32,
              "3xtf32": BRS_PLANE_3XTF32}


class BrsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {brsmooth_strerror(code)} ({code})"
        if code in (BRS_ERR_CUDA, BRS_ERR_NOMEM):
            msg += f": {brsmooth_cuda_error_string()}"
        super().__init__(msg)


class brs_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ax", ctypes.c_double), ("ay", ctypes.c_double), ("az", ctypes.c_double),
                ("block", ctypes.c_int), ("method", ctypes.c_int), ("dtype", ctypes.c_int),
                ("omega", ctypes.c_double), ("plane_math", ctypes.c_int),
                ("bx", ctypes.c_int), ("by", ctypes.c_int), ("bz", ctypes.c_int)]


_lib = None


def build(verbose: bool = False) -> Path:
    """Compile the CUDA library for sm_103a (nvcc; works without a GPU)."""
    from . import builder as _b

    return _b.build(verbose=verbose)


def lib():
    """The loaded CUDA library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_1208_1975_gb300.build())")
    L = ctypes.CDLL(str(LIB_PATH))
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.brsmooth_create.argtypes = [ctypes.POINTER(brs_params), ctypes.POINTER(P)]
    L.brsmooth_sweep.argtypes = [P, P, P, I, P]
    L.brsmooth_residual.argtypes = [P, P, P, P, ctypes.POINTER(D), P]
    L.brsmooth_sweep_host.argtypes = [P, P, P, I, P]
    L.brsmooth_sweep_host_async.argtypes = [P, P, P, I, P]
    L.brsmooth_destroy.argtypes = [P]
    L.brsmooth_last_error.argtypes = [P]
    L.brsmooth_strerror.argtypes = [I]
    L.brsmooth_strerror.restype = ctypes.c_char_p
    L.brsmooth_cuda_error_string.argtypes = []
    L.brsmooth_cuda_error_string.restype = ctypes.c_char_p
    L.brsmooth_cells.argtypes = [P]
    L.brsmooth_cells.restype = ctypes.c_longlong
    L.brsmooth_create_batched.argtypes = [I, P, ctypes.POINTER(brs_params), ctypes.POINTER(P)]
    L.brsmooth_sweep_batched.argtypes = [P, P, P, I, P]
    L.brsmooth_create_level.argtypes = [I, P, P, ctypes.POINTER(brs_params), ctypes.POINTER(P)]
    L.brsmooth_create_level.restype = I
    IP = ctypes.POINTER(ctypes.c_int)
    L.brsmooth_batched_config.argtypes = [P, IP, IP, IP, IP]
    L.brsmooth_level_keep_ghosts.argtypes = [P, I]
    L.brsmooth_level_keep_ghosts.restype = I
    DP = ctypes.POINTER(D)
    L.brsmooth_defect_correction.argtypes = [P, P, P, P, D, I, I, IP, DP, DP, P]
    L.brsmooth_defect_correction.restype = I
    L.brsmooth_adjoint_sweep.argtypes = [P, P, P, P, P, P, P]
    L.brsmooth_adjoint_sweep.restype = I
    for name in ("brsmooth_create", "brsmooth_sweep", "brsmooth_residual", "brsmooth_sweep_host",
                 "brsmooth_sweep_host_async",
                 "brsmooth_destroy", "brsmooth_last_error", "brsmooth_create_batched",
                 "brsmooth_sweep_batched", "brsmooth_batched_config"):
        getattr(L, name).restype = I
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != BRS_OK:
        raise BrsError(rc, where)


def _stream_handle(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t, dtype_code: int, cells: int, name: str):
    """Device pointer of a contiguous CUDA tensor of the context dtype and size."""
    import torch

    want = torch.float64 if dtype_code == BRS_F64 else torch.float32
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != want or not t.is_contiguous() or t.numel() != cells:
        raise ValueError(f"{name}: need a contiguous {want} tensor with {cells} elements")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ C-named functions

def brsmooth_strerror(code: int) -> str:
    return lib().brsmooth_strerror(int(code)).decode()


def brsmooth_cuda_error_string() -> str:
    return lib().brsmooth_cuda_error_string().decode()


def brsmooth_create(p: brs_params):
    h = ctypes.c_void_p()
    rc = lib().brsmooth_create(ctypes.byref(p), ctypes.byref(h))
    return rc, h


def brsmooth_sweep(ctx, u_ptr, b_ptr, nsweeps: int, stream) -> int:
    return lib().brsmooth_sweep(ctx, u_ptr, b_ptr, int(nsweeps), ctypes.c_void_p(stream))


def brsmooth_residual(ctx, u_ptr, b_ptr, r_ptr, want_norm: bool, stream):
    nrm = ctypes.c_double(0.0)
    rc = lib().brsmooth_residual(ctx, u_ptr, b_ptr, r_ptr, ctypes.byref(nrm) if want_norm else None,
                                 ctypes.c_void_p(stream))
    return rc, nrm.value


def brsmooth_sweep_host(ctx, u_host_ptr, b_host_ptr, nsweeps: int, stream) -> int:
    return lib().brsmooth_sweep_host(ctx, u_host_ptr, b_host_ptr, int(nsweeps), ctypes.c_void_p(stream))


def brsmooth_sweep_host_async(ctx, u_host_ptr, b_host_ptr, nsweeps: int, stream) -> int:
    return lib().brsmooth_sweep_host_async(ctx, u_host_ptr, b_host_ptr, int(nsweeps),
                                           ctypes.c_void_p(stream))


def brsmooth_destroy(ctx) -> int:
    return lib().brsmooth_destroy(ctx)


def brsmooth_last_error(ctx) -> int:
    return lib().brsmooth_last_error(ctx)


def brsmooth_cells(ctx) -> int:
    return int(lib().brsmooth_cells(ctx))


def brsmooth_create_batched(dims, p: brs_params):
    import numpy as np

    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1))
    h = ctypes.c_void_p()
    rc = lib().brsmooth_create_batched(len(d) // 3, ctypes.c_void_p(d.ctypes.data), ctypes.byref(p),
                                       ctypes.byref(h))
    return rc, h


def brsmooth_create_level(dims, nbr, p: brs_params):
    import numpy as np

    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1))
    nb = np.ascontiguousarray(np.asarray(nbr, dtype=np.int32).reshape(-1))
    h = ctypes.c_void_p()
    rc = lib().brsmooth_create_level(len(d) // 3, ctypes.c_void_p(d.ctypes.data),
                                     ctypes.c_void_p(nb.ctypes.data), ctypes.byref(p),
                                     ctypes.byref(h))
    return rc, h


def brsmooth_sweep_batched(ctx, u_ptr, b_ptr, nsweeps: int, stream) -> int:
    return lib().brsmooth_sweep_batched(ctx, u_ptr, b_ptr, int(nsweeps), ctypes.c_void_p(stream))


def brsmooth_level_keep_ghosts(ctx, on: bool) -> int:
    return lib().brsmooth_level_keep_ghosts(ctx, 1 if on else 0)


def brsmooth_batched_config(ctx):
    v = [ctypes.c_int() for _ in range(4)]
    rc = lib().brsmooth_batched_config(ctx, *[ctypes.byref(x) for x in v])
    return rc, tuple(x.value for x in v)


# ------------------------------------------------------------------ convenience wrapper

class Context:
    """One brs_ctx: a grid shape, coefficients, block shape, method and dtype."""

    def __init__(self, nx: int, ny: int, nz: int, a=(1.0, 1.0, 1.0), *, block: str = "line",
                 method: str = "jacobi", dtype: str = "f64", omega: float = 0.0,
                 plane_math: str = "auto", box=(0, 0, 0)):
        """block 'box' takes box=(bx, by, bz); plane_math also selects the box arithmetic."""
        self.shape = (nz, ny, nx)
        self.dtype_code = DTYPES[dtype]
        bx, by, bz = (int(v) for v in box)
        self.p = brs_params(nx, ny, nz, float(a[0]), float(a[1]), float(a[2]), BLOCKS[block],
                            METHODS[method], self.dtype_code, float(omega), PLANE_MATH[plane_math],
                            bx, by, bz)
        rc, h = brsmooth_create(self.p)
        _check(rc, "brsmooth_create")
        self.h = h
        self.cells = nx * ny * nz

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            brsmooth_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sweep(self, u, b, nsweeps: int = 1, stream=None):
        """nsweeps sweeps on CUDA tensors u (in/out) and b; enqueued on `stream`."""
        rc = brsmooth_sweep(self.h, _dptr(u, self.dtype_code, self.cells, "u"),
                            _dptr(b, self.dtype_code, self.cells, "b"), nsweeps, _stream_handle(stream))
        _check(rc, "brsmooth_sweep")
        return u

    def residual(self, u, b, r=None, norm: bool = True, stream=None):
        """r = b - A u into `r` (optional) and ||r||_2 (FP64; synchronises when norm=True)."""
        rp = _dptr(r, self.dtype_code, self.cells, "r") if r is not None else None
        rc, nrm = brsmooth_residual(self.h, _dptr(u, self.dtype_code, self.cells, "u"),
                                    _dptr(b, self.dtype_code, self.cells, "b"), rp, norm,
                                    _stream_handle(stream))
        _check(rc, "brsmooth_residual")
        return nrm if norm else None

    def sweep_host(self, u_host, b_host, nsweeps: int = 1, stream=None, wait: bool = True):
        """Sweeps on host arrays (numpy or CPU tensors, contiguous, context dtype), in place on
        u.  wait=False only enqueues the copies and sweeps on `stream` (brsmooth_sweep_host_async):
        u is valid, and both arrays may be touched again, once the stream has reached it."""
        import numpy as np

        def hptr(x, name):
            if hasattr(x, "data_ptr"):
                if x.is_cuda or not x.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous CPU tensor")
                return ctypes.c_void_p(x.data_ptr()), x.numel(), str(x.dtype)
            if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
                raise ValueError(f"{name} must be a C-contiguous numpy array")
            return ctypes.c_void_p(x.ctypes.data), x.size, str(x.dtype)

        up, un, ud = hptr(u_host, "u")
        bp, bn, bd = hptr(b_host, "b")
        want = "float64" if self.dtype_code == BRS_F64 else "float32"
        if un != self.cells or bn != self.cells or want not in ud or want not in bd:
            raise ValueError(f"host arrays need {self.cells} {want} elements")
        fn = brsmooth_sweep_host if wait else brsmooth_sweep_host_async
        rc = fn(self.h, up, bp, nsweeps, _stream_handle(stream))
        _check(rc, fn.__name__)
        return u_host

    def last_error(self) -> int:
        return brsmooth_last_error(self.h)


def brsmooth_defect_correction(outer, inner, u_ptr, b_ptr, rtol: float, inner_sweeps: int,
                               max_outer: int, stream):
    done = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    hist = (ctypes.c_double * (max_outer + 1))()
    rc = lib().brsmooth_defect_correction(outer, inner, u_ptr, b_ptr, float(rtol), int(inner_sweeps),
                                          int(max_outer), ctypes.byref(done), ctypes.byref(rel), hist,
                                          ctypes.c_void_p(stream))
    return rc, done.value, rel.value, list(hist)[: done.value + 1]


def defect_correction(outer: "Context", inner: "Context", u, b, *, rtol: float = 1e-10,
                      inner_sweeps: int = 32, max_outer: int = 1000, stream=None):
    """Mixed-precision defect correction: FP64 outer residual/correction, FP32 inner sweeps.

    `u` (FP64, in/out) and `b` (FP64) are CUDA tensors of outer's shape.  Returns
    (corrections applied, final ||r||/||b||, history of ||r||/||b||).
    """
    rc, done, rel, hist = brsmooth_defect_correction(
        outer.h, inner.h, _dptr(u, BRS_F64, outer.cells, "u"), _dptr(b, BRS_F64, outer.cells, "b"),
        rtol, inner_sweeps, max_outer, _stream_handle(stream))
    _check(rc, "brsmooth_defect_correction")
    return done, rel, hist


def brsmooth_adjoint_sweep(ctx, lam_ptr, u_ptr, b_ptr, gb_ptr, ga_ptr, stream) -> int:
    return lib().brsmooth_adjoint_sweep(ctx, lam_ptr, u_ptr, b_ptr, gb_ptr, ga_ptr,
                                        ctypes.c_void_p(stream))


def _adjoint_step(c: "Context", lam, u_k, b, gb, ga, stream=None):
    import torch

    if ga.dtype != torch.float64 or not ga.is_cuda or ga.numel() != 3:
        raise ValueError("grad_a must be a CUDA float64 tensor of 3 elements")
    rc = brsmooth_adjoint_sweep(c.h, _dptr(lam, c.dtype_code, c.cells, "lam"),
                                _dptr(u_k, c.dtype_code, c.cells, "u_k"),
                                _dptr(b, c.dtype_code, c.cells, "b"),
                                _dptr(gb, c.dtype_code, c.cells, "grad_b"),
                                ctypes.c_void_p(ga.data_ptr()), _stream_handle(stream))
    _check(rc, "brsmooth_adjoint_sweep")


# Contexts of recent block_smooth shapes, most recent last: creating one allocates and
# uploads tables (synchronising), so repeated calls with the same grid, coefficients and
# dtype reuse it.  An evicted context is destroyed once no autograd graph holds it.
_SMOOTH_CTX = {}


def _smooth_context(nx, ny, nz, av, dt, omega, device=None):
    key = (nx, ny, nz, av, dt, float(omega), device)
    c = _SMOOTH_CTX.pop(key, None)
    if c is None:
        c = Context(nx, ny, nz, av, block="line", method="jacobi", dtype=dt, omega=omega)
    _SMOOTH_CTX[key] = c
    while len(_SMOOTH_CTX) > 2:
        _SMOOTH_CTX.pop(next(iter(_SMOOTH_CTX)))
    return c


def _block_smooth_fn():
    import torch

    class BlockSmoothFn(torch.autograd.Function):
        """u_K = K damped x-line block-Jacobi sweeps from u0 with right-hand side b.

        Differentiable in b, u0 and the coefficients a = (ax, ay, az).  The forward keeps
        the iterate every `ckpt` sweeps; the backward recomputes each segment from its
        checkpoint and runs the library's adjoint sweeps from the last sweep to the first.
        """

        @staticmethod
        def forward(fctx, b, u0, a, nsweeps: int, ckpt: int, omega: float):
            nz, ny, nx = b.shape
            dt = "f64" if b.dtype == torch.float64 else "f32"
            av = tuple(float(x) for x in a.detach().cpu().tolist())
            c = _smooth_context(nx, ny, nz, av, dt, omega, b.device.index)
            b = b.detach().contiguous()
            u = u0.detach().clone().contiguous()
            ckpt = max(1, int(ckpt))
            saved = []
            for k in range(0, nsweeps, ckpt):
                saved.append(u.clone())
                c.sweep(u, b, min(ckpt, nsweeps - k))
            fctx.c, fctx.nsweeps, fctx.ckpt = c, int(nsweeps), ckpt
            fctx.a_meta = (a.dtype, a.device)
            fctx.save_for_backward(b, *saved)
            return u

        @staticmethod
        def backward(fctx, grad_u):
            c, K, ck = fctx.c, fctx.nsweeps, fctx.ckpt
            b, *saved = fctx.saved_tensors
            lam = grad_u.detach().clone().contiguous()
            gb = torch.zeros_like(b)
            ga = torch.zeros(3, dtype=torch.float64, device=b.device)
            for seg in range(len(saved) - 1, -1, -1):
                k0 = seg * ck
                k1 = min(K, k0 + ck)
                us = [saved[seg]]
                for _ in range(k0 + 1, k1):
                    nxt = us[-1].clone()
                    c.sweep(nxt, b, 1)
                    us.append(nxt)
                for k in range(k1 - 1, k0 - 1, -1):
                    _adjoint_step(c, lam, us[k - k0], b, gb, ga)
            adt, adev = fctx.a_meta
            return gb, lam, ga.to(dtype=adt, device=adev), None, None, None

    return BlockSmoothFn


_BSF = None


def block_smooth(b, u0, a, nsweeps: int = 8, *, ckpt: int = 4, omega: float = 0.8):
    """Differentiable K-sweep x-line block Jacobi (see BlockSmoothFn)."""
    global _BSF
    if _BSF is None:
        _BSF = _block_smooth_fn()
    return _BSF.apply(b, u0, a, nsweeps, ckpt, omega)


class BatchedContext:
    """Many patches (x-line blocks, common coefficients/method/dtype) in one packed array."""

    def __init__(self, dims, a=(1.0, 1.0, 1.0), *, method: str = "gs", dtype: str = "f32",
                 omega: float = 0.0, nbr=None):
        """nbr (npatch x 6 face neighbours, -1 = boundary) makes the patches a level with
        ghost exchange after every step (brsmooth_create_level)."""
        import numpy as np

        self.dims = np.asarray(dims, dtype=np.int64).reshape(-1, 3)
        self.dtype_code = DTYPES[dtype]
        p = brs_params(1, 1, 1, float(a[0]), float(a[1]), float(a[2]), BRS_XLINE, METHODS[method],
                       self.dtype_code, float(omega), BRS_PLANE_AUTO)
        if nbr is None:
            rc, h = brsmooth_create_batched(self.dims, p)
            _check(rc, "brsmooth_create_batched")
        else:
            rc, h = brsmooth_create_level(self.dims, nbr, p)
            _check(rc, "brsmooth_create_level")
        self.h = h
        sizes = self.dims.prod(axis=1)
        self.offsets = np.concatenate([[0], np.cumsum(sizes)])
        self.cells = int(self.offsets[-1])

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            brsmooth_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sweep(self, u, b, nsweeps: int = 1, stream=None):
        rc = brsmooth_sweep_batched(self.h, _dptr(u, self.dtype_code, self.cells, "u"),
                                    _dptr(b, self.dtype_code, self.cells, "b"), nsweeps,
                                    _stream_handle(stream))
        _check(rc, "brsmooth_sweep_batched")
        return u

    def keep_ghosts(self, on: bool = True):
        """Level contexts: keep the ghost layers across calls (the caller leaves the iterate
        untouched between calls), so a call's first step does not gather them."""
        _check(brsmooth_level_keep_ghosts(self.h, on), "brsmooth_level_keep_ghosts")
        return self

    def config(self):
        rc, cfg = brsmooth_batched_config(self.h)
        _check(rc, "brsmooth_batched_config")
        return dict(zip(("kchunk", "warps_per_cta", "ctas", "work_items"), cfg))

    def patch(self, arr, q):
        """View of patch q of a packed array as (nz, ny, nx)."""
        nx, ny, nz = (int(v) for v in self.dims[q])
        return arr[int(self.offsets[q]):int(self.offsets[q + 1])].reshape(nz, ny, nx)

    def last_error(self) -> int:
        return brsmooth_last_error(self.h)


def cell_updates(dims, sweeps: int) -> int:
    """Cell updates of `sweeps` sweeps over patches `dims` [(nx, ny, nz), ...] (the rate's numerator)."""
    return int(sum(int(a) * int(b) * int(c) for a, b, c in dims)) * int(sweeps)


def brsmooth_line_jacobi_noalloc(nx: int, ny: int, nz: int, a, omega: float, dtype_code: int,
                                 u_ptr, b_ptr, nsweeps: int, stream) -> int:
    """Allocation-free x-line block-Jacobi sweeps on device pointers (see the C header)."""
    fn = lib().brsmooth_line_jacobi_noalloc
    D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    fn.argtypes = [I, I, I, D, D, D, D, I, P, P, I, P]
    fn.restype = I
    return fn(int(nx), int(ny), int(nz), float(a[0]), float(a[1]), float(a[2]), float(omega),
              int(dtype_code), u_ptr, b_ptr, int(nsweeps), ctypes.c_void_p(stream))


def brsmooth_selftest_wait(ctx, limit_ns: int, stream) -> int:
    """Bounded wait on a never-signalled device barrier (see the C header)."""
    fn = lib().brsmooth_selftest_wait
    fn.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn(ctx, int(limit_ns), ctypes.c_void_p(stream))


def brsmooth_probe_fp64_fma(out_ptr, blocks: int, iters: int, stream) -> int:
    """FP64 FMA-bound measurement kernel (see the C header): blocks*256*iters*8 FMAs."""
    fn = lib().brsmooth_probe_fp64_fma
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn(out_ptr, int(blocks), int(iters), ctypes.c_void_p(stream))
