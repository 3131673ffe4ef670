"""FP64 CPU oracle for block relaxation on a 3D constant-coefficient 7-point stencil.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA library and
never imports it; the two meet only in the seeded generators of ``brs_inputs``.

Arrays are numpy float64 with shape (nz, ny, nx) (x fastest).  The heavy loops are the
plain C routines of ``brs_oracle.c`` (compiled with gcc by :func:`build`); this module adds
the pieces whose plain definition is a library primitive or a closed form:

* :func:`exact_solve` -- u* = A^{-1} b by the orthonormal 3D DST-I (A is diagonal in the
  sine basis; Sec. 1.1 operator with zero Dirichlet values), via ``scipy.fft.dstn``.
* :func:`eigenvalues` / :func:`mode_factor` -- the closed-form spectrum of A and of the
  line/plane block diagonal, and the exact per-sweep damping of one sine mode.
* :func:`adjoint_gradients` -- reverse-mode gradients of L = 0.5 ||u_K - u_t||^2 through K
  block-Jacobi sweeps (Eq. blockiteration2), stepping lambda_k = G^T lambda_{k+1}.
* :func:`sweep` with ``block="box"`` and :func:`box_inverse` -- bx*by*bz blocks whose
  inverse comes from a dense Cholesky factorisation (Sec. 4.3 inverts once per block
  shape); the visiting orders of block GS (Eq. sm:blockm) as lexicographic, reverse and
  two-colour.
* :func:`level_sweep` -- a level of patches whose ghost layers hold the face neighbours'
  values from before the step (Sec. 2), one x-line sweep per patch.

Parity status: every function here is pinned by a CPU test (``tests/test_oracle_*.py``):
closed forms, dense solves, equalities between independently built block forms (box = line
= plane = permuted line), Young's relation between block Jacobi and two-colour block GS.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "brs_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libbrs_oracle.so"
_lib = None

JACOBI = "jacobi"
GS_LEX = "gs_lex"
GS_REVERSE = "gs_reverse"
GS_ZEBRA = "gs_zebra"
_GS_ORDER = {GS_LEX: 0, GS_REVERSE: 1, GS_ZEBRA: 2}


def build(force: bool = False) -> Path:
    """Compile brs_oracle.c with gcc (FP64, no FMA contraction, OpenMP)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               str(_SRC), "-lm", "-o", str(tmp)]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(str(build()))
    D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
    sig = {
        "orc_apply_A": [I, I, I, D, D, D, P, P],
        "orc_residual": [I, I, I, D, D, D, P, P, P],
        "orc_thomas": [I, D, D, P, P, P, P],
        "orc_line_minv": [I, I, I, D, D, D, P, P],
        "orc_line_jacobi": [I, I, I, D, D, D, D, P, P, P, P],
        "orc_line_gs": [I, I, I, D, D, D, D, I, P, P],
        "orc_plane_factor": [I, I, D, D, D, P],
        "orc_plane_solve": [I, I, P, P],
        "orc_plane_minv": [I, I, I, P, P, P],
        "orc_plane_jacobi": [I, I, I, D, D, D, D, P, P, P, P, P],
        "orc_plane_gs": [I, I, I, D, D, D, D, I, P, P, P, P],
        "orc_box_inverse": [I, I, I, D, D, D, P, P],
        "orc_box_minv": [I, I, I, I, I, I, P, P, P],
        "orc_box_jacobi": [I, I, I, I, I, I, D, D, D, D, P, P, P, P, P],
        "orc_box_gs": [I, I, I, I, I, I, D, D, D, D, I, P, P, P],
        "orc_level_sweep": [I, P, P, P, D, D, D, D, I, P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I if name in ("orc_plane_factor", "orc_box_inverse") else None
    lib.orc_sumsq.argtypes = [L, P]
    lib.orc_sumsq.restype = D
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(u):
    nz, ny, nx = u.shape
    return nx, ny, nz


def num_threads() -> int:
    """Threads the OpenMP loops of the oracle use (OMP_NUM_THREADS, else all cores)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env:
        return int(env)
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


# ---------------------------------------------------------------- operator, residual

def apply_A(u, a):
    """A u for the 7-point stencil with coefficients a = (ax, ay, az), zero outside (Sec. 1.1)."""
    u = _f64(u)
    out = np.empty_like(u)
    _load().orc_apply_A(*_dims(u), *map(float, a), _ptr(u), _ptr(out))
    return out


def residual(u, b, a):
    """r = b - A u (Eq. blockiteration2)."""
    u, b = _f64(u), _f64(b)
    r = np.empty_like(u)
    _load().orc_residual(*_dims(u), *map(float, a), _ptr(u), _ptr(b), _ptr(r))
    return r


def residual_norm(u, b, a) -> float:
    """||b - A u||_2 over the interior cells, accumulated in FP64."""
    r = residual(u, b, a)
    return float(np.sqrt(_load().orc_sumsq(r.size, _ptr(r))))


def thomas(off: float, diag: float, rhs):
    """Solve diag*x_i + off*(x_{i-1}+x_{i+1}) = rhs_i by the textbook Thomas algorithm."""
    rhs = _f64(rhs)
    n = rhs.size
    x, cp, dp = np.empty(n), np.empty(n), np.empty(n)
    _load().orc_thomas(n, float(off), float(diag), _ptr(rhs), _ptr(x), _ptr(cp), _ptr(dp))
    return x


# ---------------------------------------------------------------- block solves

class PlaneFactor:
    """Banded Cholesky of the xy-plane block M_plane, computed once and reused (Sec. 4.3)."""

    def __init__(self, nx: int, ny: int, a):
        self.nx, self.ny, self.a = nx, ny, tuple(map(float, a))
        self.L = np.zeros(nx * ny * (nx + 1))
        rc = _load().orc_plane_factor(nx, ny, *self.a, _ptr(self.L))
        if rc != 0:
            raise ValueError("plane block is not positive definite")

    def solve(self, rhs_plane):
        x = _f64(rhs_plane).copy()
        _load().orc_plane_solve(self.nx, self.ny, _ptr(self.L), _ptr(x))
        return x


_factor_cache: dict = {}


def plane_factor(nx: int, ny: int, a) -> PlaneFactor:
    key = (nx, ny, tuple(map(float, a)))
    if key not in _factor_cache:
        _factor_cache.clear()  # keep at most one (the 256^2 factor is 135 MB)
        _factor_cache[key] = PlaneFactor(nx, ny, a)
    return _factor_cache[key]


_box_cache: dict = {}


def box_inverse(box, a) -> np.ndarray:
    """Ahat_b = A_b^{-1} (n x n, n = bx by bz, local order x fastest) of the box block A_b,
    computed once per block shape and coefficients (Sec. 4.3) by a dense Cholesky solve."""
    bx, by, bz = (int(v) for v in box)
    key = (bx, by, bz, tuple(map(float, a)))
    if key not in _box_cache:
        n = bx * by * bz
        inv, work = np.empty((n, n)), np.empty((n, n))
        if _load().orc_box_inverse(bx, by, bz, *key[3], _ptr(inv), _ptr(work)) != 0:
            raise ValueError("box block is not positive definite")
        _box_cache[key] = inv
    return _box_cache[key]


def _check_box(nx, ny, nz, box):
    bx, by, bz = (int(v) for v in box)
    if min(bx, by, bz) < 1 or nx % bx or ny % by or nz % bz:
        raise ValueError(f"box {box} does not tile the {nx}x{ny}x{nz} grid")
    return bx, by, bz


def block_minv(r, a, block: str, box=None):
    """M^{-1} r for the block diagonal M of the x-line ('line'), xy-plane ('plane') or
    bx*by*bz box ('box', with box=(bx, by, bz)) partition."""
    r = _f64(r)
    nx, ny, nz = _dims(r)
    out = np.empty_like(r)
    if block == "line":
        _load().orc_line_minv(nx, ny, nz, *map(float, a), _ptr(r), _ptr(out))
    elif block == "plane":
        f = plane_factor(nx, ny, a)
        _load().orc_plane_minv(nx, ny, nz, _ptr(f.L), _ptr(r), _ptr(out))
    elif block == "box":
        bx, by, bz = _check_box(nx, ny, nz, box)
        inv = box_inverse((bx, by, bz), a)
        _load().orc_box_minv(nx, ny, nz, bx, by, bz, _ptr(inv), _ptr(r), _ptr(out))
    else:
        raise ValueError(block)
    return out


# ---------------------------------------------------------------- sweeps

def sweep(u, b, a, *, block: str = "line", method: str = JACOBI, omega: float = 0.8,
          box=None):
    """One block-relaxation sweep; returns the new iterate (inputs are not modified).

    method 'jacobi': v = u + omega M^{-1}(b - A u) from the old iterate only (Alg. 2).
    methods 'gs_lex' / 'gs_reverse' / 'gs_zebra': block Gauss-Seidel (Eq. sm:blockm),
    blocks visited lexicographically, in reverse, or in two colours (even-then-odd j+k for
    lines, k for planes, bi+bj+bk for boxes), newest values read.
    block 'box' takes box=(bx, by, bz) (the spatial blocks of Sec. 2 and Sec. 3).
    """
    u, b = _f64(u), _f64(b)
    nx, ny, nz = _dims(u)
    lib = _load()
    a = tuple(map(float, a))
    if block == "box":
        bx, by, bz = _check_box(nx, ny, nz, box)
        inv = box_inverse((bx, by, bz), a)
        if method == JACOBI:
            v, work = np.empty_like(u), np.empty_like(u)
            lib.orc_box_jacobi(nx, ny, nz, bx, by, bz, *a, float(omega), _ptr(inv), _ptr(u),
                               _ptr(b), _ptr(v), _ptr(work))
            return v
        v = u.copy()
        lib.orc_box_gs(nx, ny, nz, bx, by, bz, *a, float(omega), _GS_ORDER[method], _ptr(inv),
                       _ptr(v), _ptr(b))
        return v
    if method == JACOBI:
        v = np.empty_like(u)
        work = np.empty_like(u)
        if block == "line":
            lib.orc_line_jacobi(nx, ny, nz, *a, float(omega), _ptr(u), _ptr(b), _ptr(v), _ptr(work))
        else:
            f = plane_factor(nx, ny, a)
            lib.orc_plane_jacobi(nx, ny, nz, *a, float(omega), _ptr(f.L), _ptr(u), _ptr(b),
                                 _ptr(v), _ptr(work))
        return v
    order = _GS_ORDER[method]
    v = u.copy()
    if block == "line":
        lib.orc_line_gs(nx, ny, nz, *a, float(omega), order, _ptr(v), _ptr(b))
    else:
        f = plane_factor(nx, ny, a)
        work = np.empty(nx * ny)
        lib.orc_plane_gs(nx, ny, nz, *a, float(omega), order, _ptr(f.L), _ptr(v), _ptr(b), _ptr(work))
    return v


def level_offsets(dims) -> np.ndarray:
    """Start of each patch in the packed arrays (patches back to back, x fastest)."""
    d = np.asarray(dims, dtype=np.int64).reshape(-1, 3)
    return np.concatenate([[0], np.cumsum(d.prod(axis=1))[:-1]]).astype(np.int64)


def level_sweep(u, b, dims, nbr, a, *, method: str = JACOBI, omega: float = 0.8):
    """One smoothing step of a level of patches (packed arrays; Sec. 2 ghost update).

    dims: (npatch, 3) patch sizes (nx, ny, nz); nbr: (npatch, 6) face neighbours in the order
    -x, +x, -y, +y, -z, +z (patch index, -1 = physical boundary).  Every patch is smoothed
    with its ghost layer fixed at the neighbours' values from before the step (Jacobi
    fashion); method 'jacobi' (x-line block Jacobi) or 'gs_lex' (x-line block GS).
    """
    u, b = _f64(u).ravel(), _f64(b).ravel()
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
    nb = np.ascontiguousarray(np.asarray(nbr, dtype=np.int32).reshape(-1, 6))
    off = np.ascontiguousarray(level_offsets(d))
    v = np.empty_like(u)
    work = np.empty(2 * int(d.prod(axis=1).max()))
    m = {JACOBI: 0, GS_LEX: 1}[method]
    _load().orc_level_sweep(len(d), _ptr(d), _ptr(nb), _ptr(off), *map(float, a), float(omega),
                            m, _ptr(u), _ptr(b), _ptr(v), _ptr(work))
    return v


def trajectory(u0, b, a, nsweeps: int, **kw):
    """List [u_1, ..., u_n] of successive sweeps from u0."""
    out, u = [], _f64(u0)
    for _ in range(nsweeps):
        u = sweep(u, b, a, **kw)
        out.append(u)
    return out


# ---------------------------------------------------------------- closed forms

def axis_eigs(n: int) -> np.ndarray:
    """Eigenvalues s_p = 2 - 2 cos(p pi/(n+1)), p = 1..n, of tridiag(-1, 2, -1) of size n."""
    p = np.arange(1, n + 1)
    return 2.0 - 2.0 * np.cos(p * np.pi / (n + 1))


def eigenvalues(nx: int, ny: int, nz: int, a) -> np.ndarray:
    """lambda_pqr = ax s_p + ay s_q + az s_r as an (nz, ny, nx) array (A = ax Tx + ay Ty + az Tz)."""
    ax, ay, az = a
    return (az * axis_eigs(nz)[:, None, None] + ay * axis_eigs(ny)[None, :, None]
            + ax * axis_eigs(nx)[None, None, :])


def block_eigenvalues(nx: int, ny: int, nz: int, a, block: str) -> np.ndarray:
    """Eigenvalues of the block diagonal M on the same sine modes.

    line:  mu_p  = ax s_p + 2 ay + 2 az        (M_line = ax Tx + 2(ay+az) I)
    plane: mu_pq = ax s_p + ay s_q + 2 az      (M_plane = ax Tx + ay Ty + 2 az I)
    """
    ax, ay, az = a
    sx = axis_eigs(nx)[None, None, :]
    if block == "line":
        mu = ax * sx + 2 * ay + 2 * az
    else:
        mu = ax * sx + ay * axis_eigs(ny)[None, :, None] + 2 * az
    return np.broadcast_to(mu, (nz, ny, nx)).copy()


def mode_factor(nx, ny, nz, a, block: str, omega: float) -> np.ndarray:
    """Per-sweep factor g_pqr = 1 - omega lambda_pqr / mu of block Jacobi on sine mode (p,q,r)."""
    return 1.0 - omega * eigenvalues(nx, ny, nz, a) / block_eigenvalues(nx, ny, nz, a, block)


def exact_solve(b, a):
    """u* = A^{-1} b by the orthonormal DST-I in x, y and z (A = S diag(lambda) S, S = S^{-1})."""
    from scipy.fft import dstn, idstn

    b = _f64(b)
    nz, ny, nx = b.shape
    bh = dstn(b, type=1, norm="ortho")
    return idstn(bh / eigenvalues(nx, ny, nz, a), type=1, norm="ortho")


# ---------------------------------------------------------------- adjoint (reverse mode)

def _axis_T(u, axis: int):
    """T_d u = 2u - u_{-1} - u_{+1} along one axis of an (nz, ny, nx) array, zero outside."""
    out = 2.0 * u
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[axis], hi[axis] = slice(0, -1), slice(1, None)
    out[tuple(lo)] -= u[tuple(hi)]
    out[tuple(hi)] -= u[tuple(lo)]
    return out


def adjoint_gradients(u0, b, a, nsweeps: int, u_target, *, block: str = "line", omega: float = 0.8):
    """Gradients of L = 0.5 ||u_K - u_t||^2 after K block-Jacobi sweeps (Eq. blockiteration2).

    Sweep: u_{k+1} = u_k + omega z_k with z_k = M^{-1}(b - A u_k); A and M are symmetric.
    Reverse recursion: lambda_K = u_K - u_t,  lambda_k = lambda_{k+1} - omega A M^{-1} lambda_{k+1}.
      dL/du0 = lambda_0
      dL/db  = omega * sum_k M^{-1} lambda_{k+1}
      dL/da_d = -omega * sum_k  (M^{-1} lambda_{k+1})^T [ (dM/da_d) z_k + (dA/da_d) u_k ]
    with dA/da_d = T_d; line blocks: dM/dax = Tx, dM/day = dM/daz = 2I;
    plane blocks: dM/dax = Tx, dM/day = Ty, dM/daz = 2I.
    Returns (L, dL/du0, dL/db, dL/da as a length-3 array).
    """
    a = tuple(map(float, a))
    us = [_f64(u0)]
    zs = []
    for _ in range(nsweeps):
        z = block_minv(residual(us[-1], b, a), a, block)
        zs.append(z)
        us.append(us[-1] + omega * z)
    lam = us[-1] - _f64(u_target)
    loss = 0.5 * float(np.sum(lam * lam))
    gb = np.zeros_like(lam)
    ga = np.zeros(3)
    axes = {0: 2, 1: 1, 2: 0}  # coefficient index -> array axis (x is the last axis)
    for k in range(nsweeps - 1, -1, -1):
        mu = block_minv(lam, a, block)
        gb += omega * mu
        uk, zk = us[k], zs[k]
        for d in range(3):
            if d == 0 or (block == "plane" and d == 1):
                dMz = _axis_T(zk, axes[d])
            else:
                dMz = 2.0 * zk
            ga[d] += -omega * float(np.sum(mu * (dMz + _axis_T(uk, axes[d]))))
        lam = lam - omega * apply_A(mu, a)
    return loss, lam, gb, ga


def sweeps_loss(u0, b, a, nsweeps, u_target, *, block="line", omega=0.8) -> float:
    """L = 0.5 ||u_K - u_t||^2 after K block-Jacobi sweeps (forward only)."""
    u = _f64(u0)
    for _ in range(nsweeps):
        u = sweep(u, b, a, block=block, method=JACOBI, omega=omega)
    d = u - _f64(u_target)
    return 0.5 * float(np.sum(d * d))


# ---------------------------------------------------------------- dense helpers for pins

def assemble_A(nx: int, ny: int, nz: int, a) -> np.ndarray:
    """Dense A (n x n, n = nx ny nz) assembled column by column from apply_A on unit vectors."""
    n = nx * ny * nz
    A = np.empty((n, n))
    e = np.zeros((nz, ny, nx))
    for c in range(n):
        e.flat[c] = 1.0
        A[:, c] = apply_A(e, a).ravel()
        e.flat[c] = 0.0
    return A


def block_of(nx: int, ny: int, nz: int, block: str, box=None) -> np.ndarray:
    """Block label of every cell (x fastest): line -> j + ny k, plane -> k,
    box -> bi + nbx (bj + nby bk) with (bi, bj, bk) = (i // bx, j // by, k // bz)."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    if block == "box":
        bx, by, bz = _check_box(nx, ny, nz, box)
        nbx, nby = nx // bx, ny // by
        return (i // bx + nbx * (j // by + nby * (k // bz))).ravel()
    return (j + ny * k).ravel() if block == "line" else k.ravel()


if __name__ == "__main__":  # build only
    print(build(force="--force" in sys.argv))
