"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This module only draws numbers and describes workload shapes; it holds none of the
relaxation method's arithmetic.  Every array is float64, drawn with numpy's PCG64
(`default_rng(seed)`) from U[-1, 1] in x-fastest order and returned with shape
(nz, ny, nx).  A float32 copy is the round-to-nearest cast of the float64 draw.

Seeds: right-hand side -> 1, initial guess -> 2, adjoint target -> 3, batched patch
dimensions -> 4.  The paper draws a random initial guess for its convergence study
(Sec. 3) and sets the source to zero (Sec. 1.1); the workloads below keep its patch
shapes and add seeded sources so that every path has non-trivial data.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_F = 1
SEED_U0 = 2
SEED_TARGET = 3
SEED_DIMS = 4

PATCH_DIM_CHOICES = (16, 24, 32, 48, 64)


def uniform_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """float64 array of `shape` (nz, ny, nx) drawn from U[lo, hi] with PCG64(seed)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    return rng.uniform(lo, hi, size=n).reshape(shape)


def grid_spacing(n: int) -> float:
    """Mesh width h = 1/(n+1) of an n-cell axis whose Dirichlet values sit at indices -1 and n."""
    return 1.0 / (n + 1)


def rhs(shape, seed: int = SEED_F, h: float | None = None) -> np.ndarray:
    """Right-hand side b = h^2 * f with f ~ U[-1, 1] (seeded); h defaults to 1/(nx+1)."""
    if h is None:
        h = grid_spacing(shape[-1])
    return (h * h) * uniform_field(shape, seed)


def initial_guess(shape, seed: int = SEED_U0, zero: bool = False) -> np.ndarray:
    """u0 ~ U[-1, 1] (seeded) or zeros."""
    if zero:
        return np.zeros(shape)
    return uniform_field(shape, seed)


def sine_mode(nx: int, ny: int, nz: int, p: int, q: int, r: int) -> np.ndarray:
    """Discrete Dirichlet sine mode sin(p pi (i+1)/(nx+1)) sin(q pi (j+1)/(ny+1)) sin(r pi (k+1)/(nz+1)).

    Shape (nz, ny, nx); p, q, r are 1-based mode numbers.
    """
    sx = np.sin(p * np.pi * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(q * np.pi * np.arange(1, ny + 1) / (ny + 1))
    sz = np.sin(r * np.pi * np.arange(1, nz + 1) / (nz + 1))
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def batched_patch_dims(npatch: int = 600, seed: int = SEED_DIMS) -> np.ndarray:
    """(npatch, 3) int array of (nx, ny, nz), each drawn independently from {16,24,32,48,64}."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.array(PATCH_DIM_CHOICES), size=(npatch, 3))


def batched_fields(dims: np.ndarray, seed: int, scale_h2: bool = False, h: float = 1.0 / 65):
    """One flat float64 array holding every patch's field back to back (x-fastest per patch).

    Patch p's values are a U[-1,1] draw of its own size from one PCG64(seed) stream, in
    patch order.  With `scale_h2` the draw is multiplied by h^2 (a right-hand side with
    the common mesh width of one refinement level).
    """
    rng = np.random.default_rng(seed)
    total = int(sum(int(a) * int(b) * int(c) for a, b, c in dims))
    out = rng.uniform(-1.0, 1.0, size=total)
    if scale_h2:
        out *= h * h
    return out


def level_tiling(P, pdim):
    """Patch layout of a Px x Py x Pz array of equal patches (patch index x fastest):
    dims (npatch, 3) and face neighbours (npatch, 6) in the order -x, +x, -y, +y, -z, +z,
    -1 on the outer boundary."""
    Px, Py, Pz = P
    dims, nbr = [], []
    idx = lambda a, b, c: a + Px * (b + Py * c)
    for k in range(Pz):
        for j in range(Py):
            for i in range(Px):
                dims.append(list(pdim))
                nbr.append([idx(i - 1, j, k) if i > 0 else -1,
                            idx(i + 1, j, k) if i + 1 < Px else -1,
                            idx(i, j - 1, k) if j > 0 else -1,
                            idx(i, j + 1, k) if j + 1 < Py else -1,
                            idx(i, j, k - 1) if k > 0 else -1,
                            idx(i, j, k + 1) if k + 1 < Pz else -1])
    return np.array(dims, dtype=np.int64), np.array(nbr, dtype=np.int64)


def table2_mixed_level():
    """The mixed set of the paper's Table 2: 80 patches, 16 each of 64^3, 72^3, 80^3, 88^3
    and 96^3.  The paper gives no adjacency; here each size class is a 4 x 2 x 2 array of
    face neighbours (five separate blocks of patches in one level)."""
    dims, nbr = [], []
    for n in (64, 72, 80, 88, 96):
        d, nb = level_tiling((4, 2, 2), (n, n, n))
        base = len(dims)
        dims.extend(d.tolist())
        nbr.extend([[x + base if x >= 0 else -1 for x in row] for row in nb.tolist()])
    return np.array(dims, dtype=np.int64), np.array(nbr, dtype=np.int64)



@dataclass(frozen=True)
class Workload:
    """A named grid workload: interior dims, coefficients, sweeps and dtype."""

    name: str
    nx: int
    ny: int
    nz: int
    coeffs: tuple = (1.0, 1.0, 1.0)
    sweeps: int = 1
    dtypes: tuple = ("f64",)
    u0_zero: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


# The grid workloads: sizes, coefficient sets, sweep counts and seeds.
SMALL_32 = Workload("grid32_iso", 32, 32, 32, (1.0, 1.0, 1.0), 10, ("f64",), u0_zero=True)
GRID_256_ISO = Workload("grid256_iso", 256, 256, 256, (1.0, 1.0, 1.0), 50, ("f64", "f32"))
GRID_256_ANISO = Workload("grid256_aniso", 256, 256, 256, (1.0, 1.0, 0.01), 50, ("f64", "f32"))
GRID_512_ANISO = Workload("grid512_aniso", 512, 512, 512, (1.0, 0.1, 0.01), 0, ("f32", "f64"), u0_zero=True)
GRID_128_ADJ = Workload("grid128_adjoint", 128, 128, 128, (1.0, 1.0, 1.0), 8, ("f64", "f32"))
GRID_384_ADJ = Workload("grid384_adjoint", 384, 384, 384, (1.0, 1.0, 1.0), 8, ("f64", "f32"),
                        extra={"checkpoint_every": 4})
