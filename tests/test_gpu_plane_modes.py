"""xy-plane sweeps in the x-sine basis on the GPU, against the FP64 oracle.

A call of several plane sweeps transforms u and b once along x (u^ = S_x u), runs every
sweep as independent y-line solves per x-mode (the plane block is diagonal in the x-sine
basis; the z coupling and the damping commute with S_x), and transforms back once.  In exact
arithmetic these are the plane sweeps' own iterates, so the checks are the plane path's:
the oracle's banded-Cholesky plane sweeps after the whole call (Jacobi, and the zebra order
for Gauss-Seidel), the closed-form damping of a sine mode over several sweeps, and the
per-sweep form on the same inputs.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs, sine_mode
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np

pytestmark = pytest.mark.gpu

# (nx, ny, nz): y rows that TMA can stage (ny * element size a multiple of 16 bytes, whole
# lane chunks), several tiles of mode rows, odd and even plane counts
SHAPES = [(32, 32, 7), (64, 96, 6), (24, 40, 5), (33, 24, 4), (128, 64, 9), (16, 16, 3),
          (96, 128, 2), (32, 512, 4), (64, 416, 3)]  # the last two: 16 cells per lane, two TMA pieces
COEFFS = [(1.0, 1.0, 1.0), (1.0, 1.0, 0.01), (1.0, 0.1, 0.01)]
MATHS = [("f64", "simt"), ("f32", "3xtf32"), ("f32", "tf32"), ("f32", "simt")]


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def tol_for(dt, math):
    return 2.0 ** -10 if math == "tf32" else TOL[dt]


def skip_unless_shape(math, nx, ny):
    if math in ("3xtf32", "tf32") and (nx % 32 or ny % 32):
        pytest.skip("tensor-core plane products need nx, ny multiples of 32")


def run(brs, u, b, a, *, dt, math, method, nsweeps, omega=0.0):
    nz, ny, nx = u.shape
    with brs.Context(nx, ny, nz, a, block="plane", method=method, dtype=dt, plane_math=math,
                     omega=omega) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        ctx.sweep(ut, bt, nsweeps)
        out = to_np(ut)
        assert ctx.last_error() == 0
    return out


@pytest.mark.parametrize("dt,math", MATHS, ids=lambda v: v)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS, ids=["iso", "aniso_z", "aniso_yz"])
def test_modes_jacobi_parity(brs, orc, dt, math, shape, a):
    """Four Jacobi sweeps in one call equal four oracle sweeps, element by element."""
    nx, ny, nz = shape
    skip_unless_shape(math, nx, ny)
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = u
    for _ in range(4):
        ref = orc.sweep(ref, b, a, block="plane", method="jacobi", omega=0.8)
    got = run(brs, u, b, a, dt=dt, math=math, method="jacobi", nsweeps=4)
    assert rel_max_err(got, ref) <= tol_for(dt, math)


@pytest.mark.parametrize("dt,math", MATHS, ids=lambda v: v)
@pytest.mark.parametrize("shape", [(32, 32, 7), (64, 96, 6), (33, 24, 4), (16, 16, 1),
                                   (32, 512, 5)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_modes_gs_equals_oracle_zebra(brs, orc, dt, math, shape, omega):
    """Gauss-Seidel in the x-sine basis: even planes, then odd planes from the new even ones,
    three sweeps in one call, equal to the oracle's zebra order element by element."""
    nx, ny, nz = shape
    skip_unless_shape(math, nx, ny)
    a = (1.0, 1.0, 0.01)
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = u
    for _ in range(3):
        ref = orc.sweep(ref, b, a, block="plane", method="gs_zebra", omega=omega)
    got = run(brs, u, b, a, dt=dt, math=math, method="gs", nsweeps=3, omega=omega)
    assert rel_max_err(got, ref) <= tol_for(dt, math)


@pytest.mark.parametrize("dt,math", [("f64", "simt"), ("f32", "3xtf32"), ("f32", "tf32")])
@pytest.mark.parametrize("n", [256, 512])
def test_modes_single_mode_damping(brs, orc, dt, math, n):
    """n x n x 4, a = (1, 0.1, 0.01): five Jacobi sweeps in one call scale a sine mode by
    g^5, g = 1 - omega lambda / mu the closed-form factor of one plane sweep."""
    nz = 4
    a = (1.0, 0.1, 0.01)
    g = orc.mode_factor(n, n, nz, a, "plane", 0.8)
    tol = 2.0 ** -9 if math == "tf32" else 8 * TOL[dt]
    with brs.Context(n, n, nz, a, block="plane", method="jacobi", dtype=dt,
                     plane_math=math) as ctx:
        for (p, q, r) in [(1, 1, 1), (n, n, 4), (37, n // 2 + 45, 2)]:
            m = rounded(sine_mode(n, n, nz, p, q, r), dt)
            ut, bt = to_dev(m, dt), to_dev(np.zeros_like(m), dt)
            ctx.sweep(ut, bt, 5)
            got = to_np(ut)
            err = np.max(np.abs(got - g[r - 1, q - 1, p - 1] ** 5 * m)) / np.max(np.abs(m))
            assert err <= tol, (p, q, r, err)
        assert ctx.last_error() == 0


@pytest.mark.parametrize("dt,math", [("f32", "3xtf32"), ("f64", "simt")])
@pytest.mark.parametrize("method", ["jacobi", "gs"])
def test_modes_full_size_256(brs, orc, dt, math, method, monkeypatch):
    """256^3, a = (1, 1, 0.01), three sweeps in one call (the benchmark's launch form):
    sampled planes equal the oracle after three sweeps (a plane after s sweeps depends only
    on planes within s of it; GS on planes within 2s), and the whole grid is within the
    parity tolerance of the per-sweep form."""
    import torch

    n, K = 256, 3
    a = (1.0, 1.0, 0.01)
    td = torch.float64 if dt == "f64" else torch.float32
    gen = torch.Generator(device="cuda").manual_seed(17)
    u0 = (torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1).to(td)
    bt = ((torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1)
          / (n + 1) ** 2).to(td)
    with brs.Context(n, n, n, a, block="plane", method=method, dtype=dt,
                     plane_math=math) as ctx:
        got_t = u0.clone()
        ctx.sweep(got_t, bt, K)
        torch.cuda.synchronize()
        assert ctx.last_error() == 0
    monkeypatch.setenv("BRSMOOTH_PLANE_MODES", "0")
    with brs.Context(n, n, n, a, block="plane", method=method, dtype=dt,
                     plane_math=math) as ctx:
        per = u0.clone()
        ctx.sweep(per, bt, K)
        torch.cuda.synchronize()
        assert ctx.last_error() == 0
    # the two forms are different arithmetic (both close to the oracle)
    assert not torch.equal(got_t, per)
    assert rel_max_err(to_np(got_t), to_np(per)) <= 2 * TOL[dt]
    u, b, got = to_np(u0), to_np(bt), to_np(got_t)
    ref_method = "jacobi" if method == "jacobi" else "gs_zebra"
    omega = 0.8 if method == "jacobi" else 1.0
    reach = K if method == "jacobi" else 2 * K
    for k in (0, 131, n - 1):
        k0, k1 = max(0, k - reach), min(n, k + reach + 1)
        if method == "gs":
            k0 -= k0 % 2  # keep the sub-grid's plane parity (the zebra colours)
        sub = u[k0:k1]
        for _ in range(K):
            sub = orc.sweep(sub, b[k0:k1], a, block="plane", method=ref_method, omega=omega)
        assert rel_max_err(got[k], sub[k - k0]) <= TOL[dt], k


@pytest.mark.parametrize("dt", ["f32"])
def test_modes_rows_not_tma_aligned_use_the_per_sweep_form(brs, orc, dt):
    """FP32 y rows that TMA cannot stage (ny = 9): the context keeps the per-sweep form, so a
    call of three sweeps equals three one-sweep calls bit for bit, and the oracle.  (FP64
    contexts take the x-sine form for any ny: see the twisted-elimination tests below.)"""
    import torch

    nx, ny, nz = 20, 9, 6
    a = (1.0, 1.0, 0.01)
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = u
    for _ in range(3):
        ref = orc.sweep(ref, b, a, block="plane", method="jacobi", omega=0.8)
    with brs.Context(nx, ny, nz, a, block="plane", method="jacobi", dtype=dt) as ctx:
        one, many, bt = to_dev(u, dt), to_dev(u, dt), to_dev(b, dt)
        ctx.sweep(one, bt, 3)
        for _ in range(3):
            ctx.sweep(many, bt, 1)
        torch.cuda.synchronize()
        assert ctx.last_error() == 0
    assert torch.equal(one, many)
    assert rel_max_err(to_np(one), ref) <= TOL[dt]


@pytest.mark.parametrize("dt,math", [("f32", "3xtf32"), ("f64", "simt")])
def test_modes_convergence_to_exact_solution(brs, orc, dt, math):
    """Plane GS in the x-sine basis, many sweeps per call, converges to A^{-1} b (FP32 to
    the level where rounding stalls it, about kappa(A) times the FP32 unit roundoff)."""
    nx, ny, nz = 32, 32, 8
    a = (1.0, 1.0, 0.01)
    u = np.zeros((nz, ny, nx))
    b = rounded(rhs((nz, ny, nx)), dt)
    exact = orc.exact_solve(b, a)
    got = run(brs, u, b, a, dt=dt, math=math, method="gs", nsweeps=600)
    assert rel_max_err(got, exact) <= (1e-10 if dt == "f64" else 1e-4)


# FP64: the twisted-elimination mode-line sweep ([k][y][p], two threads per y-line), any ny
TWIST_SHAPES = [(20, 9, 6), (7, 1, 5), (33, 17, 4), (5, 2, 3), (16, 16, 1), (48, 40, 7),
                (1, 12, 4), (70, 3, 2)]


@pytest.mark.parametrize("shape", TWIST_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS, ids=["iso", "aniso_z", "aniso_yz"])
def test_modes_f64_twisted_jacobi_any_shape(brs, orc, shape, a):
    nx, ny, nz = shape
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    ref = u
    for _ in range(4):
        ref = orc.sweep(ref, b, a, block="plane", method="jacobi", omega=0.8)
    got = run(brs, u, b, a, dt="f64", math="simt", method="jacobi", nsweeps=4)
    assert rel_max_err(got, ref) <= TOL["f64"]


@pytest.mark.parametrize("shape", TWIST_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_modes_f64_twisted_gs_equals_oracle_zebra(brs, orc, shape, omega):
    nx, ny, nz = shape
    a = (1.0, 0.1, 0.01)
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    ref = u
    for _ in range(3):
        ref = orc.sweep(ref, b, a, block="plane", method="gs_zebra", omega=omega)
    got = run(brs, u, b, a, dt="f64", math="simt", method="gs", nsweeps=3, omega=omega)
    assert rel_max_err(got, ref) <= TOL["f64"]


def test_modes_f64_twisted_equals_lane_scan_form(brs, orc, monkeypatch):
    """256 x 256 x 6 FP64: the twisted form and the lane-scan mode form (BRSMOOTH_MODE_TWIST=0)
    agree to FP64 rounding after a call of 5 sweeps."""
    nx, ny, nz = 256, 256, 6
    a = (1.0, 1.0, 0.01)
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    tw = run(brs, u, b, a, dt="f64", math="simt", method="jacobi", nsweeps=5)
    monkeypatch.setenv("BRSMOOTH_MODE_TWIST", "0")
    sc = run(brs, u, b, a, dt="f64", math="simt", method="jacobi", nsweeps=5)
    assert rel_max_err(tw, sc) <= 1e-13


@pytest.mark.parametrize("shape", [(256, 64, 4), (255, 33, 3), (33, 17, 4), (1, 9, 3), (2, 5, 3)],
                         ids=lambda s: "x".join(map(str, s)))
def test_modes_f64_folded_transforms_equal_plain_products(brs, orc, shape, monkeypatch):
    """The FP64 x-DST by the sine basis's even/odd symmetry (two half-size products) against
    the plain products (BRSMOOTH_MODE_FOLD=0), even and odd nx, after a call of 3 sweeps; and
    the oracle."""
    nx, ny, nz = shape
    a = (1.0, 0.1, 0.01)
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    ref = u
    for _ in range(3):
        ref = orc.sweep(ref, b, a, block="plane", method="jacobi", omega=0.8)
    fold = run(brs, u, b, a, dt="f64", math="simt", method="jacobi", nsweeps=3)
    monkeypatch.setenv("BRSMOOTH_MODE_FOLD", "0")
    plain = run(brs, u, b, a, dt="f64", math="simt", method="jacobi", nsweeps=3)
    assert rel_max_err(fold, plain) <= 1e-13
    assert rel_max_err(fold, ref) <= TOL["f64"]
