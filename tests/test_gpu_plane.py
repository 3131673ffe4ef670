"""xy-plane block sweeps on the GPU (sine-basis plane solve) against the FP64 oracle.

The oracle solves each plane block with a once-factored banded Cholesky, so the two
paths share nothing but the definition of the block.  Jacobi: element-wise per-sweep
parity.  Gauss-Seidel on the GPU visits the even planes, then the odd ones: element-wise
parity with the oracle's zebra order, plus the Perron bound, the residual bracket and
convergence to A^{-1} b.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs, sine_mode
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 8), (32, 24, 5), (33, 17, 4), (1, 1, 3), (64, 64, 4), (5, 70, 3),
          (1, 9, 2), (100, 3, 3)]
COEFFS = [(1.0, 1.0, 1.0), (1.0, 1.0, 0.01), (1.0, 0.1, 0.01)]


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def gpu_run(brs, u, b, a, *, dt, method="jacobi", nsweeps=1, math="auto", omega=0.0):
    nz, ny, nx = u.shape
    with brs.Context(nx, ny, nz, a, block="plane", method=method, dtype=dt, plane_math=math,
                     omega=omega) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        ctx.sweep(ut, bt, nsweeps)
        out = to_np(ut)
        assert ctx.last_error() == 0
    return out


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS, ids=["iso", "aniso_z", "aniso_yz"])
def test_plane_jacobi_one_sweep_parity(brs, orc, dt, shape, a):
    nx, ny, nz = shape
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = orc.sweep(u, b, a, block="plane", method="jacobi", omega=0.8)
    got = gpu_run(brs, u, b, a, dt=dt)
    assert rel_max_err(got, ref) <= TOL[dt]


@pytest.mark.parametrize("block", ["line", "plane"])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_single_mode_damping_on_gpu(brs, orc, block, dt):
    """A sine mode is scaled by exactly g = 1 - omega lambda/mu per Jacobi sweep (b = 0)."""
    nx, ny, nz = 24, 20, 12
    a = (1.0, 0.1, 0.01)
    g = orc.mode_factor(nx, ny, nz, a, block, 0.8)
    for (p, q, r) in [(1, 1, 1), (24, 20, 12), (5, 17, 3)]:
        m = rounded(sine_mode(nx, ny, nz, p, q, r), dt)
        with brs.Context(nx, ny, nz, a, block=block, method="jacobi", dtype=dt) as ctx:
            ut, bt = to_dev(m, dt), to_dev(np.zeros_like(m), dt)
            ctx.sweep(ut, bt, 1)
            got = to_np(ut)
        # measured against the input's magnitude: a strongly damped mode (|g| << 1) is a
        # small difference of O(|m|) terms, so its rounding scales with |m|, not with g|m|
        err = np.max(np.abs(got - g[r - 1, q - 1, p - 1] * m)) / np.max(np.abs(m))
        assert err <= 4 * TOL[dt]


def test_plane_trajectory_and_norms(brs, orc):
    n = 24
    a = (1.0, 1.0, 0.01)
    b = rhs((n, n, n))
    u0 = initial_guess((n, n, n))
    traj = orc.trajectory(u0, b, a, 6, block="plane", method="jacobi", omega=0.8)
    with brs.Context(n, n, n, a, block="plane", method="jacobi", dtype="f64") as ctx:
        ut, bt = to_dev(u0, "f64"), to_dev(b, "f64")
        for k in range(6):
            ctx.sweep(ut, bt, 1)
            assert rel_max_err(to_np(ut), traj[k]) <= 1e-12
            ref = orc.residual_norm(traj[k], b, a)
            assert abs(ctx.residual(ut, bt) - ref) <= 1e-11 * ref


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_plane_gs_perron_bound(brs, orc, dt):
    nx, ny, nz = 32, 24, 20
    a = (1.0, 1.0, 1.0)
    m = sine_mode(nx, ny, nz, 1, 1, 1)
    g = orc.mode_factor(nx, ny, nz, a, "plane", 1.0)[0, 0, 0]
    slack = 1e-13 if dt == "f64" else 2e-6
    with brs.Context(nx, ny, nz, a, block="plane", method="gs", dtype=dt) as ctx:
        ut, bt = to_dev(m, dt), to_dev(np.zeros_like(m), dt)
        mr = to_np(ut)
        for k in range(1, 7):
            ctx.sweep(ut, bt, 1)
            u = to_np(ut)
            assert np.all(u >= -slack * k)
            assert np.all(u <= g ** k * mr + slack * (1 + k))


def test_plane_gs_bracket_and_convergence(brs, orc):
    n = 16
    a = (1.0, 1.0, 0.01)
    b = rhs((n, n, n))
    u0 = initial_guess((n, n, n))
    refs = {}
    for meth in ("jacobi", "gs_lex", "gs_zebra", "gs_reverse"):
        u, norms = u0, []
        for _ in range(8):
            u = orc.sweep(u, b, a, block="plane", method=meth, omega=1.0)
            norms.append(orc.residual_norm(u, b, a))
        refs[meth] = np.array(norms)
    lo = np.minimum(np.minimum(refs["gs_lex"], refs["gs_zebra"]), refs["gs_reverse"])
    with brs.Context(n, n, n, a, block="plane", method="gs", dtype="f64") as ctx:
        ut, bt = to_dev(u0, "f64"), to_dev(b, "f64")
        for k in range(8):
            ctx.sweep(ut, bt, 1)
            r = ctx.residual(ut, bt)
            assert 0.9 * lo[k] <= r <= 1.1 * refs["jacobi"][k]
        ctx.sweep(ut, bt, 400)
        assert rel_max_err(to_np(ut), orc.exact_solve(b, a)) <= 1e-10


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_full_size_256_sampled_planes(brs, orc, dt):
    """256^3 plane Jacobi, launch configuration of the benchmark; three planes vs the oracle."""
    import torch

    n = 256
    a = (1.0, 1.0, 0.01)
    gen = torch.Generator(device="cuda").manual_seed(3)
    ut = torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
    bt = (torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1) / (n + 1) ** 2
    if dt == "f32":
        ut, bt = ut.float(), bt.float()
    u, b = to_np(ut), to_np(bt)
    with brs.Context(n, n, n, a, block="plane", method="jacobi", dtype=dt) as ctx:
        ctx.sweep(ut, bt, 1)
        torch.cuda.synchronize()
    got = to_np(ut)
    for k in (0, 131, n - 1):
        k0, k1 = max(0, k - 1), min(n, k + 2)
        sub = orc.sweep(u[k0:k1], b[k0:k1], a, block="plane", method="jacobi", omega=0.8)
        assert rel_max_err(got[k], sub[k - k0]) <= TOL[dt]


# ----------------------------------------------------------------- tensor-core plane solve

TC_SHAPES = [(32, 32, 4), (64, 96, 3), (96, 64, 5), (256, 256, 3), (160, 128, 2)]


@pytest.mark.parametrize("kernel", ["tile64", "tile128", "persistent128", "persistent64",
                                    "persistent256"])
@pytest.mark.parametrize("shape", TC_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS, ids=["iso", "aniso_z", "aniso_yz"])
def test_plane_3xtf32_one_sweep_parity(brs, orc, shape, a, kernel, monkeypatch):
    """Split-TF32 tcgen05 products hold the FP32 per-sweep tolerance (every kernel shape)."""
    pers = kernel.startswith("persistent")
    tile = kernel[len("persistent"):] if pers else kernel[len("tile"):]
    monkeypatch.setenv("BRSMOOTH_TC_PERSISTENT", "1" if pers else "0")
    monkeypatch.setenv("BRSMOOTH_TC_PBN" if pers else "BRSMOOTH_TC_BN", tile)
    nx, ny, nz = shape
    u = rounded(initial_guess((nz, ny, nx)), "f32")
    b = rounded(rhs((nz, ny, nx)), "f32")
    ref = orc.sweep(u, b, a, block="plane", method="jacobi", omega=0.8)
    got = gpu_run(brs, u, b, a, dt="f32", math="3xtf32")
    assert rel_max_err(got, ref) <= TOL["f32"]


@pytest.mark.parametrize("persistent", ["0", "1", "256"])
@pytest.mark.parametrize("shape", [(32, 32, 4), (160, 128, 2), (256, 256, 2)], ids=str)
def test_plane_single_tf32_error_is_tf32_level(brs, orc, shape, persistent, monkeypatch):
    monkeypatch.setenv("BRSMOOTH_TC_PERSISTENT", "0" if persistent == "0" else "1")
    if persistent == "256":
        monkeypatch.setenv("BRSMOOTH_TC_PBN", "256")
    """One TF32 pass per product: per-sweep error at the TF32 unit roundoff 2^-11 ~ 4.9e-4
    (not held to the FP32 bar; used inside defect correction, where FP64 decides)."""
    nx, ny, nz = shape
    a = (1.0, 1.0, 0.01)
    u = rounded(initial_guess((nz, ny, nx)), "f32")
    b = rounded(rhs((nz, ny, nx)), "f32")
    ref = orc.sweep(u, b, a, block="plane", method="jacobi", omega=0.8)
    err = rel_max_err(gpu_run(brs, u, b, a, dt="f32", math="tf32"), ref)
    assert err <= 2.0 ** -11


def test_plane_3xtf32_gs_perron_and_defect_correction(brs, orc):
    nx, ny, nz = 64, 32, 12
    a = (1.0, 1.0, 1.0)
    m = sine_mode(nx, ny, nz, 1, 1, 1)
    g = orc.mode_factor(nx, ny, nz, a, "plane", 1.0)[0, 0, 0]
    with brs.Context(nx, ny, nz, a, block="plane", method="gs", dtype="f32", plane_math="3xtf32") as c:
        ut, bt = to_dev(m, "f32"), to_dev(np.zeros_like(m), "f32")
        mr = to_np(ut)
        for k in range(1, 6):
            c.sweep(ut, bt, 1)
            u = to_np(ut)
            assert np.all(u >= -1e-6 * k) and np.all(u <= g ** k * mr + 2e-6 * (1 + k))
    # single-pass TF32 inner sweeps still reach an FP64 residual of 1e-10 under defect correction
    n = 64
    a = (1.0, 0.1, 0.01)
    b = rhs((n, n, n))
    with brs.Context(n, n, n, a, block="plane", dtype="f64") as o64, \
            brs.Context(n, n, n, a, block="plane", dtype="f32", plane_math="tf32") as i32:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        done, rel, _ = brs.defect_correction(o64, i32, ut, bt, rtol=1e-10, inner_sweeps=16,
                                             max_outer=500)
        u = to_np(ut)
    assert rel <= 1e-10
    assert orc.residual_norm(u, b, a) <= 1.05e-10 * np.linalg.norm(b)


def test_plane_tensor_core_unsupported_shapes(brs):
    for (nx, ny, dt, math) in [(33, 32, "f32", "3xtf32"), (32, 48, "f32", "tf32"), (32, 32, "f64", "tf32")]:
        p = brs.brs_params(nx, ny, 4, 1.0, 1.0, 1.0, brs.BRS_XYPLANE, brs.BRS_JACOBI,
                           brs.DTYPES[dt], 0.0, brs.PLANE_MATH[math])
        rc, h = brs.brsmooth_create(p)
        assert rc == brs.BRS_ERR_UNSUPPORTED and not h.value


# ----------------------------------------------------------------- x-DST + y-Thomas form

XDST_SHAPES = [(32, 32, 4), (64, 96, 3), (256, 256, 3), (96, 64, 5)]


@pytest.mark.parametrize("dt,math", [("f64", "simt"), ("f32", "simt"), ("f32", "3xtf32"),
                                     ("f32", "tf32")])
@pytest.mark.parametrize("shape", XDST_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS, ids=["iso", "aniso_z", "aniso_yz"])
def test_plane_xdst_ythomas_form_parity(brs, orc, dt, math, shape, a, monkeypatch):
    """Plane block solved by a sine transform in x and exact y-Thomas per x-mode."""
    monkeypatch.setenv("BRSMOOTH_PLANE_FORM", "1")
    nx, ny, nz = shape
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = orc.sweep(u, b, a, block="plane", method="jacobi", omega=0.8)
    got = gpu_run(brs, u, b, a, dt=dt, math=math)
    tol = 2.0 ** -11 if math == "tf32" else TOL[dt]
    assert rel_max_err(got, ref) <= tol


FUSED_SHAPES = [(32, 32, 4), (64, 96, 3), (96, 64, 5), (160, 128, 2), (256, 256, 3),
                (128, 224, 3)]


@pytest.mark.parametrize("math", ["3xtf32", "tf32"])
@pytest.mark.parametrize("method", ["jacobi", "gs"])
@pytest.mark.parametrize("shape", FUSED_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS, ids=["iso", "aniso_z", "aniso_yz"])
def test_plane_fused_xdst_ythomas_product(brs, orc, shape, a, method, math, monkeypatch):
    """x-DST product with the y elimination in its epilogue (tile N = 64/128/256 holding a
    whole y line, partial mode tiles, y lines shorter than the tile): one sweep against the
    oracle, Jacobi and the even/odd plane order of GS."""
    monkeypatch.setenv("BRSMOOTH_PLANE_FORM", "1")
    monkeypatch.setenv("BRSMOOTH_TC_PERSISTENT", "1")
    monkeypatch.setenv("BRSMOOTH_PLANE_FUSE", "1")
    nx, ny, nz = shape
    u = rounded(initial_guess((nz, ny, nx)), "f32")
    b = rounded(rhs((nz, ny, nx)), "f32")
    if method == "jacobi":
        ref = orc.sweep(u, b, a, block="plane", method="jacobi", omega=0.8)
        got = gpu_run(brs, u, b, a, dt="f32", math=math, omega=0.8)
    else:
        ref = orc.sweep(u, b, a, block="plane", method="gs_zebra", omega=1.0)
        got = gpu_run(brs, u, b, a, dt="f32", math=math, method="gs", omega=1.0)
    # one TF32 pass per product: 2^-11 per solve; under GS the odd planes solve with the even
    # planes' new values, so two solves' errors add
    tol = (2.0 ** -11 if method == "jacobi" else 2.0 ** -10) if math == "tf32" else TOL["f32"]
    assert rel_max_err(got, ref) <= tol


@pytest.mark.parametrize("shape", [(33, 17, 4), (5, 70, 3), (1, 9, 2), (100, 3, 3)], ids=str)
def test_plane_xdst_form_ragged_simt(brs, orc, shape, monkeypatch):
    monkeypatch.setenv("BRSMOOTH_PLANE_FORM", "1")
    nx, ny, nz = shape
    a = (1.0, 0.1, 0.01)
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    ref = orc.sweep(u, b, a, block="plane", method="jacobi", omega=0.8)
    assert rel_max_err(gpu_run(brs, u, b, a, dt="f64", math="simt"), ref) <= 1e-12
    # chaotic GS in the same form (even planes, then odd planes)
    with brs.Context(nx, ny, nz, a, block="plane", method="gs", dtype="f64") as c:
        ut, bt = to_dev(u, "f64"), to_dev(b, "f64")
        c.sweep(ut, bt, 200)
        assert c.residual(ut, bt) < orc.residual_norm(u, b, a)


# ----------------------------------------------------------------- GS order, bench sizes

@pytest.mark.parametrize("dt,math", [("f64", "simt"), ("f32", "3xtf32"), ("f32", "simt")])
@pytest.mark.parametrize("shape", [(32, 32, 7), (64, 96, 6), (33, 17, 5)], ids=str)
@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_plane_gs_equals_oracle_zebra(brs, orc, dt, math, shape, omega):
    """Plane Gauss-Seidel on the GPU updates the even planes, then the odd planes from the
    new even ones: the oracle's zebra order, element by element (3 sweeps)."""
    nx, ny, nz = shape
    if math == "3xtf32" and (nx % 32 or ny % 32):
        pytest.skip("tensor-core plane products need nx, ny multiples of 32")
    a = (1.0, 1.0, 0.01)
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = u
    for _ in range(3):
        ref = orc.sweep(ref, b, a, block="plane", method="gs_zebra", omega=omega)
    got = gpu_run(brs, u, b, a, dt=dt, method="gs", nsweeps=3, math=math, omega=omega)
    assert rel_max_err(got, ref) <= TOL[dt]


@pytest.fixture(scope="module")
def plane512(orc):
    """512 x 512 x 3, a = (1, 0.1, 0.01) (the 512^3 defect-correction coefficients): inputs
    representable in FP32 (one input for every arithmetic) and the oracle's Jacobi sweep,
    whose banded Cholesky of the 512^2 plane block is factored once."""
    n, nz = 512, 3
    a = (1.0, 0.1, 0.01)
    u = rounded(initial_guess((nz, n, n)), "f32")
    b = rounded(rhs((nz, n, n)), "f32")
    return u, b, a, orc.sweep(u, b, a, block="plane", method="jacobi", omega=0.8)


@pytest.mark.parametrize("dt,math", [("f32", "3xtf32"), ("f32", "tf32"), ("f64", "simt")])
def test_plane_512_jacobi_vs_banded_cholesky(brs, plane512, dt, math):
    """The 512-wide plane solve that the 512^3 workload runs, every plane against the
    oracle's banded Cholesky."""
    u, b, a, ref = plane512
    got = gpu_run(brs, u, b, a, dt=dt, math=math)
    assert rel_max_err(got, ref) <= (2.0 ** -11 if math == "tf32" else TOL[dt])


@pytest.mark.parametrize("dt,math", [("f32", "3xtf32"), ("f32", "tf32"), ("f64", "simt")])
def test_plane_512_single_mode_damping(brs, orc, dt, math):
    """512 x 512 x 4: a sine mode is scaled by the closed-form g = 1 - omega lambda/mu."""
    nx = ny = 512
    nz = 4
    a = (1.0, 0.1, 0.01)
    g = orc.mode_factor(nx, ny, nz, a, "plane", 0.8)
    tol = 2.0 ** -10 if math == "tf32" else 4 * TOL[dt]
    with brs.Context(nx, ny, nz, a, block="plane", method="jacobi", dtype=dt,
                     plane_math=math) as ctx:
        for (p, q, r) in [(1, 1, 1), (512, 512, 4), (37, 301, 2)]:
            m = rounded(sine_mode(nx, ny, nz, p, q, r), dt)
            ut, bt = to_dev(m, dt), to_dev(np.zeros_like(m), dt)
            ctx.sweep(ut, bt, 1)
            got = to_np(ut)
            err = np.max(np.abs(got - g[r - 1, q - 1, p - 1] * m)) / np.max(np.abs(m))
            assert err <= tol, (p, q, r, err)
        assert ctx.last_error() == 0


@pytest.mark.parametrize("dt,math", [("f32", "3xtf32"), ("f64", "simt")])
def test_full_size_256_plane_three_sweeps_in_one_call(brs, orc, dt, math, monkeypatch):
    """256^3 plane Jacobi (a = (1, 1, 0.01)) in the per-sweep form (the x-sine form of
    calls of several sweeps switched off; it is tested in test_gpu_plane_modes.py): 3 sweeps
    in one call equal 3 one-sweep calls bit for bit, and sampled planes equal the oracle
    after 3 sweeps (a plane after s sweeps depends only on planes within s of it)."""
    import torch

    monkeypatch.setenv("BRSMOOTH_PLANE_MODES", "0")

    n, K = 256, 3
    a = (1.0, 1.0, 0.01)
    td = torch.float64 if dt == "f64" else torch.float32
    gen = torch.Generator(device="cuda").manual_seed(13)
    u0 = (torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1).to(td)
    bt = ((torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1)
          / (n + 1) ** 2).to(td)
    with brs.Context(n, n, n, a, block="plane", method="jacobi", dtype=dt,
                     plane_math=math) as ctx:
        one = u0.clone()
        ctx.sweep(one, bt, K)
        many = u0.clone()
        for _ in range(K):
            ctx.sweep(many, bt, 1)
        torch.cuda.synchronize()
        assert ctx.last_error() == 0
    assert torch.equal(one, many)
    u, b, got = to_np(u0), to_np(bt), to_np(one)
    for k in (0, 131, n - 1):
        k0, k1 = max(0, k - K), min(n, k + K + 1)
        sub = u[k0:k1]
        for _ in range(K):
            sub = orc.sweep(sub, b[k0:k1], a, block="plane", method="jacobi", omega=0.8)
        assert rel_max_err(got[k], sub[k - k0]) <= TOL[dt]
