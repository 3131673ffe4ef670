"""x-line block sweeps on the GPU against the FP64 oracle (Sec. 2, Alg. 1 / Alg. 2).

Block Jacobi is deterministic: one GPU sweep from a given iterate is compared element by
element with the oracle's sweep from the same iterate (relative max-norm <= 1e-12 FP64,
<= 1e-5 FP32).  FP64 chaotic Gauss-Seidel visits the lines in the red-black order (j+k even,
then odd), which the oracle's zebra order reproduces element by element.  FP32 chaotic
Gauss-Seidel is not reproducible; it is judged by the componentwise Perron bound, a
residual bracket and convergence to the exact solution.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs, sine_mode
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np

pytestmark = pytest.mark.gpu

# (nx, ny, nz): TMA-path shapes, ragged y tiles, the plain-load path (rows not 16-byte
# aligned or nx not a multiple of the lane chunk), degenerate 1-cell axes, widest lines.
SHAPES = [(32, 32, 32), (24, 13, 7), (33, 17, 9), (48, 20, 11), (1, 1, 1), (4, 1, 1),
          (1, 5, 3), (130, 5, 5), (100, 7, 5), (256, 9, 6), (384, 5, 4), (512, 3, 3),
          (16, 16, 40)]
COEFFS = [(1.0, 1.0, 1.0), (1.0, 1.0, 0.01), (1.0, 0.1, 0.01)]


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def gpu_sweep(brs, u, b, a, *, dt, method="jacobi", omega=0.0, nsweeps=1, block="line"):
    nz, ny, nx = u.shape
    with brs.Context(nx, ny, nz, a, block=block, method=method, dtype=dt, omega=omega) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        ctx.sweep(ut, bt, nsweeps)
        out = to_np(ut)
        assert ctx.last_error() == 0
    return out


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS, ids=["iso", "aniso_z", "aniso_yz"])
def test_jacobi_one_sweep_parity(brs, orc, dt, shape, a):
    nx, ny, nz = shape
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = orc.sweep(u, b, a, block="line", method="jacobi", omega=0.8)
    got = gpu_sweep(brs, u, b, a, dt=dt)
    assert rel_max_err(got, ref) <= TOL[dt]


@pytest.mark.parametrize("shape", [(24, 13, 7), (33, 17, 9), (1, 5, 3), (4, 1, 1), (256, 9, 6),
                                   (512, 3, 3), (7, 32, 5)], ids=str)
@pytest.mark.parametrize("omega", [1.0, 0.7])
@pytest.mark.parametrize("a", [(1.0, 1.0, 1.0), (1.0, 0.1, 0.01)], ids=["iso", "aniso_yz"])
def test_gs_f64_red_black_equals_oracle_zebra(brs, orc, shape, omega, a):
    """FP64 x-line GS = the oracle's zebra order (j+k even lines, then odd), 3 sweeps."""
    nx, ny, nz = shape
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    ref = u
    for _ in range(3):
        ref = orc.sweep(ref, b, a, block="line", method="gs_zebra", omega=omega)
    got = gpu_sweep(brs, u, b, a, dt="f64", method="gs", omega=omega, nsweeps=3)
    assert rel_max_err(got, ref) <= 1e-12


@pytest.mark.parametrize("shape", [(32, 32, 32), (33, 17, 9), (256, 9, 6), (100, 7, 5)], ids=str)
def test_f64_lane_scan_kernel_still_matches(brs, orc, shape, monkeypatch):
    """BRSMOOTH_LINE_SEQ=0 selects the lane-scan kernel for FP64 (also what the adjoint's
    undamped sweeps run); it stays within 1e-12 of the oracle."""
    monkeypatch.setenv("BRSMOOTH_LINE_SEQ", "0")
    nx, ny, nz = shape
    a = (1.0, 1.0, 0.01)
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    ref = orc.sweep(orc.sweep(u, b, a, block="line", omega=0.8), b, a, block="line", omega=0.8)
    got = gpu_sweep(brs, u, b, a, dt="f64", nsweeps=2)
    assert rel_max_err(got, ref) <= 1e-12


@pytest.mark.parametrize("omega", [0.5, 1.0, 1.3])
def test_jacobi_omega(brs, orc, omega):
    shape = (3, 8, 40)
    u, b = initial_guess(shape), rhs(shape)
    ref = orc.sweep(u, b, (1.0, 0.5, 2.0), block="line", method="jacobi", omega=omega)
    got = gpu_sweep(brs, u, b, (1.0, 0.5, 2.0), dt="f64", omega=omega)
    assert rel_max_err(got, ref) <= 1e-12


def test_trajectory_32cubed_residual_per_sweep(brs, orc):
    """32^3, a=(1,1,1), h=1/33, u0=0: 10 line-Jacobi sweeps, iterate and ||r|| per sweep."""
    n = 32
    a = (1.0, 1.0, 1.0)
    b = rhs((n, n, n))
    u0 = np.zeros_like(b)
    traj = orc.trajectory(u0, b, a, 10, block="line", method="jacobi", omega=0.8)
    with brs.Context(n, n, n, a, block="line", method="jacobi", dtype="f64") as ctx:
        ut, bt = to_dev(u0, "f64"), to_dev(b, "f64")
        for k in range(10):
            ctx.sweep(ut, bt, 1)
            got = to_np(ut)
            assert rel_max_err(got, traj[k]) <= 1e-12
            nrm = ctx.residual(ut, bt)
            ref = orc.residual_norm(traj[k], b, a)
            assert abs(nrm - ref) <= 1e-12 * ref


def test_multi_sweep_odd_and_even_counts(brs, orc):
    shape = (6, 10, 24)
    u, b = initial_guess(shape), rhs(shape)
    a = (1.0, 1.0, 1.0)
    for ns in (0, 1, 2, 5):
        ref = u
        for _ in range(ns):
            ref = orc.sweep(ref, b, a, block="line", method="jacobi", omega=0.8)
        got = gpu_sweep(brs, u, b, a, dt="f64", nsweeps=ns)
        assert rel_max_err(got, ref) <= 1e-12


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_jacobi_is_bitwise_deterministic(brs, dt):
    shape = (20, 30, 64)
    u, b = initial_guess(shape), rhs(shape)
    g1 = gpu_sweep(brs, u, b, (1, 1, 1), dt=dt, nsweeps=3)
    g2 = gpu_sweep(brs, u, b, (1, 1, 1), dt=dt, nsweeps=3)
    assert np.array_equal(g1, g2)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (33, 17, 9), (1, 1, 1)], ids=str)
def test_residual_and_norm(brs, orc, dt, shape):
    import torch

    nx, ny, nz = shape
    a = (1.0, 0.1, 0.01)
    u = rounded(initial_guess((nz, ny, nx)), dt)
    b = rounded(rhs((nz, ny, nx)), dt)
    ref = orc.residual(u, b, a)
    with brs.Context(nx, ny, nz, a, dtype=dt) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        r = torch.empty_like(ut)
        nrm = ctx.residual(ut, bt, r)
    tol = 1e-13 if dt == "f64" else 2e-6
    scale = np.max(np.abs(b)) + 2 * sum(a) * np.max(np.abs(u))
    assert np.max(np.abs(to_np(r) - ref)) <= tol * scale
    assert abs(nrm - np.linalg.norm(ref)) <= (1e-12 if dt == "f64" else 1e-5) * np.linalg.norm(ref)


def test_host_buffer_path_matches_device_path(brs):
    shape = (16, 24, 32)
    u, b = initial_guess(shape), rhs(shape)
    dev = gpu_sweep(brs, u, b, (1, 1, 1), dt="f64", nsweeps=3)
    with brs.Context(32, 24, 16, (1, 1, 1)) as ctx:
        uh = u.copy()
        ctx.sweep_host(uh, b, 3)
    assert np.array_equal(uh, dev)


def test_async_host_path_on_two_streams(brs):
    """Independent problems alternating over two contexts and two streams through the
    asynchronous host entry point (the end-to-end benchmark's pattern): each result equals
    the synchronous call's, bit for bit."""
    import torch

    shape = (16, 24, 32)
    b = torch.from_numpy(rhs(shape)).pin_memory()
    us = [torch.from_numpy(initial_guess(shape)).pin_memory(),
          torch.from_numpy(0.5 * initial_guess(shape)).pin_memory()]
    refs = []
    for u in us:
        with brs.Context(32, 24, 16, (1, 0.5, 0.25)) as ctx:
            uh = u.clone()
            ctx.sweep_host(uh, b, 7)
            ctx.sweep_host(uh, b, 7)
            refs.append(uh)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ctxs = [brs.Context(32, 24, 16, (1, 0.5, 0.25)) for _ in range(2)]
    try:
        for q in range(4):  # two calls per problem, enqueued without waiting
            ctxs[q % 2].sweep_host(us[q % 2], b, 7, stream=streams[q % 2], wait=False)
        torch.cuda.synchronize()
        for q in range(2):
            assert ctxs[q].last_error() == 0
            assert torch.equal(us[q], refs[q])
    finally:
        for cx in ctxs:
            cx.close()


def test_argument_errors(brs):
    import torch

    with brs.Context(8, 8, 8) as ctx:
        u = torch.zeros(512, dtype=torch.float64, device="cuda")
        b = torch.zeros(513, dtype=torch.float64, device="cuda")
        rc = brs.brsmooth_sweep(ctx.h, u.data_ptr(), u.data_ptr(), 1, 0)
        assert rc == brs.BRS_ERR_ARG  # u aliases b
        rc = brs.brsmooth_sweep(ctx.h, u.data_ptr(), b[1:].data_ptr(), 1, 0)
        assert rc == brs.BRS_ERR_ARG  # misaligned b
        rc = brs.brsmooth_sweep(ctx.h, u.data_ptr(), b.data_ptr(), -1, 0)
        assert rc == brs.BRS_ERR_ARG
        assert brs.brsmooth_sweep(ctx.h, u.data_ptr(), b.data_ptr(), 0, 0) == brs.BRS_OK
    p = brs.brs_params(2000, 4, 4, 1.0, 1.0, 1.0, 0, 0, 0, 0.0, 0)
    rc, h = brs.brsmooth_create(p)
    assert rc == brs.BRS_ERR_UNSUPPORTED and not h.value


# ----------------------------------------------------------------- chaotic Gauss-Seidel

@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 40, 48), (33, 17, 9)], ids=str)
def test_chaotic_gs_perron_bound(brs, orc, dt, shape):
    """b = 0, u0 = positive mode: 0 <= u_k <= g_111^k u0 componentwise for any race outcome.

    A is an M-matrix, so M^{-1} >= 0 and N = M - A >= 0; every read returns an old or a
    newer (smaller, still non-negative) value, so each update is bounded by the Jacobi
    update of the old iterate, which maps the positive sine mode to g_111 times itself.
    """
    nx, ny, nz = shape
    a = (1.0, 1.0, 1.0)
    m = sine_mode(nx, ny, nz, 1, 1, 1)
    g = orc.mode_factor(nx, ny, nz, a, "line", 1.0)[0, 0, 0]
    slack = 1e-13 if dt == "f64" else 2e-6
    with brs.Context(nx, ny, nz, a, block="line", method="gs", dtype=dt) as ctx:
        ut = to_dev(m, dt)
        bt = to_dev(np.zeros_like(m), dt)
        mr = to_np(ut)
        for k in range(1, 9):
            ctx.sweep(ut, bt, 1)
            u = to_np(ut)
            assert np.all(u >= -slack)
            assert np.all(u <= g ** k * mr + slack * (1 + k))


def test_chaotic_gs_residual_bracket_32cubed(brs, orc):
    """||r_k|| of chaotic line GS lies between the ordered GS sweeps and Jacobi (omega=1)."""
    n = 32
    a = (1.0, 1.0, 1.0)
    b = rhs((n, n, n))
    u0 = initial_guess((n, n, n))
    refs = {}
    for meth, om in (("jacobi", 1.0), ("gs_lex", 1.0), ("gs_zebra", 1.0), ("gs_reverse", 1.0)):
        u, norms = u0, []
        for _ in range(10):
            u = orc.sweep(u, b, a, block="line", method=meth, omega=om)
            norms.append(orc.residual_norm(u, b, a))
        refs[meth] = np.array(norms)
    lo = np.minimum(np.minimum(refs["gs_lex"], refs["gs_zebra"]), refs["gs_reverse"])
    with brs.Context(n, n, n, a, block="line", method="gs", dtype="f64") as ctx:
        ut, bt = to_dev(u0, "f64"), to_dev(b, "f64")
        for k in range(10):
            ctx.sweep(ut, bt, 1)
            r = ctx.residual(ut, bt)
            assert 0.9 * lo[k] <= r <= 1.1 * refs["jacobi"][k], (k, r, lo[k], refs["jacobi"][k])


def test_chaotic_gs_converges_to_exact_solution(brs, orc):
    n = 32
    a = (1.0, 1.0, 1.0)
    b = rhs((n, n, n))
    ustar = orc.exact_solve(b, a)
    with brs.Context(n, n, n, a, block="line", method="gs", dtype="f64") as ctx:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        ctx.sweep(ut, bt, 6000)  # rho ~ 0.9932 when each plane reads old neighbours
        assert ctx.last_error() == 0
        assert rel_max_err(to_np(ut), ustar) <= 1e-10


def test_jacobi_converges_to_exact_solution(brs, orc):
    n = 32
    a = (1.0, 1.0, 0.01)
    b = rhs((n, n, n))
    ustar = orc.exact_solve(b, a)
    with brs.Context(n, n, n, a, block="line", method="jacobi", dtype="f64") as ctx:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        ctx.sweep(ut, bt, 6000)  # rho ~ 0.9928 for a = (1, 1, 0.01)
        assert rel_max_err(to_np(ut), ustar) <= 1e-10


# ----------------------------------------------------------------- full-size sampled parity

def _sampled_lines(orc, u, b, a, got, lines, omega=0.8):
    """Oracle Jacobi for selected lines from a 3x3-line neighbourhood sub-grid."""
    nz, ny, nx = u.shape
    worst = 0.0
    for (j, k) in lines:
        j0, j1 = max(0, j - 1), min(ny, j + 2)
        k0, k1 = max(0, k - 1), min(nz, k + 2)
        sub = orc.sweep(u[k0:k1, j0:j1], b[k0:k1, j0:j1], a, block="line", method="jacobi",
                        omega=omega)
        ref = sub[k - k0, j - j0]
        worst = max(worst, rel_max_err(got[k, j], ref))
    return worst


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("a", [(1.0, 1.0, 1.0), (1.0, 1.0, 0.01)], ids=["iso", "aniso"])
def test_full_size_256_sampled_lines(brs, orc, dt, a):
    """256^3 in the benchmark's launch configuration; ~60 lines checked against the oracle."""
    import torch

    n = 256
    rng = np.random.default_rng(7)
    ut = torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=torch.Generator(
        device="cuda").manual_seed(2)) * 2 - 1
    bt = (torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=torch.Generator(
        device="cuda").manual_seed(1)) * 2 - 1) / (n + 1) ** 2
    if dt == "f32":
        ut, bt = ut.float(), bt.float()
    u, b = to_np(ut), to_np(bt)
    with brs.Context(n, n, n, a, dtype=dt) as ctx:
        ctx.sweep(ut, bt, 1)
        torch.cuda.synchronize()
        assert ctx.last_error() == 0
    got = to_np(ut)
    lines = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (7, 8), (8, 7), (128, 129)]
    lines += [tuple(x) for x in rng.integers(0, n, size=(50, 2))]
    assert _sampled_lines(orc, u, b, a, got, lines) <= TOL[dt]


def _sampled_lines_after(orc, u, b, a, got, lines, nsweeps, omega=0.8):
    """Oracle Jacobi after `nsweeps` sweeps for selected lines, each from the sub-grid of
    lines within distance `nsweeps` in j and k (a line's value after s sweeps depends only
    on the lines within distance s; cut edges that are not grid boundaries corrupt lines at
    most s-1 away from them, never the centre)."""
    nz, ny, nx = u.shape
    worst = 0.0
    for (j, k) in lines:
        j0, j1 = max(0, j - nsweeps), min(ny, j + nsweeps + 1)
        k0, k1 = max(0, k - nsweeps), min(nz, k + nsweeps + 1)
        sub_u, sub_b = u[k0:k1, j0:j1], b[k0:k1, j0:j1]
        for _ in range(nsweeps):
            sub_u = orc.sweep(sub_u, sub_b, a, block="line", method="jacobi", omega=omega)
        worst = max(worst, rel_max_err(got[k, j], sub_u[k - k0, j - j0]))
    return worst


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_full_size_256_five_sweeps_in_one_call(brs, orc, dt):
    """256^3 x-line Jacobi in the benchmark's launch configuration, 5 sweeps in one call
    (back-to-back dependent launches): bitwise equal to 5 one-sweep calls, and sampled lines
    equal to the oracle after 5 sweeps."""
    import torch

    n, K = 256, 5
    a = (1.0, 1.0, 1.0)
    td = torch.float64 if dt == "f64" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(11)
    u0 = (torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=g) * 2 - 1).to(td)
    bt = ((torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=g) * 2 - 1)
          / (n + 1) ** 2).to(td)
    with brs.Context(n, n, n, a, dtype=dt) as ctx:
        one = u0.clone()
        ctx.sweep(one, bt, K)
        many = u0.clone()
        for _ in range(K):
            ctx.sweep(many, bt, 1)
        torch.cuda.synchronize()
        assert ctx.last_error() == 0
    assert torch.equal(one, many)
    u, b, got = to_np(u0), to_np(bt), to_np(one)
    rng = np.random.default_rng(5)
    lines = [(0, 0), (n - 1, n - 1), (3, n - 2), (128, 129)]
    lines += [tuple(x) for x in rng.integers(0, n, size=(12, 2))]
    assert _sampled_lines_after(orc, u, b, a, got, lines, K) <= TOL[dt]


# ----------------------------------------------------------------- two-warp lines (385-512)

PAIR_SHAPES = [(416, 9, 5), (480, 6, 7), (512, 13, 8), (448, 1, 3)]


@pytest.mark.parametrize("shape", PAIR_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("a", COEFFS + [(2.0, 0.001, 0.001)],
                         ids=["iso", "aniso_z", "aniso_yz", "strong_x"])
def test_two_warp_lines_jacobi_parity(brs, orc, shape, a):
    """FP32 lines of 416-512 cells (two warps per line, the halves' carries crossing through
    shared memory): one sweep and a call of three sweeps against the oracle, and within the
    tolerance of the one-warp form (BRSMOOTH_LINE_PAIR=0)."""
    nx, ny, nz = shape
    u = rounded(initial_guess((nz, ny, nx)), "f32")
    b = rounded(rhs((nz, ny, nx)), "f32")
    ref1 = orc.sweep(u, b, a, block="line", method="jacobi", omega=0.8)
    ref3 = orc.sweep(orc.sweep(ref1, b, a, block="line", omega=0.8), b, a, block="line",
                     omega=0.8)
    assert rel_max_err(gpu_sweep(brs, u, b, a, dt="f32"), ref1) <= TOL["f32"]
    assert rel_max_err(gpu_sweep(brs, u, b, a, dt="f32", nsweeps=3), ref3) <= TOL["f32"]


def test_two_warp_lines_equal_one_warp_form(brs, orc, monkeypatch):
    nx, ny, nz = 512, 11, 6
    a = (1.0, 0.1, 0.01)
    u = rounded(initial_guess((nz, ny, nx)), "f32")
    b = rounded(rhs((nz, ny, nx)), "f32")
    pair = gpu_sweep(brs, u, b, a, dt="f32", nsweeps=2)
    monkeypatch.setenv("BRSMOOTH_LINE_PAIR", "0")
    one = gpu_sweep(brs, u, b, a, dt="f32", nsweeps=2)
    assert rel_max_err(pair, one) <= 2 * TOL["f32"]


def test_two_warp_lines_chaotic_gs_perron_and_convergence(brs, orc):
    """Chaotic GS on 512-cell lines: the Perron bound on the slowest sine mode (b = 0) and
    convergence to A^{-1} b."""
    nx, ny, nz = 512, 6, 5
    a = (1.0, 1.0, 1.0)
    m = sine_mode(nx, ny, nz, 1, 1, 1)
    g = orc.mode_factor(nx, ny, nz, a, "line", 1.0)[0, 0, 0]
    with brs.Context(nx, ny, nz, a, block="line", method="gs", dtype="f32") as ctx:
        ut, bt = to_dev(m, "f32"), to_dev(np.zeros_like(m), "f32")
        mr = to_np(ut)
        for k in range(1, 6):
            ctx.sweep(ut, bt, 1)
            got = to_np(ut)
            assert np.all(got >= -1e-6 * k) and np.all(got <= g ** k * mr + 2e-6 * (1 + k))
        b = rounded(rhs((nz, ny, nx)), "f32")
        ut, bt = to_dev(np.zeros_like(b), "f32"), to_dev(b, "f32")
        ctx.sweep(ut, bt, 300)
        assert ctx.last_error() == 0
        assert rel_max_err(to_np(ut), orc.exact_solve(b, a)) <= 1e-4
