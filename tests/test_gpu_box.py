"""Box-block sweeps on the GPU (precomputed inverse applied as one matrix product per
pass) against the FP64 oracle.

The library builds the inverse from the block's own sine basis; the oracle from a dense
Cholesky factorisation.  Jacobi and the two-colour Gauss-Seidel order are deterministic,
so both are compared element by element, sweep by sweep.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np

pytestmark = pytest.mark.gpu

PAPER_SIZES = [(2, 2, 2), (4, 2, 2), (4, 4, 2), (4, 4, 4), (8, 4, 4), (8, 8, 4), (8, 8, 8)]
COEFFS = [(1.0, 1.0, 1.0), (1.0, 0.1, 0.01)]
# grids x boxes spanning several 128-row tiles with a ragged last tile, odd block counts
# per axis (two-colour passes of unequal size), boxes with bx not a multiple of 4
CASES = [((40, 24, 16), (4, 4, 4)), ((64, 32, 24), (8, 8, 8)), ((64, 64, 32), (8, 4, 4)),
         ((36, 20, 12), (4, 2, 2)), ((30, 18, 10), (2, 2, 2)), ((24, 18, 15), (6, 3, 5)),
         ((9, 7, 5), (1, 1, 1)), ((48, 8, 8), (48, 1, 1)), ((12, 12, 3), (12, 12, 1)),
         # y-lines and z-lines (the blocks for y- or z-dominant coefficients)
         ((10, 40, 6), (1, 40, 1)), ((6, 9, 36), (1, 1, 36))]


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def gpu_sweeps(brs, u, b, a, box, *, dt, method="jacobi", nsweeps=1, math="auto", omega=0.0):
    """The iterate after each of nsweeps sweeps."""
    nz, ny, nx = u.shape
    out = []
    with brs.Context(nx, ny, nz, a, block="box", box=box, method=method, dtype=dt,
                     plane_math=math, omega=omega) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        for _ in range(nsweeps):
            ctx.sweep(ut, bt, 1)
            out.append(to_np(ut))
        assert ctx.last_error() == 0
    return out


def inputs(shape, dt):
    nx, ny, nz = shape
    return rounded(initial_guess((nz, ny, nx)), dt), rounded(rhs((nz, ny, nx)), dt)


def oracle_steps(orc, u, b, a, box, method, omega, nsweeps):
    out = []
    for _ in range(nsweeps):
        u = orc.sweep(u, b, a, block="box", box=box, method=method, omega=omega)
        out.append(u)
    return out


@pytest.mark.parametrize("dt,math", [("f64", "auto"), ("f32", "simt"), ("f32", "3xtf32")])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
@pytest.mark.parametrize("method", ["jacobi", "gs"])
def test_box_parity(brs, orc, dt, math, case, method):
    shape, box = case
    n = box[0] * box[1] * box[2]
    if math == "3xtf32" and (n % 4 or n < 32):
        pytest.skip("tensor path needs bx*by*bz a multiple of 4 and >= 32")
    a = (1.0, 0.1, 0.01)
    u, b = inputs(shape, dt)
    om = 0.8 if method == "jacobi" else 1.0
    ref = oracle_steps(orc, u, b, a, box, "jacobi" if method == "jacobi" else "gs_zebra", om, 3)
    # FP32 sweeps start each step from the device's own iterate; compare sweep by sweep
    # against the oracle applied to that iterate (per-sweep parity)
    got = gpu_sweeps(brs, u, b, a, box, dt=dt, method=method, nsweeps=3, math=math)
    assert rel_max_err(got[0], ref[0]) <= TOL[dt]
    prev = got[0]
    for k in (1, 2):
        step = orc.sweep(prev, b, a, block="box", box=box,
                         method="jacobi" if method == "jacobi" else "gs_zebra", omega=om)
        assert rel_max_err(got[k], step) <= TOL[dt], k
        prev = got[k]
    if dt == "f64":
        assert rel_max_err(got[2], ref[2]) <= TOL[dt]


@pytest.mark.parametrize("box", PAPER_SIZES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_paper_block_sizes_64cubed(brs, orc, box, dt):
    """The paper's seven block sizes on its 64^3 patch: Jacobi and GS, one sweep each."""
    a = (1.0, 1.0, 1.0)
    u, b = inputs((64, 64, 64), dt)
    for method, omethod, om in (("jacobi", "jacobi", 0.8), ("gs", "gs_zebra", 1.0)):
        ref = orc.sweep(u, b, a, block="box", box=box, method=omethod, omega=om)
        got = gpu_sweeps(brs, u, b, a, box, dt=dt, method=method)[0]
        assert rel_max_err(got, ref) <= TOL[dt], method


@pytest.mark.parametrize("box", [(8, 8, 8), (4, 4, 4), (8, 4, 4)], ids=lambda s: "x".join(map(str, s)))
def test_tf32_box_within_derived_bound(brs, orc, box):
    """Single TF32: both operands carry a relative rounding of at most u = 2^-11 each, so
    |x_gpu - x| <= (2u + u^2 + n 2^-24) sum_m |Ahat_lm| |R_m| <= that * ||Ahat||_inf * max|R|,
    with max|R| <= max|b| + 2 (ax + ay + az) max|u|; the update scales it by omega."""
    a = (1.0, 1.0, 1.0)
    u, b = inputs((64, 64, 32), "f32")
    ref = orc.sweep(u, b, a, block="box", box=box, method="jacobi", omega=0.8)
    got = gpu_sweeps(brs, u, b, a, box, dt="f32", method="jacobi", math="tf32")[0]
    n = box[0] * box[1] * box[2]
    inv_norm = np.abs(orc.box_inverse(box, a)).sum(axis=1).max()
    rmax = np.abs(b).max() + 2 * sum(a) * np.abs(u).max()
    uu = 2.0 ** -11
    bound = 0.8 * (2 * uu + uu * uu + n * 2.0 ** -24) * inv_norm * rmax + 1e-6 * np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= bound
    assert rel_max_err(got, ref) <= 2e-3  # and it is a TF32-level answer, not garbage


def test_box_converges_fp64(brs, orc):
    n = 32
    a = (1.0, 1.0, 1.0)
    b = rhs((n, n, n))
    ref = orc.exact_solve(b, a)
    with brs.Context(n, n, n, a, block="box", box=(4, 4, 4), method="gs", dtype="f64") as ctx:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        ctx.sweep(ut, bt, 700)  # the oracle's two-colour GS reaches 1e-11 after 623
        got = to_np(ut)
    assert rel_max_err(got, ref) <= 1e-10


@pytest.mark.parametrize("a,box", [((0.01, 1.0, 0.01), (1, 32, 1)), ((0.01, 0.01, 1.0), (1, 1, 32))],
                         ids=["y_dominant", "z_dominant"])
def test_lines_along_the_strong_coupling_converge_faster(brs, orc, a, box):
    """Strongly anisotropic coefficients: lines along the dominant direction (1 x 32 x 1 or
    1 x 1 x 32 boxes) contract the residual far faster than x-lines, as the oracle's ten-sweep
    ratios on the same input show; the GPU ratios match the oracle's."""
    n = 32
    u, b = inputs((n, n, n), "f64")
    b = np.zeros_like(b)
    r0 = orc.residual_norm(u, b, a)
    ratios = {}
    for blk in (box, (n, 1, 1)):
        got = gpu_sweeps(brs, u, b, a, blk, dt="f64", method="jacobi", nsweeps=10)[-1]
        ref = u
        for _ in range(10):
            ref = orc.sweep(ref, b, a, block="box", box=blk, method="jacobi", omega=0.8)
        ratios[blk] = orc.residual_norm(got, b, a) / r0
        assert abs(ratios[blk] - orc.residual_norm(ref, b, a) / r0) <= 1e-10
    assert ratios[box] < 0.05 * ratios[(n, 1, 1)], ratios


@pytest.mark.parametrize("bn", ["0", "256"], ids=["tileN128", "tileN256"])
def test_box_full_size_one_sweep(brs, orc, bn, monkeypatch):
    """256^3 FP32, 8^3 boxes, split-TF32, the launch the benchmark times: one Jacobi sweep
    against the oracle over the whole grid (product tiles of 128 and of 256 local cells)."""
    monkeypatch.setenv("BRSMOOTH_BOX_BN", bn)
    nx = ny = nz = 256
    a = (1.0, 1.0, 1.0)
    u, b = inputs((nx, ny, nz), "f32")
    ref = orc.sweep(u, b, a, block="box", box=(8, 8, 8), method="jacobi", omega=0.8)
    got = gpu_sweeps(brs, u, b, a, (8, 8, 8), dt="f32", method="jacobi")[0]
    assert rel_max_err(got, ref) <= TOL["f32"]


def test_box_argument_errors(brs):
    with pytest.raises(brs.BrsError) as e:
        brs.Context(30, 16, 16, block="box", box=(4, 4, 4), dtype="f32")  # 4 does not divide 30
    assert e.value.code == brs.BRS_ERR_ARG
    with pytest.raises(brs.BrsError) as e:
        brs.Context(16, 16, 16, block="box", box=(0, 4, 4), dtype="f32")
    assert e.value.code == brs.BRS_ERR_ARG
    with pytest.raises(brs.BrsError) as e:
        brs.Context(16, 16, 32, block="box", box=(16, 16, 4), dtype="f32")  # n = 1024 > 512
    assert e.value.code == brs.BRS_ERR_UNSUPPORTED
    with pytest.raises(brs.BrsError) as e:
        brs.Context(16, 16, 16, block="box", box=(4, 4, 4), dtype="f64", plane_math="3xtf32")
    assert e.value.code == brs.BRS_ERR_UNSUPPORTED
    with pytest.raises(brs.BrsError) as e:
        brs.Context(16, 16, 16, block="box", box=(2, 2, 2), dtype="f32", plane_math="tf32")
    assert e.value.code == brs.BRS_ERR_UNSUPPORTED


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("case", [((32, 32, 16), (8, 8, 8)), ((24, 18, 15), (6, 3, 5)),
                                  ((10, 40, 6), (1, 40, 1)), ((40, 24, 16), (8, 4, 4)),
                                  ((28, 14, 8), (7, 7, 1))],
                         ids=lambda c: "b" + "x".join(map(str, c[1])))
@pytest.mark.parametrize("method", ["jacobi", "gs"])
def test_box_parity_classes_equal_full_product(brs, orc, dt, case, method, monkeypatch):
    """CUDA-core boxes: the inverse applied by parity classes (rows folded into sums and
    differences of mirrored cells, one product per class, unfolded in the update) against the
    full n x n product (BRSMOOTH_BOX_FOLD=0), two sweeps, even and odd box extents (every
    case has a class of 16 or more cells, so the classes are used)."""
    shape, box = case
    a = (1.0, 0.1, 0.01)
    u, b = inputs(shape, dt)
    fold = gpu_sweeps(brs, u, b, a, box, dt=dt, method=method, nsweeps=2, math="simt")
    monkeypatch.setenv("BRSMOOTH_BOX_FOLD", "0")
    full = gpu_sweeps(brs, u, b, a, box, dt=dt, method=method, nsweeps=2, math="simt")
    tol = 1e-13 if dt == "f64" else 2 * TOL["f32"]
    assert rel_max_err(fold[1], full[1]) <= tol


def test_box_parity_classes_full_size_fp64_gs(brs, orc):
    """256^3 FP64 two-colour GS with 8^3 boxes (the paper's block and precision), by parity
    classes: one sweep on sampled blocks against the oracle's zebra order."""
    import torch

    n = 256
    a = (1.0, 1.0, 1.0)
    box = (8, 8, 8)
    gen = torch.Generator(device="cuda").manual_seed(29)
    u0 = torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
    bt = (torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen) * 2 - 1) \
        / (n + 1) ** 2
    with brs.Context(n, n, n, a, block="box", box=box, method="gs", dtype="f64") as ctx:
        ut = u0.clone()
        ctx.sweep(ut, bt, 1)
        torch.cuda.synchronize()
        assert ctx.last_error() == 0
    u, b, got = to_np(u0), to_np(bt), to_np(ut)
    # a block after one zebra sweep depends on the blocks within distance 2 (colours kept)
    for (bi, bj, bk) in [(0, 0, 0), (17, 9, 30), (31, 31, 31)]:
        lo = [max(0, q - 2) for q in (bi, bj, bk)]
        if sum(lo) % 2:
            d = next(q for q in range(3) if lo[q] > 0)
            lo[d] -= 1
        hi = [min(32, q + 3) for q in (bi, bj, bk)]
        sl = (slice(lo[2] * 8, hi[2] * 8), slice(lo[1] * 8, hi[1] * 8), slice(lo[0] * 8, hi[0] * 8))
        ref = orc.sweep(np.ascontiguousarray(u[sl]), np.ascontiguousarray(b[sl]), a, block="box",
                        box=box, method="gs_zebra", omega=1.0)
        c = [(q - l) * 8 for q, l in zip((bi, bj, bk), lo)]
        own = ref[c[2]:c[2] + 8, c[1]:c[1] + 8, c[0]:c[0] + 8]
        g = got[bk * 8:bk * 8 + 8, bj * 8:bj * 8 + 8, bi * 8:bi * 8 + 8]
        assert float(np.max(np.abs(g - own))) <= 1e-12 * float(np.max(np.abs(u))), (bi, bj, bk)
