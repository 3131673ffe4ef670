"""y-line and z-line block sweeps on the GPU (x-line sweeps of the grid with permuted axes)
against the oracle's 1 x ny x 1 and 1 x 1 x nz box sweeps (dense Cholesky inverse), which
the oracle pins separately to its x-line sweep of the permuted grid.

Jacobi is deterministic: element-wise parity, sweep by sweep and for several sweeps in one
call (the permutation in, the inner sweeps with the Jacobi buffer swap, the permutation
back).  Chaotic GS: convergence to A^{-1} b.  At 256^3 (the benchmark's launch) one sweep
is compared with the oracle's x-line sweep of the permuted grid.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np

pytestmark = pytest.mark.gpu

# (nx, ny, nz): ragged tiles, odd extents, line lengths from 3 to 96
SHAPES = [(16, 24, 8), (13, 7, 11), (8, 96, 6), (33, 17, 40), (5, 3, 64)]
COEFFS = {"yline": [(0.01, 1.0, 0.01), (1.0, 0.5, 0.25)],
          "zline": [(0.01, 0.01, 1.0), (0.3, 2.0, 0.7)]}


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def box_of(block, shape):
    nx, ny, nz = shape
    return (1, ny, 1) if block == "yline" else (1, 1, nz)


def inputs(shape, dt):
    nx, ny, nz = shape
    return rounded(initial_guess((nz, ny, nx)), dt), rounded(rhs((nz, ny, nx)), dt)


@pytest.mark.parametrize("block", ["yline", "zline"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_jacobi_parity_per_sweep(brs, orc, block, shape, dt):
    nx, ny, nz = shape
    for a in COEFFS[block]:
        u, b = inputs(shape, dt)
        with brs.Context(nx, ny, nz, a, block=block, method="jacobi", dtype=dt) as ctx:
            ut, bt = to_dev(u, dt), to_dev(b, dt)
            prev = u
            for k in range(3):
                ctx.sweep(ut, bt, 1)
                got = to_np(ut)
                ref = orc.sweep(prev, b, a, block="box", box=box_of(block, shape),
                                method="jacobi", omega=0.8)
                assert rel_max_err(got, ref) <= TOL[dt], (a, k)
                prev = got
            assert ctx.last_error() == 0


@pytest.mark.parametrize("block", ["yline", "zline"])
@pytest.mark.parametrize("nsweeps", [1, 2, 5])
def test_several_sweeps_in_one_call(brs, orc, block, nsweeps):
    shape = (13, 7, 11)
    nx, ny, nz = shape
    a = COEFFS[block][1]
    u, b = inputs(shape, "f64")
    ref = u
    for _ in range(nsweeps):
        ref = orc.sweep(ref, b, a, block="box", box=box_of(block, shape), method="jacobi",
                        omega=0.8)
    with brs.Context(nx, ny, nz, a, block=block, method="jacobi", dtype="f64") as ctx:
        ut, bt = to_dev(u, "f64"), to_dev(b, "f64")
        ctx.sweep(ut, bt, nsweeps)
        got = to_np(ut)
        # b is read only and the residual sees the original layout
        assert np.array_equal(to_np(bt), b)
        r = ctx.residual(ut, bt)
    assert rel_max_err(got, ref) <= TOL["f64"]
    assert abs(r - orc.residual_norm(got, b, a)) <= 1e-12 * orc.residual_norm(got, b, a)


@pytest.mark.parametrize("block,a", [("yline", (0.01, 1.0, 0.01)), ("zline", (0.01, 0.01, 1.0))])
def test_gs_converges_to_exact(brs, orc, block, a):
    n = (12, 10, 14)
    nx, ny, nz = n
    b = rhs((nz, ny, nx))
    ref = orc.exact_solve(b, a)
    with brs.Context(nx, ny, nz, a, block=block, method="gs", dtype="f64") as ctx:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        ctx.sweep(ut, bt, 300)
        got = to_np(ut)
    assert rel_max_err(got, ref) <= 1e-10


@pytest.mark.parametrize("block", ["yline", "zline"])
def test_full_size_one_sweep(brs, orc, block):
    """256^3 FP32 Jacobi, the benchmark's launch, against the oracle's x-line sweep of the
    permuted grid (equal to the 1 x 256 x 1 / 1 x 1 x 256 box sweep, pinned in the oracle)."""
    shape = (256, 256, 256)
    a = COEFFS[block][0]
    u, b = inputs(shape, "f32")
    if block == "yline":
        fwd, back, ap = (0, 2, 1), (0, 2, 1), (a[1], a[0], a[2])
    else:
        fwd, back, ap = (1, 2, 0), (2, 0, 1), (a[2], a[0], a[1])
    ref = orc.sweep(np.ascontiguousarray(u.transpose(fwd)), np.ascontiguousarray(b.transpose(fwd)),
                    ap, block="line", method="jacobi", omega=0.8).transpose(back)
    with brs.Context(256, 256, 256, a, block=block, method="jacobi", dtype="f32") as ctx:
        ut, bt = to_dev(u, "f32"), to_dev(b, "f32")
        ctx.sweep(ut, bt, 1)
        got = to_np(ut)
    assert rel_max_err(got, ref) <= TOL["f32"]


def test_unsupported_line_length(brs):
    with pytest.raises(brs.BrsError) as e:
        brs.Context(8, 1024, 8, block="yline", dtype="f32")  # y-lines of 1024 > 512
    assert e.value.code == brs.BRS_ERR_UNSUPPORTED
