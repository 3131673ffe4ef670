"""Mixed-precision defect correction: FP64 outer residual and correction, FP32 inner sweeps.

Acceptance is the FP64 residual the oracle recomputes on the CPU from the returned iterate
(<= rtol * ||b||), and the distance to the oracle's exact DST solution.
"""
import numpy as np
import pytest

from brs_inputs import rhs
from gpu_common import rel_max_err, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


@pytest.mark.parametrize("block,method,n,a,m", [
    ("plane", "jacobi", 32, (1.0, 0.1, 0.01), 16),
    ("plane", "gs", 48, (1.0, 0.1, 0.01), 32),
    ("line", "gs", 32, (1.0, 1.0, 1.0), 64),
    ("line", "jacobi", 24, (1.0, 1.0, 0.01), 64),
])
def test_defect_correction_reaches_fp64_residual(brs, orc, block, method, n, a, m):
    b = rhs((n, n, n))
    rtol = 1e-10
    with brs.Context(n, n, n, a, block=block, method=method, dtype="f64") as outer, \
            brs.Context(n, n, n, a, block=block, method=method, dtype="f32") as inner:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        done, rel, hist = brs.defect_correction(outer, inner, ut, bt, rtol=rtol, inner_sweeps=m,
                                                max_outer=2000)
        u = to_np(ut)
    assert rel <= rtol and done >= 1
    assert hist[0] == pytest.approx(1.0)
    assert all(h2 < h1 for h1, h2 in zip(hist, hist[1:]))
    # independent check of the claimed residual, and of the solution itself
    assert orc.residual_norm(u, b, a) <= 1.05 * rtol * np.linalg.norm(b)
    assert rel_max_err(u, orc.exact_solve(b, a)) <= 1e-7


@pytest.mark.parametrize("method", ["jacobi", "gs"])
def test_defect_correction_512_wide_planes(brs, orc, method):
    """The 512 x 512 plane solve of the 512^3 workload (a = (1, 0.1, 0.01)) inside the
    defect-correction loop, on a 512 x 512 x 6 slab: FP64 residual 1e-10, recomputed by the
    oracle, and the distance to the exact DST solution."""
    nx = ny = 512
    nz = 6
    a = (1.0, 0.1, 0.01)
    b = rhs((nz, ny, nx))
    with brs.Context(nx, ny, nz, a, block="plane", method="jacobi", dtype="f64") as outer, \
            brs.Context(nx, ny, nz, a, block="plane", method=method, dtype="f32") as inner:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        done, rel, _ = brs.defect_correction(outer, inner, ut, bt, rtol=1e-10, inner_sweeps=32,
                                             max_outer=4000)
        u = to_np(ut)
    assert rel <= 1e-10 and done >= 1
    assert orc.residual_norm(u, b, a) <= 1.05e-10 * np.linalg.norm(b)
    assert rel_max_err(u, orc.exact_solve(b, a)) <= 1e-7


def test_defect_correction_argument_errors(brs):
    import torch

    with brs.Context(8, 8, 8, dtype="f64") as o64, brs.Context(8, 8, 8, dtype="f32") as i32, \
            brs.Context(8, 8, 4, dtype="f32") as bad:
        u = torch.zeros(512, dtype=torch.float64, device="cuda")
        b = torch.ones(512, dtype=torch.float64, device="cuda")
        up, bp = u.data_ptr(), b.data_ptr()
        assert brs.brsmooth_defect_correction(i32.h, o64.h, up, bp, 1e-8, 4, 5, 0)[0] == brs.BRS_ERR_ARG
        assert brs.brsmooth_defect_correction(o64.h, bad.h, up, bp, 1e-8, 4, 5, 0)[0] == brs.BRS_ERR_ARG
        assert brs.brsmooth_defect_correction(o64.h, i32.h, up, bp, 1e-8, 0, 5, 0)[0] == brs.BRS_ERR_ARG
        rc, done, rel, _ = brs.brsmooth_defect_correction(o64.h, i32.h, up, bp, 1e-8, 8, 0, 0)
        assert rc == brs.BRS_OK and done == 0 and rel == pytest.approx(1.0)
