"""The allocation-free x-line block-Jacobi entry point against the context-based one.

Callers whose device memory belongs to another allocator, or whose loops cannot afford
cudaMalloc's synchronisation, use brsmooth_line_jacobi_noalloc: it keeps its second
vector and factor tables in fixed library-owned device arrays.  Two calls in a row (with
different shapes and dtypes, so the shared arrays are reused with other contents) must
match brsmooth_sweep on a BRS_XLINE / BRS_JACOBI context within the per-sweep tolerance.
This file is collected last so that a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_sweep_two_calls_in_a_row():
    import torch

    import paper_1208_1975_gb300 as brs

    brs.build()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [((24, 20, 12), (1.0, 1.0, 1.0), "f64", 3),
             ((64, 17, 9), (1.0, 0.1, 0.01), "f32", 2)]
    for (nx, ny, nz), a, dt, ns in cases:
        shape = (nz, ny, nx)
        u0 = rounded(initial_guess(shape), dt)
        b = rounded(rhs(shape), dt)
        with brs.Context(nx, ny, nz, a, block="line", method="jacobi", dtype=dt) as ctx:
            ur, br = to_dev(u0, dt), to_dev(b, dt)
            ctx.sweep(ur, br, ns)
            ref = to_np(ur)
        un, bn = to_dev(u0, dt), to_dev(b, dt)
        rc = brs.brsmooth_line_jacobi_noalloc(nx, ny, nz, a, 0.0, brs.DTYPES[dt], un.data_ptr(),
                                              bn.data_ptr(), ns, stream)
        assert rc == brs.BRS_OK, brs.brsmooth_strerror(rc)
        torch.cuda.synchronize()
        assert rel_max_err(to_np(un), ref) <= TOL[dt]


def test_noalloc_rejects_grids_beyond_its_fixed_scratch():
    import torch

    import paper_1208_1975_gb300 as brs

    brs.build()
    u = torch.zeros(16, dtype=torch.float64, device="cuda")
    b = torch.zeros(16, dtype=torch.float64, device="cuda")
    too_many = (1 << 20) + 1
    rc = brs.brsmooth_line_jacobi_noalloc(too_many, 1, 1, (1, 1, 1), 0.0, brs.BRS_F64,
                                          u.data_ptr(), b.data_ptr(), 1, 0)
    assert rc == brs.BRS_ERR_UNSUPPORTED
    rc = brs.brsmooth_line_jacobi_noalloc(128, 128, 65, (1, 1, 1), 0.0, brs.BRS_F64,
                                          u.data_ptr(), b.data_ptr(), 1, 0)
    assert rc == brs.BRS_ERR_UNSUPPORTED
