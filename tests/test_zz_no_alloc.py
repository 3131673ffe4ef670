"""The allocation-free x-line block-Jacobi entry point.

Callers whose device memory belongs to another allocator, or whose loops cannot afford
cudaMalloc's synchronisation, use brsmooth_line_jacobi_noalloc: it keeps its second
vector and factor tables in fixed library-owned device arrays and builds the tables on
the device.  Calls in a row (different shapes, dtypes and lane layouts, so the shared
arrays are reused with other contents) must match brsmooth_sweep on a BRS_XLINE /
BRS_JACOBI context and the FP64 oracle within the per-sweep tolerance.
This file is collected last so that a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np

pytestmark = pytest.mark.gpu

# (nx, ny, nz), coefficients, dtype, sweeps: lane layouts E = 4 (G = 8, 16), E = 8 and E = 16
CASES = [((24, 20, 12), (1.0, 1.0, 1.0), "f64", 3),
         ((64, 17, 9), (1.0, 0.1, 0.01), "f32", 2),
         ((200, 7, 5), (1.0, 1.0, 0.01), "f64", 2),
         ((500, 6, 4), (1.0, 0.5, 0.25), "f32", 3)]


def test_noalloc_matches_context_sweep_and_oracle_calls_in_a_row(orc):
    import torch

    import paper_1208_1975_gb300 as brs

    brs.build()
    stream = torch.cuda.current_stream().cuda_stream
    for (nx, ny, nz), a, dt, ns in CASES:
        shape = (nz, ny, nx)
        u0 = rounded(initial_guess(shape), dt)
        b = rounded(rhs(shape), dt)
        with brs.Context(nx, ny, nz, a, block="line", method="jacobi", dtype=dt) as ctx:
            ur, br = to_dev(u0, dt), to_dev(b, dt)
            ctx.sweep(ur, br, ns)
            ref_ctx = to_np(ur)
        ref = u0
        for _ in range(ns):
            ref = orc.sweep(ref, b, a, block="line", method="jacobi", omega=0.8)
        un, bn = to_dev(u0, dt), to_dev(b, dt)
        rc = brs.brsmooth_line_jacobi_noalloc(nx, ny, nz, a, 0.0, brs.DTYPES[dt], un.data_ptr(),
                                              bn.data_ptr(), ns, stream)
        assert rc == brs.BRS_OK, brs.brsmooth_strerror(rc)
        torch.cuda.synchronize()
        got = to_np(un)
        assert rel_max_err(got, ref_ctx) <= TOL[dt], (nx, ny, nz, dt)
        assert rel_max_err(got, ref) <= TOL[dt], (nx, ny, nz, dt)


def test_noalloc_rejections():
    import torch

    import paper_1208_1975_gb300 as brs

    brs.build()
    # large enough for every shape below, so that no call could reach past them
    u = torch.zeros(128 * 128 * 65, dtype=torch.float64, device="cuda")
    b = torch.zeros(128 * 128 * 65, dtype=torch.float64, device="cuda")
    up, bp = u.data_ptr(), b.data_ptr()
    call = lambda nx, ny, nz, a=(1, 1, 1), om=0.0: brs.brsmooth_line_jacobi_noalloc(
        nx, ny, nz, a, om, brs.BRS_F64, up, bp, 1, 0)
    # the fixed arrays: lines beyond the 512-cell lane layouts, and grids beyond the cell
    # maximum with a line length the layouts cover
    assert call(513, 1, 1) == brs.BRS_ERR_UNSUPPORTED
    assert 128 * 128 * 65 > (1 << 20)  # BRSMOOTH_NOALLOC_MAX_CELLS in the header
    assert call(128, 128, 65) == brs.BRS_ERR_UNSUPPORTED
    # argument errors, before any device work
    for om in (float("-inf"), float("inf"), float("nan"), 2.0):
        assert call(8, 8, 8, om=om) == brs.BRS_ERR_ARG, om
    for a in ((0.0, 1, 1), (1, -1.0, 1), (1, 1, float("inf")), (float("nan"), 1, 1)):
        assert call(8, 8, 8, a=a) == brs.BRS_ERR_ARG, a
    assert brs.brsmooth_line_jacobi_noalloc(8, 8, 8, (1, 1, 1), 0.0, brs.BRS_F64, up, up, 1,
                                            0) == brs.BRS_ERR_ARG  # u aliases b
    torch.cuda.synchronize()
    assert torch.count_nonzero(u) == 0  # rejected calls touched nothing


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_calls_captured_in_a_cuda_graph(orc, dt):
    """Two calls (2 and 3 sweeps) captured into one CUDA graph on a side stream: nothing
    is copied from the host, so the graph replays on its own.  Every replay from the same
    start equals the same two calls run directly, bit for bit, and the result matches 5
    sweeps of the context path and of the oracle."""
    import torch

    import paper_1208_1975_gb300 as brs

    brs.build()
    nx, ny, nz, a = 64, 12, 10, (1.0, 0.3, 0.1)
    shape = (nz, ny, nx)
    u0 = rounded(initial_guess(shape), dt)
    b = rounded(rhs(shape), dt)
    call = lambda u, bb, ns, s: brs.brsmooth_line_jacobi_noalloc(
        nx, ny, nz, a, 0.0, brs.DTYPES[dt], u.data_ptr(), bb.data_ptr(), ns, s)
    # direct calls (also the first call on the device, which must precede any capture)
    ud, bd = to_dev(u0, dt), to_dev(b, dt)
    cur = torch.cuda.current_stream().cuda_stream
    assert call(ud, bd, 2, cur) == brs.BRS_OK
    assert call(ud, bd, 3, cur) == brs.BRS_OK
    torch.cuda.synchronize()
    direct = to_np(ud)
    # the same two calls captured
    ug, bg = to_dev(u0, dt), to_dev(b, dt)
    start = ug.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        rc1 = call(ug, bg, 2, side.cuda_stream)
        rc2 = call(ug, bg, 3, side.cuda_stream)
    assert rc1 == brs.BRS_OK and rc2 == brs.BRS_OK
    for _ in range(2):
        ug.copy_(start)
        graph.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_np(ug), direct)
    with brs.Context(nx, ny, nz, a, block="line", method="jacobi", dtype=dt) as ctx:
        ur, br = to_dev(u0, dt), to_dev(b, dt)
        ctx.sweep(ur, br, 5)
        ref_ctx = to_np(ur)
    ref = u0
    for _ in range(5):
        ref = orc.sweep(ref, b, a, block="line", method="jacobi", omega=0.8)
    assert rel_max_err(direct, ref_ctx) <= TOL[dt]
    assert rel_max_err(direct, ref) <= TOL[dt]
