"""Failure detection without a GPU fault.

* A device-side wait that nothing satisfies gives up after its bound, records
  BRS_ERR_TIMEOUT in the sticky status, and the context stays usable after the status is read.
* An allocation the device cannot satisfy is reported as BRS_ERR_NOMEM (no abort).
* Invalid arguments never reach the device.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs
from gpu_common import rel_max_err, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def test_bounded_wait_sets_sticky_timeout_and_context_recovers(brs, orc):
    import torch

    shape = (6, 10, 24)
    u0, b = initial_guess(shape), rhs(shape)
    with brs.Context(24, 10, 6, (1, 1, 1)) as ctx:
        stream = torch.cuda.current_stream().cuda_stream
        assert brs.brsmooth_selftest_wait(ctx.h, 1_000_000, stream) == brs.BRS_OK  # 1 ms
        torch.cuda.synchronize()
        ut, bt = to_dev(u0, "f64"), to_dev(b, "f64")
        # the next call reports the sticky status instead of launching
        assert brs.brsmooth_sweep(ctx.h, ut.data_ptr(), bt.data_ptr(), 1, stream) == brs.BRS_ERR_TIMEOUT
        assert ctx.last_error() == brs.BRS_ERR_TIMEOUT
        assert ctx.last_error() == brs.BRS_OK  # read clears it
        ctx.sweep(ut, bt, 1)
        ref = orc.sweep(u0, b, (1, 1, 1), block="line", method="jacobi", omega=0.8)
        assert rel_max_err(to_np(ut), ref) <= 1e-12
    with brs.Context(8, 8, 8) as ctx:
        assert brs.brsmooth_selftest_wait(ctx.h, -1, 0) == brs.BRS_ERR_ARG
        assert brs.brsmooth_selftest_wait(ctx.h, 2_000_000_000, 0) == brs.BRS_ERR_ARG
        assert brs.brsmooth_selftest_wait(None, 1000, 0) == brs.BRS_ERR_ARG


def test_unsatisfiable_allocation_is_reported(brs):
    # 1024 x 1024 x 80000 FP64 cells = 671 GB per grid buffer: more than the device holds
    p = brs.brs_params(1024, 1024, 80000, 1.0, 1.0, 1.0, brs.BRS_XYPLANE, brs.BRS_JACOBI,
                       brs.BRS_F64, 0.0, 0)
    rc, h = brs.brsmooth_create(p)
    assert rc == brs.BRS_ERR_NOMEM and not h.value
    assert "memory" in brs.brsmooth_cuda_error_string().lower()
    # the device is still usable afterwards
    with brs.Context(16, 8, 4) as ctx:
        import torch

        u = torch.zeros(16 * 8 * 4, dtype=torch.float64, device="cuda")
        b = torch.ones_like(u)
        ctx.sweep(u, b, 2)
        assert torch.isfinite(u).all()
