"""Many-patch x-line sweeps (one persistent launch per sweep, replayed as a CUDA graph).

Each patch is an independent grid: block Jacobi results must equal the oracle patch by
patch (and the single-grid library path bit for bit, since both use the same lane
layout and arithmetic); chaotic GS must satisfy the Perron bound on every patch.
"""
import numpy as np
import pytest

from brs_inputs import PATCH_DIM_CHOICES, batched_fields, batched_patch_dims, sine_mode
from gpu_common import TOL, rel_max_err, to_dev, to_np

pytestmark = pytest.mark.gpu

SMALL_DIMS = [(16, 16, 16), (24, 32, 16), (64, 48, 24), (48, 16, 64), (32, 24, 48),
              (20, 9, 5), (17, 3, 7), (1, 1, 1), (128, 5, 6), (7, 33, 2), (64, 64, 64)]


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def _packed(dims, seed_u, seed_b, dt, h=1.0 / 65):
    u = batched_fields(dims, seed_u)
    b = batched_fields(dims, seed_b, scale_h2=True, h=h)
    if dt == "f32":
        u, b = u.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    return u, b


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_batched_jacobi_matches_oracle_per_patch(brs, orc, dt):
    a = (1.0, 1.0, 1.0)
    u, b = _packed(SMALL_DIMS, 2, 1, dt)
    with brs.BatchedContext(SMALL_DIMS, a, method="jacobi", dtype=dt) as bc:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        bc.sweep(ut, bt, 2)
        got = to_np(ut)
        for q in range(len(SMALL_DIMS)):
            up, bp = bc.patch(u, q), bc.patch(b, q)
            ref = orc.sweep(orc.sweep(up, bp, a, block="line", omega=0.8), bp, a, block="line",
                            omega=0.8)
            assert rel_max_err(bc.patch(got, q), ref) <= 2 * TOL[dt], q


def test_batched_jacobi_equals_single_grid_bitwise(brs):
    dims = [(d, e, f) for d, e, f in zip((16, 24, 32, 48, 64), (64, 48, 32, 24, 16), (8, 16, 24, 8, 4))]
    u, b = _packed(dims, 5, 6, "f32")
    with brs.BatchedContext(dims, (1, 1, 1), method="jacobi", dtype="f32") as bc:
        ut, bt = to_dev(u, "f32"), to_dev(b, "f32")
        bc.sweep(ut, bt, 3)
        got = to_np(ut)
        for q, (nx, ny, nz) in enumerate(dims):
            with brs.Context(nx, ny, nz, (1, 1, 1), method="jacobi", dtype="f32") as ctx:
                us, bs_ = to_dev(bc.patch(u, q), "f32"), to_dev(bc.patch(b, q), "f32")
                ctx.sweep(us, bs_, 3)
                assert np.array_equal(to_np(us), bc.patch(got, q)), q


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_batched_gs_perron_bound_and_graph_replay(brs, orc, dt):
    a = (1.0, 1.0, 1.0)
    dims = SMALL_DIMS
    modes = [sine_mode(nx, ny, nz, 1, 1, 1).ravel() for nx, ny, nz in dims]
    u0 = np.concatenate(modes)
    gs = [orc.mode_factor(nx, ny, nz, a, "line", 1.0)[0, 0, 0] for nx, ny, nz in dims]
    slack = 1e-13 if dt == "f64" else 2e-6
    with brs.BatchedContext(dims, a, method="gs", dtype=dt) as bc:
        ut, bt = to_dev(u0, dt), to_dev(np.zeros_like(u0), dt)
        u0r = to_np(ut)
        done = 0
        for step in (3, 3, 5):  # the same (u, b, 3) call replays the captured graph
            bc.sweep(ut, bt, step)
            done += step
            got = to_np(ut)
            for q in range(len(dims)):
                pq = bc.patch(got, q)
                assert np.all(pq >= -slack * done)
                assert np.all(pq <= gs[q] ** done * bc.patch(u0r, q) + slack * (1 + done)), q
        assert bc.last_error() == 0


def test_batched_gs_converges(brs, orc):
    a = (1.0, 1.0, 1.0)
    dims = [(16, 16, 16), (24, 16, 8), (16, 32, 24)]
    _, b = _packed(dims, 2, 1, "f64")
    with brs.BatchedContext(dims, a, method="gs", dtype="f64") as bc:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        bc.sweep(ut, bt, 3000)
        got = to_np(ut)
        for q in range(len(dims)):
            ref = orc.exact_solve(bc.patch(b, q), a)
            assert rel_max_err(bc.patch(got, q), ref) <= 1e-10


def test_600_patch_workload_sampled(brs, orc):
    """The 600-patch set (dims from {16,24,32,48,64}), FP32, in the tuned launch shape."""
    dims = batched_patch_dims(600)
    assert set(np.unique(dims)) <= set(PATCH_DIM_CHOICES)
    a = (1.0, 1.0, 1.0)
    u, b = _packed(dims, 2, 1, "f32")
    with brs.BatchedContext(dims, a, method="jacobi", dtype="f32") as bc:
        cfg = bc.config()
        assert cfg["work_items"] > 0 and cfg["ctas"] > 0
        ut, bt = to_dev(u, "f32"), to_dev(b, "f32")
        bc.sweep(ut, bt, 1)
        got = to_np(ut)
        rng = np.random.default_rng(11)
        for q in list(rng.choice(600, 25, replace=False)) + [0, 599]:
            ref = orc.sweep(bc.patch(u, q), bc.patch(b, q), a, block="line", omega=0.8)
            assert rel_max_err(bc.patch(got, q), ref) <= TOL["f32"], q


def test_600_patch_gs_perron_bound_20_sweep_graph_calls(brs, orc):
    """The 600-patch set, FP32 chaotic line GS, 20 sweeps per call as the benchmark runs it
    (one persistent launch per sweep, the call replayed as a CUDA graph), two calls: with
    b = 0 and the positive (1,1,1) mode in every patch, 0 <= u_k <= g^k u_0 componentwise
    after 20 and 40 sweeps (g: the undamped x-line Jacobi factor of each patch's mode)."""
    dims = batched_patch_dims(600)
    a = (1.0, 1.0, 1.0)
    u0 = np.concatenate([sine_mode(nx, ny, nz, 1, 1, 1).ravel() for nx, ny, nz in dims])
    g = np.array([orc.mode_factor(nx, ny, nz, a, "line", 1.0)[0, 0, 0] for nx, ny, nz in dims])
    sizes = dims.prod(axis=1)
    with brs.BatchedContext(dims, a, method="gs", dtype="f32") as bc:
        ut, bt = to_dev(u0, "f32"), to_dev(np.zeros_like(u0), "f32")
        u0r = to_np(ut)
        for done in (20, 40):
            bc.sweep(ut, bt, 20)
            got = to_np(ut)
            slack = 2e-6 * (1 + done)
            assert np.all(got >= -slack)
            assert np.all(got <= np.repeat(g ** done, sizes) * u0r + slack)
        assert bc.last_error() == 0


def test_batched_argument_errors(brs):
    p = brs.brs_params(1, 1, 1, 1.0, 1.0, 1.0, brs.BRS_XLINE, brs.BRS_CHAOTIC_GS, brs.BRS_F32, 0.0, 0)
    assert brs.brsmooth_create_batched([(16, 16, 0)], p)[0] == brs.BRS_ERR_ARG
    assert brs.brsmooth_create_batched([(256, 16, 16)], p)[0] == brs.BRS_ERR_UNSUPPORTED
    p.block = brs.BRS_XYPLANE
    assert brs.brsmooth_create_batched([(16, 16, 16)], p)[0] == brs.BRS_ERR_UNSUPPORTED
    assert brs.brsmooth_sweep_batched(None, None, None, 1, 0) == brs.BRS_ERR_ARG
