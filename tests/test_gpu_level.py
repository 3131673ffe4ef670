"""A level of patches on the GPU (x-line sweeps inside patches, ghost exchange between face
neighbours after every step, Sec. 2) against the oracle's level sweep.

Jacobi inside patches is deterministic: element-wise parity sweep by sweep, on a regular
tiling, on patches of different y extents sharing y faces, with a periodic direction, and
on the paper's 96 x 64^3 level.  Chaotic GS inside patches: convergence of a tiled level to
the global A^{-1} b.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs, uniform_field
from gpu_common import TOL, rel_max_err, rounded, to_dev, to_np
from test_oracle_level import pack, tiling, unpack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def layouts():
    out = {}
    d, n = tiling((2, 2, 2), (16, 12, 8))
    out["tiled2x2x2"] = (d, n)
    d, n = tiling((3, 1, 2), (24, 20, 6))
    out["tiled3x1x2"] = (d, n)
    # two columns of patches with different ny stacked along y (x and z extents agree)
    out["uneven_y"] = (np.array([[32, 8, 6], [32, 14, 6], [32, 5, 6]]),
                       np.array([[-1, -1, -1, 1, -1, -1], [-1, -1, 0, 2, -1, -1],
                                 [-1, -1, 1, -1, -1, -1]]))
    # periodic in x (a patch is its own x neighbour) next to a plain patch along z
    out["periodic_x"] = (np.array([[16, 10, 7], [16, 10, 9]]),
                         np.array([[0, 0, -1, -1, -1, 1], [-1, -1, -1, -1, 0, -1]]))
    return out


LAYOUTS = layouts()


def run_level(brs, dims, nbr, u, b, a, dt, nsweeps, method="jacobi"):
    with brs.BatchedContext(dims, a, method=method, dtype=dt, nbr=nbr) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        out = []
        for _ in range(nsweeps):
            ctx.sweep(ut, bt, 1)
            out.append(to_np(ut))
        assert brs.brsmooth_last_error(ctx.h) == 0
    return out


@pytest.mark.parametrize("name", list(LAYOUTS))
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_level_jacobi_parity(brs, orc, name, dt):
    dims, nbr = LAYOUTS[name]
    n = int(np.prod(dims, axis=1).sum())
    u = rounded(uniform_field((n,), 31), dt)
    b = rounded(uniform_field((n,), 32) * 1e-3, dt)
    a = (1.0, 0.5, 0.25)
    got = run_level(brs, dims, nbr, u, b, a, dt, 3)
    prev = u
    for k in range(3):
        ref = orc.level_sweep(prev, b, dims, nbr, a, method="jacobi", omega=0.8)
        assert rel_max_err(got[k], ref) <= TOL[dt], (name, k)
        prev = got[k]  # per-sweep parity from the device's own iterate


@pytest.mark.parametrize("name", list(LAYOUTS))
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_level_multi_sweep_call_matches_single_calls(brs, name, dt):
    """Within one call, steps after the first take their ghosts from the faces the previous
    step wrote directly into the second ghost buffer; across calls, from the gather of the
    iterate.  Both give the same level Jacobi iterate, bit for bit."""
    dims, nbr = LAYOUTS[name]
    n = int(np.prod(dims, axis=1).sum())
    u = rounded(uniform_field((n,), 33), dt)
    b = rounded(uniform_field((n,), 34) * 1e-3, dt)
    one = run_level(brs, dims, nbr, u, b, (1.0, 0.5, 0.25), dt, 4)[-1]
    with brs.BatchedContext(dims, (1.0, 0.5, 0.25), method="jacobi", dtype=dt, nbr=nbr) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        ctx.sweep(ut, bt, 4)
        four = to_np(ut)
        assert brs.brsmooth_last_error(ctx.h) == 0
    assert np.array_equal(one, four)


@pytest.mark.parametrize("push", ["0", "1"], ids=["gather_every_step", "face_push"])
def test_paper_level_three_steps_per_call(brs, push, monkeypatch):
    """The 96 x 64^3 level, FP32 Jacobi, three steps in one call (the launch sequence the
    benchmark times, with and without the face pushes) equals three single-step calls."""
    monkeypatch.setenv("BRSMOOTH_LEVEL_PUSH", push)
    P, pdim = (4, 4, 6), (64, 64, 64)
    dims, nbr = tiling(P, pdim)
    n = 96 * 64 ** 3
    u = rounded(uniform_field((n,), 37), "f32")
    b = rounded(uniform_field((n,), 38) * (1.0 / 65) ** 2, "f32")
    one = run_level(brs, dims, nbr, u, b, (1, 1, 1), "f32", 3)[-1]
    with brs.BatchedContext(dims, (1, 1, 1), method="jacobi", dtype="f32", nbr=nbr) as ctx:
        ut, bt = to_dev(u, "f32"), to_dev(b, "f32")
        ctx.sweep(ut, bt, 3)
        three = to_np(ut)
        assert brs.brsmooth_last_error(ctx.h) == 0
    assert np.array_equal(one, three)


@pytest.mark.parametrize("name", list(LAYOUTS))
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_level_ghosts_kept_across_calls(brs, orc, name, dt):
    """With the ghosts kept across calls (the iterate untouched in between), the last step
    of a call writes its faces for the next call's first step: 4 calls of 3 steps equal one
    call of 12 steps bit for bit, and the oracle's level Jacobi after 12 steps.  Odd step
    counts per call exercise both ghost buffers at a call's start."""
    dims, nbr = LAYOUTS[name]
    n = int(np.prod(dims, axis=1).sum())
    a = (1.0, 0.5, 0.25)
    u = rounded(uniform_field((n,), 41), dt)
    b = rounded(uniform_field((n,), 42) * 1e-3, dt)
    with brs.BatchedContext(dims, a, method="jacobi", dtype=dt, nbr=nbr) as ctx:
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        ctx.sweep(ut, bt, 12)
        twelve = to_np(ut)
    with brs.BatchedContext(dims, a, method="jacobi", dtype=dt, nbr=nbr) as ctx:
        ctx.keep_ghosts(True)
        ut, bt = to_dev(u, dt), to_dev(b, dt)
        for _ in range(4):
            ctx.sweep(ut, bt, 3)
        kept = to_np(ut)
        assert brs.brsmooth_last_error(ctx.h) == 0
    assert np.array_equal(twelve, kept)
    ref = u.astype(np.float64)
    for _ in range(12):
        ref = orc.level_sweep(ref, b.astype(np.float64), dims, nbr, a, method="jacobi", omega=0.8)
    assert rel_max_err(kept, ref) <= TOL[dt] * 12


def test_level_keep_ghosts_paper_level_and_errors(brs):
    """The 96 x 64^3 level, FP32 Jacobi, three steps per call with the ghosts kept (the
    benchmark's chained form): 3 calls equal one call of 9 steps bit for bit; switching off
    returns to a gather at every call's start; a batched context without faces is refused."""
    P, pdim = (4, 4, 6), (64, 64, 64)
    dims, nbr = tiling(P, pdim)
    n = 96 * 64 ** 3
    u = rounded(uniform_field((n,), 43), "f32")
    b = rounded(uniform_field((n,), 44) * (1.0 / 65) ** 2, "f32")
    with brs.BatchedContext(dims, (1, 1, 1), method="jacobi", dtype="f32", nbr=nbr) as ctx:
        ut, bt = to_dev(u, "f32"), to_dev(b, "f32")
        ctx.sweep(ut, bt, 9)
        nine = to_np(ut)
        ut.copy_(to_dev(u, "f32"))
        ctx.keep_ghosts(True)
        for _ in range(3):
            ctx.sweep(ut, bt, 3)
        assert np.array_equal(to_np(ut), nine)
        # off again: the next call gathers; the iterate changed outside the context meanwhile
        ctx.keep_ghosts(False)
        ut.copy_(to_dev(u, "f32"))
        ctx.sweep(ut, bt, 9)
        assert np.array_equal(to_np(ut), nine)
        assert brs.brsmooth_last_error(ctx.h) == 0
    with brs.BatchedContext([[16, 8, 8]], (1, 1, 1), method="jacobi", dtype="f32") as plain:
        assert brs.brsmooth_level_keep_ghosts(plain.h, True) == brs.BRS_ERR_ARG


def test_level_gs_converges_to_global_solution(brs, orc):
    P, pdim = (2, 2, 2), (12, 10, 8)
    dims, nbr = tiling(P, pdim)
    a = (1.0, 1.0, 1.0)
    bg = rhs((16, 20, 24))
    ref = orc.exact_solve(bg, a)
    b = pack(bg, P, pdim)
    with brs.BatchedContext(dims, a, method="gs", dtype="f64", nbr=nbr) as ctx:
        ut, bt = to_dev(np.zeros_like(b), "f64"), to_dev(b, "f64")
        ctx.sweep(ut, bt, 2500)  # the oracle's lexicographic level GS needs 757 to 1e-11
        got = to_np(ut)
    assert rel_max_err(unpack(got, P, pdim), ref) <= 1e-10


def test_paper_level_96_patches_of_64cubed(brs, orc):
    """The paper's 96 x 64^3 level (a 4 x 4 x 6 array of patches), FP32, one Jacobi step."""
    P, pdim = (4, 4, 6), (64, 64, 64)
    dims, nbr = tiling(P, pdim)
    n = 96 * 64 ** 3
    u = rounded(uniform_field((n,), 35), "f32")
    b = rounded(uniform_field((n,), 36) * (1.0 / 65) ** 2, "f32")
    got = run_level(brs, dims, nbr, u, b, (1, 1, 1), "f32", 1)[0]
    ref = orc.level_sweep(u, b, dims, nbr, (1, 1, 1), method="jacobi", omega=0.8)
    assert rel_max_err(got, ref) <= TOL["f32"]
