"""The block-size study of Sec. 3 on the GPU (FP64, a = (1,1,1), b = 0, random initial
guess): ||r_3|| / ||r_0|| and the sliding-window factor (||r_{i+k}|| / ||r_i||)^(1/k).

* Point, x-line and xy-plane block Jacobi: the factor is the slowest sine mode's closed form.
* The paper's seven box sizes: the GPU's three-sweep ratios equal the oracle's (Jacobi and
  two-colour GS, both deterministic) and fall as the block grows.
* Their asymptotic Jacobi factors fall as well: the sizes are nested (each block is a union
  of blocks of the size before), the splittings are regular splittings of an M-matrix with
  the larger block keeping fewer couplings in N, so Varga's comparison theorem orders the
  spectral radii of M^{-1} N; with omega = 0.8 the slowest mode sets the factor because the
  most negative eigenvalue of the damped iteration is above -0.6.
* Two-colour block GS contracts with the square of the undamped block-Jacobi factor (Young:
  the two-colour block matrix is 2-cyclic and consistently ordered), which the GPU's GS and
  damped-Jacobi factors satisfy for every paper size.
"""
import math

import numpy as np
import pytest

from brs_inputs import initial_guess
from gpu_common import to_dev, to_np

pytestmark = pytest.mark.gpu

PAPER_SIZES = [(2, 2, 2), (4, 2, 2), (4, 4, 2), (4, 4, 4), (8, 4, 4), (8, 8, 4), (8, 8, 8)]
N = 32


@pytest.fixture(scope="module")
def brs():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs


def window_factor(brs, block, box, method, i, k):
    a = (1.0, 1.0, 1.0)
    u0 = initial_guess((N, N, N))
    with brs.Context(N, N, N, a, block=block, box=box, method=method, dtype="f64") as c:
        u, b = to_dev(u0, "f64"), to_dev(np.zeros_like(u0), "f64")
        c.sweep(u, b, i)
        ri = c.residual(u, b)
        c.sweep(u, b, k)
        rk = c.residual(u, b)
        assert c.last_error() == 0
    return (rk / ri) ** (1.0 / k)


@pytest.mark.parametrize("block,box", [("box", (1, 1, 1)), ("line", (0, 0, 0)),
                                       ("plane", (0, 0, 0))], ids=["point", "xline", "xyplane"])
def test_jacobi_factor_closed_form(brs, block, box):
    s1 = 2 - 2 * math.cos(math.pi / (N + 1))
    mu = {"box": 6.0, "line": s1 + 4, "plane": 2 * s1 + 2}[block]
    g = 1 - 0.8 * 3 * s1 / mu
    fac = window_factor(brs, block, box, "jacobi", 4000, 100)
    assert abs(fac - g) <= 1e-6, (fac, g)


@pytest.mark.parametrize("method,omethod", [("jacobi", "jacobi"), ("gs", "gs_zebra")])
def test_three_sweep_ratios_match_oracle_and_fall(brs, orc, method, omethod):
    a = (1.0, 1.0, 1.0)
    u0 = initial_guess((N, N, N))
    b = np.zeros_like(u0)
    r0 = orc.residual_norm(u0, b, a)
    om = 0.8 if method == "jacobi" else 1.0
    ratios = []
    for box in PAPER_SIZES:
        got = None
        with brs.Context(N, N, N, a, block="box", box=box, method=method, dtype="f64") as c:
            ut, bt = to_dev(u0, "f64"), to_dev(b, "f64")
            c.sweep(ut, bt, 3)
            got = to_np(ut)
        ref = u0
        for _ in range(3):
            ref = orc.sweep(ref, b, a, block="box", box=box, method=omethod, omega=om)
        rg, rr = orc.residual_norm(got, b, a) / r0, orc.residual_norm(ref, b, a) / r0
        assert abs(rg - rr) <= 1e-10 * rr, box
        ratios.append(rg)
    assert all(x > y for x, y in zip(ratios, ratios[1:])), ratios


def test_asymptotic_jacobi_factor_falls_with_block_size(brs):
    facs = [window_factor(brs, "box", box, "jacobi", 2000, 100) for box in PAPER_SIZES]
    assert all(0 < f < 1 for f in facs), facs
    assert all(x > y for x, y in zip(facs, facs[1:])), facs


@pytest.mark.parametrize("block,box", [("box", b) for b in PAPER_SIZES]
                         + [("line", (0, 0, 0)), ("plane", (0, 0, 0))],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else v)
def test_two_colour_gs_factor_is_square_of_jacobi(brs, block, box):
    """Also for FP64 x-lines (red-black lines, j+k even then odd) and xy-planes (even, then
    odd planes): both block partitions are 2-cyclic in those colours."""
    gj = window_factor(brs, block, box, "jacobi", 2000, 100)
    gg = window_factor(brs, block, box, "gs", 1000, 100)
    rho = 1 - (1 - gj) / 0.8
    assert abs(gg - rho * rho) <= 2e-5, (gj, gg, rho * rho)
