"""Pins of the oracle's patch-level sweep (Sec. 2: patches smoothed with their ghost layers
fixed, ghost cells updated in a Jacobi fashion after each complete smoothing step).

* A regular tiling of a global grid by px*py*pz patches: one level x-line Jacobi step equals
  block Jacobi with (px, 1, 1) box blocks on the assembled grid -- every neighbour value a
  line segment reads, inside its patch or across a face, is from the previous iterate.  The
  box oracle (dense Cholesky inverse) is pinned on its own.
* A single patch with no neighbours is the plain line sweep (Jacobi and GS).
* A tiled level converges to the global A^{-1} b (the DST-I closed form).
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs, uniform_field


def tiling(P, pdim):
    """dims and neighbour table of a Px x Py x Pz array of equal patches (index x fastest)."""
    Px, Py, Pz = P
    dims, nbr = [], []
    for k in range(Pz):
        for j in range(Py):
            for i in range(Px):
                dims.append(pdim)
                idx = lambda a, b, c: a + Px * (b + Py * c)
                nbr.append([idx(i - 1, j, k) if i > 0 else -1, idx(i + 1, j, k) if i + 1 < Px else -1,
                            idx(i, j - 1, k) if j > 0 else -1, idx(i, j + 1, k) if j + 1 < Py else -1,
                            idx(i, j, k - 1) if k > 0 else -1, idx(i, j, k + 1) if k + 1 < Pz else -1])
    return np.array(dims), np.array(nbr)


def pack(g, P, pdim):
    """Global (NZ, NY, NX) grid -> packed patch arrays (patch order of `tiling`)."""
    px, py, pz = pdim
    out = []
    for k in range(P[2]):
        for j in range(P[1]):
            for i in range(P[0]):
                out.append(g[k * pz:(k + 1) * pz, j * py:(j + 1) * py, i * px:(i + 1) * px].ravel())
    return np.concatenate(out)


def unpack(flat, P, pdim):
    px, py, pz = pdim
    g = np.empty((P[2] * pz, P[1] * py, P[0] * px))
    n = px * py * pz
    q = 0
    for k in range(P[2]):
        for j in range(P[1]):
            for i in range(P[0]):
                g[k * pz:(k + 1) * pz, j * py:(j + 1) * py, i * px:(i + 1) * px] = \
                    flat[q * n:(q + 1) * n].reshape(pz, py, px)
                q += 1
    return g


CASES = [((2, 2, 2), (4, 3, 2)), ((3, 1, 2), (5, 4, 3)), ((1, 2, 3), (6, 2, 2)),
         ((2, 3, 1), (3, 3, 5)), ((1, 1, 1), (7, 5, 4))]


@pytest.mark.parametrize("P,pdim", CASES)
@pytest.mark.parametrize("a", [(1.0, 1.0, 1.0), (1.0, 0.1, 0.01), (0.3, 2.0, 0.7)])
@pytest.mark.parametrize("omega", [0.8, 1.0])
def test_level_jacobi_is_segment_block_jacobi(orc, P, pdim, a, omega):
    NX, NY, NZ = P[0] * pdim[0], P[1] * pdim[1], P[2] * pdim[2]
    ug = uniform_field((NZ, NY, NX), 21)
    bg = uniform_field((NZ, NY, NX), 22)
    dims, nbr = tiling(P, pdim)
    got = orc.level_sweep(pack(ug, P, pdim), pack(bg, P, pdim), dims, nbr, a, omega=omega)
    ref = orc.sweep(ug, bg, a, block="box", box=(pdim[0], 1, 1), method="jacobi", omega=omega)
    assert np.abs(unpack(got, P, pdim) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("method", ["jacobi", "gs_lex"])
def test_single_patch_is_line_sweep(orc, method):
    nx, ny, nz = 9, 6, 5
    u, b = initial_guess((nz, ny, nx)), rhs((nz, ny, nx))
    a = (1.0, 0.5, 0.2)
    om = 0.8 if method == "jacobi" else 1.0
    got = orc.level_sweep(u.ravel(), b.ravel(), [[nx, ny, nz]], [[-1] * 6], a, method=method,
                          omega=om)
    ref = orc.sweep(u, b, a, block="line", method=method, omega=om)
    assert np.abs(got.reshape(nz, ny, nx) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_level_converges_to_global_solution(orc):
    P, pdim = (2, 2, 2), (6, 5, 4)
    NX, NY, NZ = 12, 10, 8
    a = (1.0, 1.0, 1.0)
    bg = rhs((NZ, NY, NX))
    ref = orc.exact_solve(bg, a)
    dims, nbr = tiling(P, pdim)
    b = pack(bg, P, pdim)
    u = np.zeros_like(b)
    for _ in range(600):
        u = orc.level_sweep(u, b, dims, nbr, a, method="gs_lex", omega=1.0)
    assert np.abs(unpack(u, P, pdim) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_level_gs_depends_on_ghosts_only_through_old_values(orc):
    """Jacobi-fashion exchange: a patch's step does not see its neighbours' new values, so
    smoothing the patches in any order gives the same level iterate."""
    P, pdim = (3, 1, 1), (4, 3, 3)
    dims, nbr = tiling(P, pdim)
    u = uniform_field((int(np.prod(pdim)) * 3,), 23)
    b = uniform_field((int(np.prod(pdim)) * 3,), 24)
    a = (1.0, 1.0, 1.0)
    one = orc.level_sweep(u, b, dims, nbr, a, method="gs_lex", omega=1.0)
    # reverse the patch order (relabel) and compare
    perm = [2, 1, 0]
    inv = {p: q for q, p in enumerate(perm)}
    dims_r = dims[perm]
    nbr_r = np.array([[inv[x] if x >= 0 else -1 for x in nbr[p]] for p in perm])
    n = int(np.prod(pdim))
    u_r = np.concatenate([u[p * n:(p + 1) * n] for p in perm])
    b_r = np.concatenate([b[p * n:(p + 1) * n] for p in perm])
    two = orc.level_sweep(u_r, b_r, dims_r, nbr_r, a, method="gs_lex", omega=1.0)
    back = np.concatenate([two[inv[p] * n:(inv[p] + 1) * n] for p in range(3)])
    assert np.array_equal(one, back)
