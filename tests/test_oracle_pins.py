"""Pins of the FP64 oracle against what mathematics fixes independently of its code.

* Thomas and the block solves against dense LU (numpy.linalg.solve) on tiny grids.
* The assembled operator against its Kronecker-sum form, its symmetry, weak diagonal
  dominance (strict on boundary rows) and its closed-form sine spectrum (Sec. 1.1 operator).
* Block Jacobi: exact one-sweep damping of a single sine mode (A and the block diagonal
  share the sine eigenvectors), and the fixed point A^{-1} b.
* Block Gauss-Seidel (Eq. sm:blockm) against the dense block-triangular splitting.
* The DST exact solver against a dense solve.
* The adjoint against central finite differences (exact for a loss quadratic in u0, b).
"""
import numpy as np
import pytest

from brs_inputs import sine_mode, uniform_field

RNG = np.random.default_rng(12345)
GRIDS = [(1, 1, 1), (5, 1, 1), (1, 4, 3), (4, 3, 2), (3, 5, 4), (6, 4, 5)]
COEFFS = [(1.0, 1.0, 1.0), (1.0, 1.0, 0.01), (1.0, 0.1, 0.01), (0.3, 2.0, 0.7)]


def tri(n):
    """tridiag(-1, 2, -1) of size n (textbook 1D Dirichlet Laplacian)."""
    return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def kron_A(nx, ny, nz, a):
    """A = az Tz (x) I (x) I + ay I (x) Ty (x) I + ax I (x) I (x) Tx for x-fastest ordering."""
    ax, ay, az = a
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    return (az * np.kron(np.kron(tri(nz), Iy), Ix) + ay * np.kron(np.kron(Iz, tri(ny)), Ix)
            + ax * np.kron(np.kron(Iz, Iy), tri(nx)))


def dense_block_diag(A, labels):
    return np.where(labels[:, None] == labels[None, :], A, 0.0)


@pytest.mark.parametrize("n", range(1, 9))
def test_thomas_vs_dense(orc, n):
    for _ in range(3):
        off = -RNG.uniform(0.1, 2.0)
        diag = 2 * abs(off) + RNG.uniform(0.01, 3.0)
        rhs = RNG.uniform(-1, 1, n)
        M = diag * np.eye(n) + off * (np.eye(n, k=1) + np.eye(n, k=-1))
        np.testing.assert_allclose(orc.thomas(off, diag, rhs), np.linalg.solve(M, rhs),
                                   rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dims", GRIDS)
@pytest.mark.parametrize("a", COEFFS)
def test_operator_is_kronecker_sum(orc, dims, a):
    nx, ny, nz = dims
    A = orc.assemble_A(nx, ny, nz, a)
    np.testing.assert_allclose(A, kron_A(nx, ny, nz, a), rtol=0, atol=1e-15)


@pytest.mark.parametrize("dims", [(4, 3, 2), (3, 5, 4), (6, 4, 5)])
@pytest.mark.parametrize("a", COEFFS)
def test_operator_symmetry_dominance_spectrum(orc, dims, a):
    nx, ny, nz = dims
    A = orc.assemble_A(nx, ny, nz, a)
    assert np.array_equal(A, A.T)
    diag = np.diag(A)
    assert np.allclose(diag, 2 * sum(a))
    off = np.abs(A).sum(axis=1) - np.abs(diag)
    slack = diag - off
    assert np.all(slack >= -1e-14)
    # equality exactly on rows without a Dirichlet neighbour, strict on boundary rows
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    boundary = ((i == 0) | (i == nx - 1) | (j == 0) | (j == ny - 1) | (k == 0) | (k == nz - 1)).ravel()
    assert np.all(slack[boundary] > 1e-3 * min(a))
    assert np.allclose(slack[~boundary], 0.0, atol=1e-13)
    ev = np.sort(np.linalg.eigvalsh(A))
    np.testing.assert_allclose(ev, np.sort(orc.eigenvalues(nx, ny, nz, a).ravel()), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("a", COEFFS)
def test_sine_modes_are_eigenvectors(orc, a):
    nx, ny, nz = 9, 7, 6
    lam = orc.eigenvalues(nx, ny, nz, a)
    for (p, q, r) in [(1, 1, 1), (2, 3, 1), (9, 7, 6), (5, 1, 4)]:
        m = sine_mode(nx, ny, nz, p, q, r)
        np.testing.assert_allclose(orc.apply_A(m, a), lam[r - 1, q - 1, p - 1] * m, atol=1e-13)


@pytest.mark.parametrize("block", ["line", "plane"])
@pytest.mark.parametrize("dims", GRIDS)
@pytest.mark.parametrize("a", COEFFS)
def test_block_solve_vs_dense(orc, block, dims, a):
    nx, ny, nz = dims
    A = kron_A(nx, ny, nz, a)
    M = dense_block_diag(A, orc.block_of(nx, ny, nz, block))
    r = RNG.uniform(-1, 1, (nz, ny, nx))
    ref = np.linalg.solve(M, r.ravel()).reshape(r.shape)
    np.testing.assert_allclose(orc.block_minv(r, a, block), ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("block", ["line", "plane"])
@pytest.mark.parametrize("omega", [0.8, 1.0, 0.55])
def test_jacobi_dense_splitting(orc, block, omega):
    nx, ny, nz = 5, 4, 3
    a = (0.9, 1.7, 0.4)
    A = kron_A(nx, ny, nz, a)
    M = dense_block_diag(A, orc.block_of(nx, ny, nz, block))
    u = RNG.uniform(-1, 1, (nz, ny, nx))
    b = RNG.uniform(-1, 1, (nz, ny, nx))
    ref = u.ravel() + omega * np.linalg.solve(M, b.ravel() - A @ u.ravel())
    got = orc.sweep(u, b, a, block=block, method="jacobi", omega=omega)
    np.testing.assert_allclose(got.ravel(), ref, rtol=1e-12, atol=1e-13)


def _visit_rank(nx, ny, nz, block, method):
    """Position of each block in the Gauss-Seidel visiting order."""
    nb = ny * nz if block == "line" else nz
    ids = np.arange(nb)
    if method == "gs_lex":
        seq = ids
    elif method == "gs_reverse":
        seq = ids[::-1]
    else:
        if block == "line":
            parity = (ids % ny + ids // ny) % 2
        else:
            parity = ids % 2
        seq = np.concatenate([ids[parity == 0], ids[parity == 1]])
    rank = np.empty(nb, dtype=int)
    rank[seq] = np.arange(nb)
    return rank


@pytest.mark.parametrize("block", ["line", "plane"])
@pytest.mark.parametrize("method", ["gs_lex", "gs_reverse", "gs_zebra"])
@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_gauss_seidel_dense_splitting(orc, block, method, omega):
    """One block GS/SOR sweep = u + (D/omega + L)^{-1}(b - A u), L = earlier-visited blocks."""
    nx, ny, nz = 4, 3, 5
    a = (1.3, 0.6, 0.9)
    A = kron_A(nx, ny, nz, a)
    lab = orc.block_of(nx, ny, nz, block)
    rank = _visit_rank(nx, ny, nz, block, method)[lab]
    D = np.where(rank[:, None] == rank[None, :], A, 0.0)
    L = np.where(rank[:, None] > rank[None, :], A, 0.0)
    u = RNG.uniform(-1, 1, (nz, ny, nx))
    b = RNG.uniform(-1, 1, (nz, ny, nx))
    ref = u.ravel() + np.linalg.solve(D / omega + L, b.ravel() - A @ u.ravel())
    got = orc.sweep(u, b, a, block=block, method=method, omega=omega)
    np.testing.assert_allclose(got.ravel(), ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("block", ["line", "plane"])
@pytest.mark.parametrize("a", COEFFS)
@pytest.mark.parametrize("omega", [0.8, 1.0])
def test_single_mode_damping_closed_form(orc, block, a, omega):
    """With b = 0 a sine mode is multiplied by exactly g = 1 - omega lambda/mu per Jacobi sweep."""
    nx, ny, nz = 12, 10, 7
    g = orc.mode_factor(nx, ny, nz, a, block, omega)
    b = np.zeros((nz, ny, nx))
    for (p, q, r) in [(1, 1, 1), (12, 10, 7), (3, 8, 2), (7, 1, 6)]:
        m = sine_mode(nx, ny, nz, p, q, r)
        got = orc.sweep(m, b, a, block=block, method="jacobi", omega=omega)
        np.testing.assert_allclose(got, g[r - 1, q - 1, p - 1] * m, atol=1e-13)


def test_mode_damping_at_32_cubed(orc):
    """The 32^3 isotropic grid: the slowest mode after 3 line-Jacobi sweeps equals g^3 exactly."""
    n = 32
    a = (1.0, 1.0, 1.0)
    g = orc.mode_factor(n, n, n, a, "line", 0.8)[0, 0, 0]
    m = sine_mode(n, n, n, 1, 1, 1)
    u = m
    for _ in range(3):
        u = orc.sweep(u, np.zeros_like(u), a, block="line", method="jacobi", omega=0.8)
    np.testing.assert_allclose(u, g ** 3 * m, atol=1e-12)


@pytest.mark.parametrize("dims", [(4, 3, 2), (3, 5, 4), (6, 4, 5), (1, 1, 7)])
@pytest.mark.parametrize("a", COEFFS)
def test_exact_solve_vs_dense(orc, dims, a):
    nx, ny, nz = dims
    b = RNG.uniform(-1, 1, (nz, ny, nx))
    ref = np.linalg.solve(kron_A(nx, ny, nz, a), b.ravel()).reshape(b.shape)
    np.testing.assert_allclose(orc.exact_solve(b, a), ref, rtol=1e-11, atol=1e-12)


def test_exact_solve_residual_large(orc):
    n = 32
    a = (1.0, 1.0, 0.01)
    b = uniform_field((n, n, n), 1) / (n + 1) ** 2
    u = orc.exact_solve(b, a)
    assert orc.residual_norm(u, b, a) <= 1e-13 * np.linalg.norm(b) * 1e3


@pytest.mark.parametrize("block", ["line", "plane"])
@pytest.mark.parametrize("method", ["jacobi", "gs_lex", "gs_zebra"])
def test_fixed_point_is_dense_solution(orc, block, method):
    nx, ny, nz = 6, 5, 4
    a = (1.0, 0.5, 0.25)
    b = RNG.uniform(-1, 1, (nz, ny, nx))
    ref = np.linalg.solve(kron_A(nx, ny, nz, a), b.ravel()).reshape(b.shape)
    u = np.zeros_like(b)
    omega = 0.8 if method == "jacobi" else 1.0
    for _ in range(400):
        u = orc.sweep(u, b, a, block=block, method=method, omega=omega)
    np.testing.assert_allclose(u, ref, rtol=1e-10, atol=1e-11)


def test_residual_norm_definition(orc):
    nx, ny, nz = 5, 4, 3
    a = (1.0, 2.0, 3.0)
    u = RNG.uniform(-1, 1, (nz, ny, nx))
    b = RNG.uniform(-1, 1, (nz, ny, nx))
    r = b.ravel() - kron_A(nx, ny, nz, a) @ u.ravel()
    np.testing.assert_allclose(orc.residual(u, b, a).ravel(), r, atol=1e-14)
    assert abs(orc.residual_norm(u, b, a) - np.linalg.norm(r)) < 1e-13


@pytest.mark.parametrize("block", ["line", "plane"])
def test_adjoint_vs_finite_differences(orc, block):
    nx, ny, nz = 5, 4, 3
    a = (1.0, 0.7, 0.3)
    K = 4
    u0 = RNG.uniform(-1, 1, (nz, ny, nx))
    b = RNG.uniform(-1, 1, (nz, ny, nx))
    ut = RNG.uniform(-1, 1, (nz, ny, nx))
    loss, gu0, gb, ga = orc.adjoint_gradients(u0, b, a, K, ut, block=block)
    assert abs(loss - orc.sweeps_loss(u0, b, a, K, ut, block=block)) < 1e-12
    d = RNG.uniform(-1, 1, (nz, ny, nx))
    eps = 1e-3  # the loss is quadratic in u0 and b: central differences are exact up to rounding
    fd_u = (orc.sweeps_loss(u0 + eps * d, b, a, K, ut, block=block)
            - orc.sweeps_loss(u0 - eps * d, b, a, K, ut, block=block)) / (2 * eps)
    fd_b = (orc.sweeps_loss(u0, b + eps * d, a, K, ut, block=block)
            - orc.sweeps_loss(u0, b - eps * d, a, K, ut, block=block)) / (2 * eps)
    assert abs(fd_u - np.sum(gu0 * d)) < 1e-9 * max(1.0, abs(fd_u))
    assert abs(fd_b - np.sum(gb * d)) < 1e-9 * max(1.0, abs(fd_b))
    for dd in range(3):
        h = 1e-5 * a[dd]
        ap, am = list(a), list(a)
        ap[dd] += h
        am[dd] -= h
        fd = (orc.sweeps_loss(u0, b, ap, K, ut, block=block)
              - orc.sweeps_loss(u0, b, am, K, ut, block=block)) / (2 * h)
        assert abs(fd - ga[dd]) < 1e-6 * max(1.0, abs(fd)), (dd, fd, ga[dd])
