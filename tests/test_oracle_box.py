"""Pins of the oracle's box-block routines (the spatial blocks of Sec. 2, sizes of Sec. 3,
inverse computed once as in Sec. 4.3) against what mathematics fixes independently.

* The block inverse against numpy's dense inverse of the Kronecker-sum block matrix.
* Block Jacobi and block Gauss-Seidel (three visiting orders, omega 1 and 0.8) against the
  dense block splitting of the Kronecker-sum operator, on grids small enough to assemble.
* A grid that is one block: one sweep with omega = 1 is the exact solve (DST-I closed form).
* 1x1x1 blocks: point Jacobi, whose damping of a sine mode has a closed form.
* nx x 1 x 1 and nx x ny x 1 boxes equal the x-line and xy-plane blocks, which the oracle
  solves by other algorithms (Thomas, banded Cholesky); 1 x ny x 1 and 1 x 1 x nz boxes (y-
  and z-lines, the blocks for other anisotropies) equal x-line sweeps of the grid with its
  axes permuted and the coefficients permuted with them.
* Convergence to A^{-1} b, and the Sec. 3 observation that a larger block lowers
  ||r_3|| / ||r_0|| from a random initial guess, over the paper's seven block sizes.
"""
import numpy as np
import pytest

from brs_inputs import initial_guess, rhs, sine_mode, uniform_field

COEFFS = [(1.0, 1.0, 1.0), (1.0, 1.0, 0.01), (0.3, 2.0, 0.7)]
PAPER_SIZES = [(2, 2, 2), (4, 2, 2), (4, 4, 2), (4, 4, 4), (8, 4, 4), (8, 8, 4), (8, 8, 8)]


def tri(n):
    """tridiag(-1, 2, -1) of size n."""
    return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def kron_A(nx, ny, nz, a):
    """A = az Tz (x) I (x) I + ay I (x) Ty (x) I + ax I (x) I (x) Tx, x-fastest ordering."""
    ax, ay, az = a
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    return (az * np.kron(np.kron(tri(nz), Iy), Ix) + ay * np.kron(np.kron(Iz, tri(ny)), Ix)
            + ax * np.kron(np.kron(Iz, Iy), tri(nx)))


def box_labels(nx, ny, nz, box):
    bx, by, bz = box
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    bi, bj, bk = i // bx, j // by, k // bz
    return (bi + (nx // bx) * (bj + (ny // by) * bk)).ravel(), (bi + bj + bk).ravel()


def visit_position(nx, ny, nz, box, order):
    """Position of each block in the visiting order (lex, reverse, two colours)."""
    bx, by, bz = box
    nb = (nx // bx) * (ny // by) * (nz // bz)
    q = np.arange(nb)
    nbx, nby = nx // bx, ny // by
    parity = (q % nbx + (q // nbx) % nby + q // (nbx * nby)) % 2
    if order == "gs_lex":
        seq = q
    elif order == "gs_reverse":
        seq = q[::-1]
    else:
        seq = np.concatenate([q[parity == 0], q[parity == 1]])
    pos = np.empty(nb, dtype=int)
    pos[seq] = np.arange(nb)
    return pos


BOX_SHAPES = [(1, 1, 1), (2, 2, 2), (4, 2, 2), (3, 2, 1), (2, 3, 4), (4, 4, 4)]


@pytest.mark.parametrize("box", BOX_SHAPES)
@pytest.mark.parametrize("a", COEFFS)
def test_box_inverse_vs_dense(orc, box, a):
    inv = orc.box_inverse(box, a)
    ref = np.linalg.inv(kron_A(*box, a))
    assert np.allclose(inv, inv.T, rtol=0, atol=1e-14 * np.abs(ref).max())
    assert np.abs(inv - ref).max() <= 1e-12 * np.abs(ref).max()


def test_box_inverse_512(orc):
    """8x8x8: Ahat_b A_b = I (the paper's largest block)."""
    A = kron_A(8, 8, 8, (1.0, 1.0, 1.0))
    inv = orc.box_inverse((8, 8, 8), (1.0, 1.0, 1.0))
    assert np.abs(inv @ A - np.eye(512)).max() < 1e-12


GRID_BOX = [((4, 4, 2), (2, 2, 1)), ((4, 4, 2), (4, 2, 2)), ((4, 4, 2), (1, 1, 1)),
            ((6, 4, 4), (2, 1, 2)), ((6, 4, 4), (3, 2, 2)), ((8, 4, 2), (4, 4, 2))]


@pytest.mark.parametrize("grid,box", GRID_BOX)
@pytest.mark.parametrize("a", COEFFS)
@pytest.mark.parametrize("omega", [1.0, 0.8])
def test_box_jacobi_dense_splitting(orc, grid, box, a, omega):
    nx, ny, nz = grid
    u0 = uniform_field((nz, ny, nx), 11)
    b = uniform_field((nz, ny, nx), 12)
    A = kron_A(nx, ny, nz, a)
    lab, _ = box_labels(nx, ny, nz, box)
    D = np.where(lab[:, None] == lab[None, :], A, 0.0)
    ref = u0.ravel() + omega * np.linalg.solve(D, b.ravel() - A @ u0.ravel())
    got = orc.sweep(u0, b, a, block="box", box=box, method="jacobi", omega=omega).ravel()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("grid,box", GRID_BOX)
@pytest.mark.parametrize("order", ["gs_lex", "gs_reverse", "gs_zebra"])
@pytest.mark.parametrize("omega", [1.0, 0.8])
def test_box_gs_dense_splitting(orc, grid, box, order, omega):
    """Block SOR in matrix form: (D + omega L) u1 = ((1 - omega) D - omega U) u0 + omega b,
    L / U the couplings to blocks visited before / after."""
    nx, ny, nz = grid
    a = (0.3, 2.0, 0.7)
    u0 = uniform_field((nz, ny, nx), 13)
    b = uniform_field((nz, ny, nx), 14)
    A = kron_A(nx, ny, nz, a)
    lab, _ = box_labels(nx, ny, nz, box)
    pos = visit_position(nx, ny, nz, box, order)[lab]
    before = pos[:, None] > pos[None, :]
    after = pos[:, None] < pos[None, :]
    D = np.where(lab[:, None] == lab[None, :], A, 0.0)
    L, U = np.where(before, A, 0.0), np.where(after, A, 0.0)
    ref = np.linalg.solve(D + omega * L, ((1 - omega) * D - omega * U) @ u0.ravel() + omega * b.ravel())
    got = orc.sweep(u0, b, a, block="box", box=box, method=order, omega=omega).ravel()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("grid", [(4, 3, 5), (8, 8, 8), (2, 6, 3)])
@pytest.mark.parametrize("method", ["jacobi", "gs_lex"])
def test_one_block_is_exact_solve(orc, grid, method):
    nx, ny, nz = grid
    a = (1.0, 0.1, 0.01)
    b = rhs((nz, ny, nx))
    u0 = initial_guess((nz, ny, nx))
    got = orc.sweep(u0, b, a, block="box", box=grid, method=method, omega=1.0)
    ref = orc.exact_solve(b, a)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("pqr", [(1, 1, 1), (2, 3, 1), (6, 5, 4), (3, 1, 2)])
@pytest.mark.parametrize("a", COEFFS)
def test_point_blocks_damp_sine_mode(orc, pqr, a):
    """1x1x1 boxes = point Jacobi: one sweep multiplies a sine mode by
    1 - omega lambda_pqr / (2 (ax + ay + az))."""
    nx, ny, nz = 6, 5, 4
    p, q, r = pqr
    e = sine_mode(nx, ny, nz, p, q, r)
    s = [2 - 2 * np.cos(m * np.pi / (n + 1)) for m, n in ((p, nx), (q, ny), (r, nz))]
    lam = a[0] * s[0] + a[1] * s[1] + a[2] * s[2]
    g = 1 - 0.8 * lam / (2 * sum(a))
    got = orc.sweep(e, np.zeros_like(e), a, block="box", box=(1, 1, 1), method="jacobi", omega=0.8)
    assert np.abs(got - g * e).max() <= 1e-13


@pytest.mark.parametrize("method", ["jacobi", "gs_lex", "gs_reverse", "gs_zebra"])
@pytest.mark.parametrize("a", COEFFS)
def test_box_equals_line_and_plane(orc, method, a):
    nx, ny, nz = 7, 6, 5
    u0 = initial_guess((nz, ny, nx))
    b = rhs((nz, ny, nx))
    om = 0.8 if method == "jacobi" else 1.0
    for box, block in (((nx, 1, 1), "line"), ((nx, ny, 1), "plane")):
        got = orc.sweep(u0, b, a, block="box", box=box, method=method, omega=om)
        ref = orc.sweep(u0, b, a, block=block, method=method, omega=om)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (box, block)


@pytest.mark.parametrize("method", ["jacobi", "gs_lex", "gs_reverse", "gs_zebra"])
@pytest.mark.parametrize("a", COEFFS + [(0.01, 1.0, 0.1)])
def test_y_and_z_line_boxes_are_permuted_x_lines(orc, method, a):
    """A 1 x ny x 1 box is an x-line of the grid with x and y exchanged; a 1 x 1 x nz box an
    x-line of the grid whose axes (x, y, z) become (z, x, y).  Both permutations keep the
    visiting order (block index i fastest) and the two-colour parity i + j + k."""
    nx, ny, nz = 5, 7, 6
    u0 = initial_guess((nz, ny, nx))
    b = rhs((nz, ny, nx))
    om = 0.8 if method == "jacobi" else 1.0
    ax, ay, az = a
    got = orc.sweep(u0, b, a, block="box", box=(1, ny, 1), method=method, omega=om)
    ref = orc.sweep(u0.transpose(0, 2, 1).copy(), b.transpose(0, 2, 1).copy(), (ay, ax, az),
                    block="line", method=method, omega=om).transpose(0, 2, 1)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), "y-lines"
    got = orc.sweep(u0, b, a, block="box", box=(1, 1, nz), method=method, omega=om)
    ref = orc.sweep(u0.transpose(1, 2, 0).copy(), b.transpose(1, 2, 0).copy(), (az, ax, ay),
                    block="line", method=method, omega=om).transpose(2, 0, 1)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), "z-lines"


@pytest.mark.parametrize("method,omega,sweeps", [("jacobi", 0.8, 400), ("gs_zebra", 1.0, 200)])
def test_box_converges_to_exact(orc, method, omega, sweeps):
    n = 8
    a = (1.0, 1.0, 1.0)
    b = rhs((n, n, n))
    ref = orc.exact_solve(b, a)
    u = np.zeros_like(b)
    for _ in range(sweeps):
        u = orc.sweep(u, b, a, block="box", box=(2, 2, 2), method=method, omega=omega)
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("method,omega", [("jacobi", 0.8), ("gs_lex", 1.0), ("gs_zebra", 1.0)])
def test_larger_blocks_smooth_more(orc, method, omega):
    """Sec. 3: ||r_3|| / ||r_0|| from a random initial guess falls as the block grows,
    over the seven block sizes of the paper's study (32^3 grid, b = 0)."""
    n = 32
    a = (1.0, 1.0, 1.0)
    u0 = initial_guess((n, n, n))
    b = np.zeros_like(u0)
    r0 = orc.residual_norm(u0, b, a)
    ratios = []
    for box in PAPER_SIZES:
        u = u0
        for _ in range(3):
            u = orc.sweep(u, b, a, block="box", box=box, method=method, omega=omega)
        ratios.append(orc.residual_norm(u, b, a) / r0)
    assert all(x > y for x, y in zip(ratios, ratios[1:])), ratios
    assert ratios[0] < 0.05  # three sweeps already reduce the residual 20-fold


@pytest.mark.parametrize("block,box", [("box", (1, 1, 1)), ("line", None), ("plane", None)])
def test_asymptotic_factor_is_slowest_sine_mode(orc, block, box):
    """Sec. 3's sliding-window factor (||r_{i+k}|| / ||r_i||)^(1/k) for block Jacobi
    (omega = 0.8) with point, x-line and xy-plane blocks: every sine mode e_pqr is an
    eigenvector, with factor 1 - omega lambda_pqr / mu (mu = the block operator's eigenvalue
    on that mode), and the slowest one is (1,1,1); on a 10^3 grid after 600 sweeps the other
    modes have died out to 1e-6."""
    n, i, k = 10, 600, 50
    a = (1.0, 1.0, 1.0)
    s1 = 2 - 2 * np.cos(np.pi / (n + 1))
    mu = {"box": 6.0, "line": s1 + 4, "plane": 2 * s1 + 2}[block]
    g = 1 - 0.8 * 3 * s1 / mu
    u = initial_guess((n, n, n))
    b = np.zeros_like(u)
    kw = {"box": box} if box else {}
    for _ in range(i):
        u = orc.sweep(u, b, a, block=block, method="jacobi", omega=0.8, **kw)
    ri = orc.residual_norm(u, b, a)
    for _ in range(k):
        u = orc.sweep(u, b, a, block=block, method="jacobi", omega=0.8, **kw)
    fac = (orc.residual_norm(u, b, a) / ri) ** (1.0 / k)
    assert abs(fac - g) <= 1e-6, (fac, g)


@pytest.mark.parametrize("box", [(1, 1, 1), (2, 2, 2), (4, 2, 2), (2, 2, 4)])
def test_two_colour_gs_factor_is_square_of_jacobi(orc, box):
    """Young's theorem: with the blocks coloured by the parity of bi + bj + bk, the block
    matrix is 2-cyclic and consistently ordered, so two-colour block GS (omega = 1) contracts
    with rho_J^2, rho_J the undamped block-Jacobi factor; damped Jacobi (omega = 0.8) has
    1 - 0.8 (1 - rho_J).  Both measured as sliding-window factors from a random guess, b = 0."""
    n, i, k = 8, 300, 40
    a = (1.0, 1.0, 1.0)
    u0 = initial_guess((n, n, n))
    b = np.zeros_like(u0)

    def factor(method, omega):
        u = u0
        for _ in range(i):
            u = orc.sweep(u, b, a, block="box", box=box, method=method, omega=omega)
        ri = orc.residual_norm(u, b, a)
        for _ in range(k):
            u = orc.sweep(u, b, a, block="box", box=box, method=method, omega=omega)
        return (orc.residual_norm(u, b, a) / ri) ** (1.0 / k)

    gj = factor("jacobi", 0.8)
    rho = 1 - (1 - gj) / 0.8
    assert abs(factor("gs_zebra", 1.0) - rho * rho) <= 1e-6, (gj, rho)


@pytest.mark.parametrize("block", ["line", "plane"])
def test_zebra_line_and_plane_gs_factor_is_square_of_jacobi(orc, block):
    """The same relation for full-extent lines (colour = parity of j + k) and planes (parity of
    k): two colours make the block matrix 2-cyclic and consistently ordered."""
    n, i, k = 8, 200, 40
    a = (1.0, 0.5, 0.25)
    u0 = initial_guess((n, n, n))
    b = np.zeros_like(u0)

    def factor(method, omega):
        u = u0
        for _ in range(i):
            u = orc.sweep(u, b, a, block=block, method=method, omega=omega)
        ri = orc.residual_norm(u, b, a)
        for _ in range(k):
            u = orc.sweep(u, b, a, block=block, method=method, omega=omega)
        return (orc.residual_norm(u, b, a) / ri) ** (1.0 / k)

    rho = 1 - (1 - factor("jacobi", 0.8)) / 0.8
    assert abs(factor("gs_zebra", 1.0) - rho * rho) <= 1e-6, rho


def test_box_must_tile_grid(orc):
    u = np.zeros((4, 4, 6))
    with pytest.raises(ValueError):
        orc.sweep(u, u, (1, 1, 1), block="box", box=(4, 4, 4))
