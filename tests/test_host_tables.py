"""CPU checks of the library's host-side table builders.

The sweeps read precomputed tables: the factor tables of the cross-lane scan Thomas solve
(one warp per line and two warps per line), the pivots of the elimination from both ends,
and the parity-class tables of the box inverse.  The builders are plain C++ headers in the
package's csrc/; a small harness (host_tables_harness.cpp) prints their output, and these
tests use the tables exactly as the kernels do -- in numpy emulations of the lane-parallel
solves -- and compare with direct dense solves.  A table entry that is wrong (an index off
by one, a multiplier over the wrong window, a sign) changes the solution and fails here.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1208_1975_gb300", "csrc")

# (a_x, a_y, a_z): isotropic, weak z, weak x, strong x
COEFFS = [(1.0, 1.0, 1.0), (1.0, 1.0, 0.01), (0.01, 1.0, 1.0), (2.0, 0.001, 0.001)]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("tables") / "host_tables")
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host_tables_harness.cpp"), "-o", exe],
                   check=True)

    def run(*args, stdin=None):
        r = subprocess.run([exe] + [str(a) for a in args], input=stdin, capture_output=True,
                           text=True, check=True)
        return r.stdout.split()

    return run


def _vec(tokens, pos, conv=float):
    n = int(tokens[pos])
    return np.array([conv(t) for t in tokens[pos + 1:pos + 1 + n]]), pos + 1 + n


def _tridiag(n, off, diag):
    return (np.diag(np.full(n, diag)) - off * np.diag(np.ones(n - 1), 1)
            - off * np.diag(np.ones(n - 1), -1))


def _scan_solve(tab, rhs, E, L, H, pair):
    """Lane-parallel Thomas solve with the tables, in the kernels' order: per-lane chunk
    summaries, Hillis-Steele scans over the lanes of each H-lane group, the carries (across
    the two groups of a pair through the group ends), then the per-lane sweeps.  Returns w
    (x_i = p_i w_i)."""
    NP = E * L
    LG = H.bit_length() - 1
    c, e = tab[:NP], tab[NP:2 * NP]
    af = lambda t, l: tab[3 * NP + t * L + l]
    ab = lambda t, l: tab[3 * NP + LG * L + t * L + l]
    r = rhs.copy()
    # forward
    B = np.zeros(L)
    for l in range(L):
        z = 0.0
        for q in range(E):
            z = c[l * E + q] * z + r[l * E + q]
        B[l] = z
    for t in range(LG):
        d = 1 << t
        nb = B.copy()
        for l in range(L):
            if l % H >= d:
                nb[l] = af(t, l) * B[l - d] + B[l]
        B = nb
    ends = B.copy()
    for l in range(L):
        carry = 0.0 if l % H == 0 else ends[l - 1]
        if pair and l >= H:
            carry += tab[3 * NP + 2 * LG * L + l] * ends[H - 1]
        z = carry
        for q in range(E):
            z = c[l * E + q] * z + r[l * E + q]
            r[l * E + q] = z
    # backward
    for l in range(L):
        w = 0.0
        for q in range(E - 1, -1, -1):
            w = e[l * E + q] * w + r[l * E + q]
        B[l] = w
    for t in range(LG):
        d = 1 << t
        nb = B.copy()
        for l in range(L):
            if l % H + d < H:
                nb[l] = ab(t, l) * B[l + d] + B[l]
        B = nb
    ends = B.copy()
    for l in range(L):
        carry = 0.0 if l % H == H - 1 else ends[l + 1]
        if pair and l < H:
            carry += tab[3 * NP + 2 * LG * L + L + l] * ends[H]
        w = carry
        for q in range(E - 1, -1, -1):
            w = e[l * E + q] * w + r[l * E + q]
            r[l * E + q] = w
    return r


# the lane layouts (cells per lane E, lanes G) of the one-warp solve
LAYOUTS = [(4, 4), (4, 8), (4, 16), (4, 32), (8, 32), (12, 32), (16, 32)]


def _scan_cases():
    prev = 0
    for E, G in LAYOUTS:
        NP = E * G
        for n in sorted({NP, NP - 3, prev + 1}):
            if n >= 1:
                yield E, G, n
        prev = NP


@pytest.mark.parametrize("a", COEFFS)
def test_scan_thomas_tables_solve_the_line(harness, a):
    """One-warp tables: the emulated solve times omega p_i equals omega M^{-1} rhs; cells
    beyond the line (set to noise) do not couple into it; the p_i block holds the pivots."""
    rng = np.random.default_rng(11)
    off, diag, omega = a[0], 2 * sum(a), 0.8
    for E, G, n in _scan_cases():
        tok = harness("scan", n, off, diag, omega, E, G, 1)
        tab, _ = _vec(tok, 0)
        NP = E * G
        LG = G.bit_length() - 1
        assert len(tab) == 4 * NP + 2 * LG * G
        rhs = rng.standard_normal(NP)
        w = _scan_solve(tab, rhs, E, G, G, pair=False)
        x = np.linalg.solve(_tridiag(n, off, diag), rhs[:n])
        got = tab[2 * NP:2 * NP + n] * w[:n]
        np.testing.assert_allclose(got, omega * x, rtol=0, atol=1e-11 * np.abs(x).max(),
                                   err_msg=f"E={E} G={G} n={n}")
        p = tab[3 * NP + 2 * LG * G:]
        np.testing.assert_allclose(p[:n] * w[:n], x, rtol=0, atol=1e-11 * np.abs(x).max())
        assert np.all(tab[2 * NP + n:3 * NP] == 0) and np.all(p[n:] == 0)


@pytest.mark.parametrize("a", COEFFS)
@pytest.mark.parametrize("n", [512, 511, 480, 416, 385, 300, 257, 256, 100])
def test_pair_tables_solve_the_line(harness, a, n):
    """Two-warp tables (64 lanes of 8 cells, two scan groups of 32 lanes joined by the
    group-end carries): the emulated solve equals the direct solve."""
    rng = np.random.default_rng(n)
    off, diag, omega = a[0], 2 * sum(a), 0.7
    tab, _ = _vec(harness("pair", n, off, diag, omega), 0)
    assert len(tab) == 3 * 512 + 768
    rhs = rng.standard_normal(512)
    w = _scan_solve(tab, rhs, 8, 64, 32, pair=True)
    x = np.linalg.solve(_tridiag(n, off, diag), rhs[:n])
    np.testing.assert_allclose(tab[1024:1024 + n] * w[:n], omega * x, rtol=0,
                               atol=1e-11 * np.abs(x).max())


def test_pair_tables_refuse_long_lines(harness):
    tab, _ = _vec(harness("pair", 513, 1.0, 6.0, 1.0), 0)
    assert len(tab) == 0


@pytest.mark.parametrize("a", COEFFS)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 64, 255, 256, 511, 512])
def test_twist_pivots_solve_the_line(harness, a, n):
    """Pivots of the elimination from both ends: left of the twist cell m = (n-1)/2 the
    forward recurrence y_i = r_i + off pv_{i-1} y_{i-1}, right of it the mirrored one, at m
    x_m = g_m (r_m + off pv_{m-1} y_{m-1} + off pv_{m+1} z_{m+1}), then substitution
    outwards x_i = pv_i (y_i + off x_{i+1}) (left) and pv_i (z_i + off x_{i-1}) (right)."""
    rng = np.random.default_rng(3 * n + 1)
    off, diag = a[0], 2 * sum(a)
    pv, _ = _vec(harness("twist", n, off, diag), 0)
    assert len(pv) == n
    r = rng.standard_normal(n)
    m = (n - 1) // 2
    y = np.zeros(n)
    z = np.zeros(n)
    for i in range(m):
        y[i] = r[i] + (off * pv[i - 1] * y[i - 1] if i else 0.0)
    for i in range(n - 1, m, -1):
        z[i] = r[i] + (off * pv[i + 1] * z[i + 1] if i < n - 1 else 0.0)
    x = np.zeros(n)
    x[m] = pv[m] * (r[m] + (off * pv[m - 1] * y[m - 1] if m >= 1 else 0.0)
                    + (off * pv[m + 1] * z[m + 1] if m + 1 < n else 0.0))
    for i in range(m - 1, -1, -1):
        x[i] = pv[i] * (y[i] + off * x[i + 1])
    for i in range(m + 1, n):
        x[i] = pv[i] * (z[i] + off * x[i - 1])
    ref = np.linalg.solve(_tridiag(n, off, diag), r) if n > 1 else r / diag
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


# ---------------------------------------------------------------- box parity classes

def _box_matrix(b, a):
    """7-point block matrix of a bx x by x bz box (cell l = x + bx (y + by z)), couplings to
    cells outside the box dropped."""
    bx, by, bz = b
    n = bx * by * bz
    A = np.zeros((n, n))
    for z in range(bz):
        for y in range(by):
            for x in range(bx):
                l = x + bx * (y + by * z)
                A[l, l] = 2 * sum(a)
                for d, (dx, dy, dz) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
                    for s in (1, -1):
                        X, Y, Z = x + s * dx, y + s * dy, z + s * dz
                        if 0 <= X < bx and 0 <= Y < by and 0 <= Z < bz:
                            A[l, X + bx * (Y + by * Z)] = -a[d]
    return A


def _fold_matrix(b):
    """G from its definition, rows in class-major order (class bit d set: differences along
    axis d), within a class the folded coordinates lexicographic with x fastest.  Along an
    axis of extent e the sums are j < ceil(e/2) (cells j and e-1-j, or the middle cell alone),
    the differences j < floor(e/2) (cell j minus cell e-1-j).  Also returns the class sizes
    and W (1/2 per mirrored pair along each axis)."""
    bx, by, bz = b
    n = bx * by * bz
    half = [(e - e // 2, e // 2) for e in b]

    def axis_rows(e, diff):
        rows = []
        for j in range(e // 2 if diff else e - e // 2):
            v = np.zeros(e)
            v[j] += 1.0
            if j < e // 2:
                v[e - 1 - j] += -1.0 if diff else 1.0
            rows.append(v)
        return rows

    G, W, sizes = [], [], []
    for cl in range(8):
        bits = [(cl >> d) & 1 for d in range(3)]
        R = [axis_rows(b[d], bits[d]) for d in range(3)]
        sizes.append(len(R[0]) * len(R[1]) * len(R[2]))
        for jz, vz in enumerate(R[2]):
            for jy, vy in enumerate(R[1]):
                for jx, vx in enumerate(R[0]):
                    G.append(np.kron(vz, np.kron(vy, vx)))
                    w = 1.0
                    for d, j in enumerate((jx, jy, jz)):
                        if j < half[d][1]:
                            w *= 0.5
                    W.append(w)
    G = np.array(G).reshape(-1, n)
    return G, np.array(W), sizes


def _apply_passes(tab, v, d):
    """One separable pass of the tables: out[o] = in[a] + sign(b) in[|b| - 1] (b = 0: in[a])."""
    n = len(v)
    t = tab[2 * d * n:2 * (d + 1) * n].reshape(n, 2)
    a, s = t[:, 0], t[:, 1]
    out = v[a].copy()
    m = s != 0
    out[m] += np.sign(s[m]) * v[np.abs(s[m]) - 1]
    return out


def _parity(harness, b, inv):
    tok = harness("parity", *b, stdin="\n".join("%.17g" % x for x in inv.ravel()))
    use = int(tok[0]) == 1
    cls_n = [int(t) for t in tok[1:9]]
    cls_off = [int(t) for t in tok[9:17]]
    pc_off = [int(t) for t in tok[17:25]]
    pc, pos = _vec(tok, 25)
    ftab, pos = _vec(tok, pos, int)
    utab, pos = _vec(tok, pos, int)
    return use, cls_n, cls_off, pc_off, pc, ftab, utab


PARITY_BOXES = [(8, 8, 8), (7, 7, 1), (5, 6, 7), (8, 4, 4), (8, 1, 8), (1, 16, 3)]


@pytest.mark.parametrize("b", PARITY_BOXES)
def test_box_parity_tables(harness, b):
    """Parity tables of the box inverse: the fold passes compose to G, the unfold passes to
    G^T, the class blocks of P are those of W G Ahat G^T W, whose blocks between different
    classes vanish (Ahat is invariant under the box's reflections), and unfold(P fold(r))
    = Ahat r."""
    a = (1.0, 0.3, 0.01)
    A = _box_matrix(b, a)
    inv = np.linalg.inv(A)
    n = A.shape[0]
    use, cls_n, cls_off, pc_off, pc, ftab, utab = _parity(harness, b, inv)
    G, W, sizes = _fold_matrix(b)
    assert use
    assert cls_n == sizes and cls_off == list(np.cumsum([0] + sizes[:-1]))
    # passes as matrices (columns of the identity pushed through)
    I = np.eye(n)
    F = np.array([_apply_passes(ftab, _apply_passes(ftab, _apply_passes(ftab, I[:, j], 0), 1), 2)
                  for j in range(n)]).T
    U = np.array([_apply_passes(utab, _apply_passes(utab, _apply_passes(utab, I[:, j], 0), 1), 2)
                  for j in range(n)]).T
    np.testing.assert_array_equal(F, G)
    np.testing.assert_array_equal(U, G.T)
    np.testing.assert_allclose(G.T @ np.diag(W) @ G, I, atol=1e-15)
    P = np.diag(W) @ G @ inv @ G.T @ np.diag(W)
    scale = np.abs(P).max()
    for cl in range(8):
        o, nc = cls_off[cl], cls_n[cl]
        blk = pc[pc_off[cl]:pc_off[cl] + nc * nc].reshape(nc, nc)
        np.testing.assert_allclose(blk, P[o:o + nc, o:o + nc], rtol=0, atol=1e-14 * scale)
        Q = P[o:o + nc].copy()
        Q[:, o:o + nc] = 0
        assert np.abs(Q).max(initial=0.0) <= 1e-13 * scale
    rng = np.random.default_rng(sum(b))
    r = rng.standard_normal(n)
    f = _apply_passes(ftab, _apply_passes(ftab, _apply_passes(ftab, r, 0), 1), 2)
    g = np.zeros(n)
    for cl in range(8):
        o, nc = cls_off[cl], cls_n[cl]
        g[o:o + nc] = pc[pc_off[cl]:pc_off[cl] + nc * nc].reshape(nc, nc) @ f[o:o + nc]
    u = _apply_passes(utab, _apply_passes(utab, _apply_passes(utab, g, 0), 1), 2)
    ref = inv @ r
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("b", [(4, 4, 4), (3, 3, 3), (6, 1, 6), (1, 1, 1), (2, 2, 1)])
def test_box_parity_tables_off_for_small_classes(harness, b):
    """Boxes whose largest class has fewer than 16 cells keep the full product."""
    inv = np.linalg.inv(_box_matrix(b, (1.0, 1.0, 1.0)))
    use, cls_n, *_ = _parity(harness, b, inv)
    assert not use
    assert sum(cls_n) == inv.shape[0] and max(cls_n) < 16
