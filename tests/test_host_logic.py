"""Host-side logic that needs no GPU: the cell-update accounting and the C ABI surface."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _table2():
    rows = []
    for line in (ROOT / "tests/golden/table2_cell_counts.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        label, patches, sweeps, printed, status = line.split("\t")
        dims = []
        for part in patches.split(","):
            edge, count = part.split("x")
            dims += [(int(edge),) * 3] * int(count)
        rows.append((label, dims, int(sweeps), int(printed), status))
    return rows


@pytest.mark.parametrize("row", _table2(), ids=lambda r: r[0])
def test_cell_updates_match_table2(row):
    """Table 2 (Sec. 4.2) counts cells x 3 sweeps; the metric's numerator must reproduce it."""
    from paper_1208_1975_gb300 import cell_updates

    label, dims, sweeps, printed, status = row
    got = cell_updates(dims, sweeps)
    if status == "exact":
        assert got == printed
    else:
        assert got == int(status.split(":")[1]) and got != printed


def _header_symbols():
    text = (ROOT / "include/brsmooth.h").read_text()
    return sorted(set(re.findall(r"\b(brsmooth_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def cuda_lib():
    import paper_1208_1975_gb300 as brs

    brs.build()
    return brs.lib()


def test_library_exports_every_declared_symbol(cuda_lib):
    syms = _header_symbols()
    assert len(syms) >= 8
    for s in syms:
        assert hasattr(cuda_lib, s), s


def test_strerror_and_null_handling(cuda_lib):
    import paper_1208_1975_gb300 as brs

    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(brs.brsmooth_strerror(code), str) and brs.brsmooth_strerror(code)
    assert brs.brsmooth_destroy(None) == brs.BRS_OK
    assert brs.brsmooth_sweep(None, None, None, 1, 0) == brs.BRS_ERR_ARG
    assert brs.brsmooth_sweep_host(None, None, None, 1, 0) == brs.BRS_ERR_ARG
    assert brs.brsmooth_sweep_host_async(None, None, None, 1, 0) == brs.BRS_ERR_ARG
    assert brs.brsmooth_residual(None, None, None, None, True, 0)[0] == brs.BRS_ERR_ARG
    assert brs.brsmooth_last_error(None) == brs.BRS_ERR_ARG
    assert brs.brsmooth_cells(None) == 0


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(ny=-1), dict(nz=0), dict(ax=0.0), dict(ay=-1.0), dict(az=float("nan")),
    dict(ax=float("inf")), dict(block=5), dict(block=-1), dict(method=5), dict(dtype=3), dict(omega=2.0),
    dict(omega=float("nan")), dict(plane_math=9), dict(block=2),
    dict(block=2, bx=2, by=2, bz=0), dict(block=2, bx=3, by=2, bz=2),
    dict(block=2, bx=2, by=16, bz=2)])
def test_create_rejects_bad_params_before_any_device_call(cuda_lib, bad):
    import paper_1208_1975_gb300 as brs

    base = dict(nx=8, ny=8, nz=8, ax=1.0, ay=1.0, az=1.0, block=0, method=0, dtype=0, omega=0.0,
                plane_math=0)
    base.update(bad)
    p = brs.brs_params(**base)
    rc, h = brs.brsmooth_create(p)
    assert rc == brs.BRS_ERR_ARG and not h.value
    rc = cuda_lib.brsmooth_create(None, ctypes.byref(ctypes.c_void_p()))
    assert rc == brs.BRS_ERR_ARG


def test_params_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of brs_params has the C header's size and field offsets."""
    import shutil
    import subprocess

    import paper_1208_1975_gb300 as brs

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in brs.brs_params._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "brsmooth.h"',
             'int main(void) {', '  printf("size %zu\\n", sizeof(brs_params));']
    lines += [f'  printf("{f} %zu\\n", offsetof(brs_params, {f}));' for f in fields]
    lines += ['  return 0;', '}']
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(brs.brs_params)
    for f in fields:
        assert int(out[f]) == getattr(brs.brs_params, f).offset, f


@pytest.mark.parametrize("case", [
    ([[4, 4, 4], [4, 4, 4]], [[-1, 1, -1, -1, -1, -1], [-1] * 6]),          # not symmetric
    ([[4, 4, 4], [4, 5, 4]], [[-1, 1, -1, -1, -1, -1], [0, -1, -1, -1, -1, -1]]),  # faces differ
    ([[4, 4, 1]], [[-1] * 6]),                                              # a dim below 2
    ([[4, 4, 4]], [[2, -1, -1, -1, -1, -1]]),                               # index out of range
    ([[4, 4, 4]], [[-2, -1, -1, -1, -1, -1]]),                              # negative index
])
def test_create_level_rejects_bad_tables_before_any_device_call(cuda_lib, case):
    import paper_1208_1975_gb300 as brs

    p = brs.brs_params(1, 1, 1, 1.0, 1.0, 1.0, 0, 1, 1, 0.0, 0)
    rc, h = brs.brsmooth_create_level(case[0], case[1], p)
    assert rc == brs.BRS_ERR_ARG and not h.value
