"""Host-side checks of the C ABI (no GPU needed): the library builds/loads, exports every
entry point declared in include/vsie.h, and rejects invalid arguments before touching
the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2607_06429_b300 import binding as B
from paper_2607_06429_b300 import build as BUILD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(vsie_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load_library()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert {"vsie_create", "vsie_apply", "vsie_solve", "vsie_adjoint_apply"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(B.EXPORTS) == declared


def test_create_rejects_null_and_bad_sizes(lib):
    h = ctypes.c_void_p()
    assert lib.vsie_create(None, None, 1.0, None, ctypes.byref(h)) == 1
    assert b"null" in lib.vsie_last_error()
    vert = np.zeros(12)
    tet = np.array([0, 1, 2, 3], dtype=np.int32)
    mesh = B._Mesh(4, vert.ctypes.data_as(ctypes.c_void_p), 1, tet.ctypes.data_as(ctypes.c_void_p), 0, None)
    rho = np.ones(1)
    mat = B._Material(1.0, 1.0, rho.ctypes.data_as(ctypes.c_void_p), rho.ctypes.data_as(ctypes.c_void_p),
                      None, None, None)
    # non-positive wavenumber is rejected before any device work
    assert lib.vsie_create(ctypes.byref(mesh), ctypes.byref(mat), -1.0, None, ctypes.byref(h)) == 1
    assert b"k0" in lib.vsie_last_error()
    assert not h.value


def test_calls_reject_null_handle(lib):
    assert lib.vsie_apply(None, None, None, 1, 32, None) == 1
    assert lib.vsie_adjoint_apply(None, None, None, 1, 32, None) == 1
    assert lib.vsie_sizes(None, None, None, None) == 1
    assert lib.vsie_solve(None, None, None, None, None, None) == 1
    assert lib.vsie_plane_wave_rhs(None, None, 0, None, None) == 1
    assert lib.vsie_far_field(None, None, 1, None, 1, None, None) == 1


def test_cuboid_create_rejects_bad_grids(lib):
    h = ctypes.c_void_p()
    e = np.array([0.0, 1.0, 2.0])
    rho = np.ones(8)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    assert lib.vsie_create_cuboid(None, P(rho), P(rho), 1.0, 1.0, 1.0, ctypes.byref(h)) == 1
    grid = B._CuboidGrid(2, 2, 2, P(e), P(e), None)
    assert lib.vsie_create_cuboid(ctypes.byref(grid), P(rho), P(rho), 1.0, 1.0, 1.0, ctypes.byref(h)) == 1
    grid = B._CuboidGrid(0, 2, 2, P(e), P(e), P(e))
    assert lib.vsie_create_cuboid(ctypes.byref(grid), P(rho), P(rho), 1.0, 1.0, 1.0, ctypes.byref(h)) == 1
    assert b"sizes" in lib.vsie_last_error()
    grid = B._CuboidGrid(2, 2, 2, P(e), P(e), P(e))
    assert lib.vsie_create_cuboid(ctypes.byref(grid), P(rho), P(rho), 1.0, 1.0, 0.0, ctypes.byref(h)) == 1
    assert b"k0" in lib.vsie_last_error()
    assert lib.vsie_create_cuboid(ctypes.byref(grid), P(rho), P(rho), 1.0, 1.0, 1.0, None) == 1
    assert not h.value


def test_field_and_frequency_calls_reject_null_handle(lib):
    pts = np.zeros(3)
    assert lib.vsie_scattered_field(None, None, 1, pts.ctypes.data_as(ctypes.c_void_p), 1, 64, None, None) == 1
    assert lib.vsie_set_frequency(None, 2.0) == 1
    assert b"vsie_set_frequency" in lib.vsie_last_error()


def test_header_is_plain_c_and_matches_the_binding_layouts(tmp_path):
    """include/vsie.h and include/vsie_bem.h compile as pedantic C99, and the structs the
    binding mirrors have the same sizes on both sides."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(
        '#include <stdio.h>\n#include "vsie.h"\n#include "vsie_bem.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(vsie_mesh), sizeof(vsie_material),\n'
        "         sizeof(vsie_options), sizeof(vsie_solve_opts), sizeof(vsie_solve_info),\n"
        "         sizeof(vsie_cuboid_grid), sizeof(vsie_bem_desc), sizeof(vsie_tuning));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                            text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(B._Mesh), ctypes.sizeof(B._Material), ctypes.sizeof(B._Options),
                     ctypes.sizeof(B._SolveOpts), ctypes.sizeof(B._SolveInfo), ctypes.sizeof(B._CuboidGrid),
                     ctypes.sizeof(B._BemDesc), ctypes.sizeof(B._Tuning)]


def test_bem_calls_reject_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.vsie_bem_create(None, ctypes.byref(h)) == 1
    d = B._BemDesc()
    d.n_interfaces = 3
    assert lib.vsie_bem_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"n_interfaces" in lib.vsie_last_error()
    from paper_2607_06429_b300.workloads import icosphere
    v, t = icosphere(1, 1.0)
    v = np.ascontiguousarray(v)
    t = np.ascontiguousarray(t, dtype=np.int32)
    d.n_interfaces = 1
    d.h_vert[0] = v.ctypes.data
    d.h_tri[0] = t.ctypes.data
    d.n_vert[0], d.n_tri[0] = v.shape[0], t.shape[0]
    d.k0, d.rho0, d.c0, d.rho[0], d.c[0] = 2.0, 1.0, 1.0, 1.5, 0.8
    d.far_order = 9
    assert lib.vsie_bem_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"order" in lib.vsie_last_error()
    d.far_order = 3
    t_bad = t.copy()
    t_bad[5, 1] = v.shape[0]
    d.h_tri[0] = t_bad.ctypes.data
    assert lib.vsie_bem_create(ctypes.byref(d), ctypes.byref(h)) == 2     # VSIE_ERR_MESH
    d.h_tri[0] = t.ctypes.data
    d.k0 = -1.0
    assert lib.vsie_bem_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert not h.value
    assert lib.vsie_bem_apply(None, None, None, 32, None) == 1
    assert lib.vsie_bem_solve(None, None, None, None, None, None) == 1
    assert lib.vsie_bem_sizes(None, None, None, None) == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without libvsie.so the binding raises instead of computing."""
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(ImportError):
        B.load_library(str(tmp_path / "libvsie.so"))


def test_bem_binding_checks_its_arguments_on_the_host(lib):
    from paper_2607_06429_b300.workloads import icosphere
    s = icosphere(1, 1.0)
    with pytest.raises(ValueError):
        B.BemOperator([s], 2.0, [1.5, 3.0], [0.8])          # one layer, two densities
    with pytest.raises(ValueError):
        B.BemOperator([s, s, s], 2.0, [1.0] * 3, [1.0] * 3)  # at most two interfaces
    with pytest.raises(B.VsieError):
        B.BemOperator([s], -2.0, [1.5], [0.8])               # rejected by the library, no device work
