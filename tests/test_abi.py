"""Host-side checks of the C-ABI library (no GPU needed).

* the library builds for this machine, loads, and exports every entry point
  declared in include/h2bem.h;
* mesh validation rejects open, inward, inconsistently oriented, degenerate and
  non-manifold meshes before any device work, with the documented codes;
* argument checks (null handles, wrong handle kinds) return codes, not crashes.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1811_05731_gb300 as pkg
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "h2bem.h")

H2_ERR_INVALID_ARG = -1
H2_ERR_MESH_OPEN = -2
H2_ERR_MESH_ORIENTATION = -3
H2_ERR_DEGENERATE_TRIANGLE = -4


@pytest.fixture(scope="module")
def L():
    pkg.build()
    return pkg.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(h2_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "h2_matvec" in names and "h2_assemble" in names and "h2_build_geometry" in names
    assert "h2_free" in names
    raw = ctypes.CDLL(pkg.lib_path())
    for n in names:
        assert hasattr(raw, n), f"{n} declared in h2bem.h but not exported"


def test_error_strings(L):
    for code in range(0, -10, -1):
        s = pkg.h2_error_string(code)
        assert s and s != "unknown status"
    assert pkg.h2_error_string(-100) == "unknown status"


def test_default_params(L):
    p = pkg.h2_default_params()
    assert (p.m, p.leaf, p.eta, p.box_inflation, p.precision, p.max_rhs) == (4, 64, 2.0, 0.25, 0, 1)


def _geom_code(xyz, tri):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    h = ctypes.c_void_p()
    lib = pkg.load()
    code = lib.h2_build_geometry(xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), xyz.shape[0],
                                 tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), tri.shape[0],
                                 None, ctypes.byref(h))
    if code == 0:
        pkg.h2_free(h.value)
    return code


def test_rejects_open_mesh(L):
    m = synth.icosphere(1)
    assert _geom_code(m.xyz, m.tri[1:]) == H2_ERR_MESH_OPEN


def test_rejects_inward_mesh(L):
    m = synth.icosphere(1)
    assert _geom_code(m.xyz, m.tri[:, ::-1]) == H2_ERR_MESH_ORIENTATION


def test_rejects_inconsistent_orientation(L):
    m = synth.icosphere(1)
    tri = m.tri.copy()
    tri[3] = tri[3, ::-1]
    assert _geom_code(m.xyz, tri) == H2_ERR_MESH_ORIENTATION


def test_rejects_degenerate_triangle(L):
    m = synth.icosphere(1)
    tri = m.tri.copy()
    tri[0, 1] = tri[0, 0]
    assert _geom_code(m.xyz, tri) == H2_ERR_DEGENERATE_TRIANGLE
    xyz = m.xyz.copy()
    a, b, c = m.tri[0]
    xyz[c] = 0.5 * (xyz[a] + xyz[b])   # collinear corners
    assert _geom_code(xyz, m.tri) in (H2_ERR_DEGENERATE_TRIANGLE, H2_ERR_MESH_ORIENTATION)


def test_rejects_pinched_vertex(L):
    # two tetrahedra sharing one vertex: every edge is shared twice, but the
    # fan around the shared vertex has two cycles
    t = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    f = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])
    xyz = np.vstack([t, -t[1:]])
    tri2 = np.array([[0, 4, 5], [0, 6, 4], [0, 5, 6], [4, 6, 5]])
    tri = np.vstack([f, tri2])
    assert _geom_code(xyz, tri) == H2_ERR_MESH_OPEN


def test_rejects_bad_indices_and_nulls(L):
    m = synth.icosphere(1)
    tri = m.tri.copy()
    tri[0, 0] = m.n_vertices
    assert _geom_code(m.xyz, tri) == H2_ERR_INVALID_ARG
    lib = pkg.load()
    h = ctypes.c_void_p()
    assert lib.h2_build_geometry(None, 4, None, 4, None, ctypes.byref(h)) == H2_ERR_INVALID_ARG
    assert lib.h2_assemble(None, None, ctypes.byref(h)) == H2_ERR_INVALID_ARG
    assert lib.h2_matvec(None, None, None, 1, None) == H2_ERR_INVALID_ARG
    assert lib.h2_free(None) == 0


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled here."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    body = "".join(f'    printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"h2bem.h\"\nint main(void) {\n"
           f'    printf("%zu\\n", sizeof({struct}));\n{body}    return 0;\n}}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        with open(c, "w") as f:
            f.write(src)
        subprocess.run([cc, "-I", os.path.dirname(HEADER), c, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("struct,cls", [("h2_params", "Params"), ("h2_stats_t", "Stats"),
                                        ("h2_tuning_t", "Tuning"), ("h2_plan_report_t", "PlanReport")])
def test_binding_structs_match_the_header(struct, cls):
    """The binding's ctypes structures have the header's size and field offsets."""
    from paper_1811_05731_gb300 import _lib
    C = getattr(_lib, cls)
    names = [n for n, _ in C._fields_]
    size, offs = _c_layout(struct, names)
    assert ctypes.sizeof(C) == size
    assert [getattr(C, n).offset for n in names] == offs


def test_default_modes(L):
    p = pkg.h2_default_params()
    assert (p.schedule, p.autotune, p.coupling, p.near_field) == (pkg.SCHEDULE_FLOW, 0, pkg.COUPLING_STORED,
                                                                  pkg.NEAR_FP64)
