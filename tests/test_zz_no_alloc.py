"""h2_matvec_noalloc: the product for callers that cannot allocate device memory.

Such callers (a time-stepping loop that reserved its device memory up front,
or an application whose device memory belongs to its own pool allocator)
call h2_matvec_noalloc, which takes its workspace from a fixed array inside
the library instead of allocating.  This test calls it through the C ABI,
twice in a row, and checks each result against h2_matvec's within the
parity tolerances of the other GPU tests (FP64 and the reduced forms, r at
and above the operator's max_rhs); it also checks that a problem larger than
the fixed scratch is refused with H2_ERR_SCRATCH_LIMIT and an r the staged
chunks cannot hold with H2_ERR_RHS_EXCEEDS_MAX.  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_1811_05731_gb300")

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-8
MIXED_TOL = 1e-5            # the reduced-precision tolerance of the other GPU parity tests
H2_ERR_RHS_EXCEEDS_MAX = -8
H2_ERR_SCRATCH_LIMIT = -10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    pkg.load()


# The max-norm error is held to twice the tolerance: a rounding error spread
# over the rows peaks at a few times its root mean square, while an error
# confined to one leaf or block at ten times the budget still fails.
MAXNORM_FACTOR = 2.0


def _rel(y, ref):
    """The larger of the relative L2 and the relative max-norm error per right-hand side."""
    l2 = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    mx = np.max(np.abs(y - ref), axis=1) / np.max(np.abs(ref), axis=1)
    return np.maximum(l2, mx / MAXNORM_FACTOR)


# (mesh, m, leaf, precision, max_rhs of the operator, r of the calls)
CASES = [
    ("cube12_fp64_r3", lambda: synth.cube_surface(12), 4, 64, 0, 3, 3),
    ("ico3_fp64_r1", lambda: synth.icosphere(3), 3, 32, 0, 1, 1),
    # reduced precision: the FP32 workspace sits in the same array after the FP64 one
    ("ico3_fp32_r3", lambda: synth.icosphere(3), 3, 32, 1, 3, 3),
    ("ico3_bf16x3_r3", lambda: synth.icosphere(3), 3, 32, 3, 3, 3),
    # more right-hand sides than the operator was assembled for (max_rhs 16, r 12
    # and 24), on the CUDA cores and on the tensor cores
    ("cube12_fp64_r12_of16", lambda: synth.cube_surface(12), 4, 64, 0, 16, 12),
    ("cube12_bf16x3_r24_of16", lambda: synth.cube_surface(12), 4, 64, 3, 16, 24),
]


def _call(L, fn, op, x, y, r, stream):
    return fn(ctypes.c_void_p(op.handle), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), r,
              ctypes.c_void_p(stream))


@pytest.mark.parametrize("name,mk,m_,leaf,prec,max_rhs,r", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_matvec_twice(name, mk, m_, leaf, prec, max_rhs, r):
    """Two calls in a row on fresh inputs: h2_matvec_noalloc (fixed scratch,
    level-wise launches) against h2_matvec on the same operator (its own
    workspace, the dataflow launch): the same segments and arithmetic in
    another order of atomic additions, so the FP64 tolerance in FP64 and the
    reduced forms' tolerance otherwise."""
    mesh = mk()
    g = pkg.Geometry(mesh.xyz, mesh.tri)
    op = pkg.Operator(g, m=m_, leaf=leaf, max_rhs=max_rhs, precision=prec)
    # h2_matvec needs r <= max_rhs: the reference for r > max_rhs comes from
    # a second operator of the same mesh and parameters assembled for r
    ref_op = op if r <= max_rhs else pkg.Operator(g, m=m_, leaf=leaf, max_rhs=r, precision=prec)
    L = pkg.load()
    stream = int(torch.cuda.current_stream().cuda_stream)
    tol = FP64_TOL if prec == 0 else MIXED_TOL
    for call in range(2):
        x = torch.from_numpy(synth.gaussian_rhs(mesh.n_vertices, r, 100 + call)).cuda()
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        assert _call(L, L.h2_matvec, ref_op, x, y_ref, r, stream) == 0
        assert _call(L, L.h2_matvec_noalloc, op, x, y, r, stream) == 0
        torch.cuda.synchronize()
        err = _rel(y.cpu().numpy(), y_ref.cpu().numpy())
        assert np.all(err <= tol), (call, err)
    assert pkg.h2_device_status(op.handle) == 0
    assert pkg.h2_device_status(ref_op.handle) == 0


def test_noalloc_refuses_r_above_eight_on_small_operators():
    """An operator assembled for at most 8 right-hand sides stages 128 input
    columns per chunk, which leaves room for at most 8 right-hand sides: r = 12
    is refused with H2_ERR_RHS_EXCEEDS_MAX (nothing launched), r = 8 runs."""
    mesh = synth.icosphere(3)
    g = pkg.Geometry(mesh.xyz, mesh.tri)
    op = pkg.Operator(g, m=3, leaf=32, max_rhs=1)
    L = pkg.load()
    stream = int(torch.cuda.current_stream().cuda_stream)
    x = torch.zeros((12, mesh.n_vertices), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _call(L, L.h2_matvec_noalloc, op, x, y, 12, stream) == H2_ERR_RHS_EXCEEDS_MAX
    assert _call(L, L.h2_matvec_noalloc, op, x, y, 33, stream) == H2_ERR_RHS_EXCEEDS_MAX
    assert _call(L, L.h2_matvec_noalloc, op, x[:8], y[:8], 8, stream) == 0
    torch.cuda.synchronize()
    assert pkg.h2_device_status(op.handle) == 0


def test_noalloc_refuses_problems_beyond_its_scratch():
    mesh = synth.cube_surface(64)
    g = pkg.Geometry(mesh.xyz, mesh.tri)
    # assembled for more than 8 right-hand sides, so that r = 32 passes the
    # staging limit and meets the scratch limit (about 150,000 rows x 32 values)
    op = pkg.Operator(g, m=4, leaf=64, max_rhs=16)
    x = torch.zeros((32, mesh.n_vertices), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    L = pkg.load()
    code = L.h2_matvec_noalloc(ctypes.c_void_p(op.handle), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), 32, None)
    assert code == H2_ERR_SCRATCH_LIMIT
    assert "scratch" in pkg.h2_error_string(code)
