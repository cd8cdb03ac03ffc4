"""h2_matvec_noalloc: the product for callers that cannot allocate device memory.

Such callers (a time-stepping loop that reserved its device memory up front,
or an application whose device memory belongs to its own pool allocator)
call h2_matvec_noalloc, which takes its workspace from a fixed array inside
the library instead of allocating.  This test calls it through the C ABI,
twice in a row, and checks each result against h2_matvec's within the FP64
parity tolerance of the other GPU tests; it also checks that a problem larger
than the fixed scratch is refused with H2_ERR_SCRATCH_LIMIT.  The file is
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
H2_ERR_SCRATCH_LIMIT = -10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    pkg.load()


def _rel(y, ref):
    return np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("mk,m_,leaf,r", [(lambda: synth.cube_surface(12), 4, 64, 3),
                                          (lambda: synth.icosphere(3), 3, 32, 1)])
def test_noalloc_matches_matvec_twice(mk, m_, leaf, r):
    mesh = mk()
    g = pkg.Geometry(mesh.xyz, mesh.tri)
    op = pkg.Operator(g, m=m_, leaf=leaf, max_rhs=r)
    L = pkg.load()
    stream = int(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        x = torch.from_numpy(synth.gaussian_rhs(mesh.n_vertices, r, 100 + call)).cuda()
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        assert L.h2_matvec(ctypes.c_void_p(op.handle), ctypes.c_void_p(x.data_ptr()),
                           ctypes.c_void_p(y_ref.data_ptr()), r, ctypes.c_void_p(stream)) == 0
        assert L.h2_matvec_noalloc(ctypes.c_void_p(op.handle), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), r, ctypes.c_void_p(stream)) == 0
        torch.cuda.synchronize()
        err = _rel(y.cpu().numpy(), y_ref.cpu().numpy())
        assert np.all(err <= FP64_TOL), (call, err)
    assert pkg.h2_device_status(op.handle) == 0


def test_noalloc_refuses_problems_beyond_its_scratch():
    mesh = synth.cube_surface(64)
    g = pkg.Geometry(mesh.xyz, mesh.tri)
    op = pkg.Operator(g, m=4, leaf=64)
    x = torch.zeros((32, mesh.n_vertices), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    L = pkg.load()
    code = L.h2_matvec_noalloc(ctypes.c_void_p(op.handle), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), 32, None)
    assert code == H2_ERR_SCRATCH_LIMIT
    assert "scratch" in pkg.h2_error_string(code)
