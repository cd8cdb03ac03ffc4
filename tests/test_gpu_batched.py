"""Batched product over several meshes of uneven size in one persistent launch
(h2_matvec_batched), against the per-operator product and the CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1811_05731_gb300 as pkg  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def rel_err(y, ref):
    return np.linalg.norm(y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


def _small_set():
    # (mesh, m, leaf, precision, r)
    return [(synth.icosphere(3), 3, 32, pkg.FP64, 2),
            (synth.cube_surface(12), 4, 64, pkg.BF16X3, 3),
            (synth.box_surface(9, 4, 3, 3.0, 1.0, 0.5), 2, 8, pkg.FP32, 1),
            (synth.cube_sphere(9), 4, 20, pkg.TF32X3, 5)]


def test_batched_small_meshes_match_oracle_and_single_products():
    items = _small_set()
    ops, xs, refs, singles = [], [], [], []
    for i, (mesh, m, leaf, prec, r) in enumerate(items):
        g = pkg.Geometry(mesh.xyz, mesh.tri)
        op = pkg.Operator(g, m=m, leaf=leaf, precision=prec, max_rhs=r)
        x = synth.gaussian_rhs(mesh.n_vertices, r, 100 + i)
        ops.append(op)
        xs.append(torch.from_numpy(x).cuda())
        refs.append(oracle.H2Oracle(mesh.xyz, mesh.tri, m, leaf, 2.0).matvec(x))
        singles.append(op.matvec(xs[-1]).cpu().numpy())
    for _ in range(2):   # the second call reuses the cached combined schedule
        ys = pkg.matvec_batched(ops, xs, [torch.full_like(x, float("nan")) for x in xs])
        torch.cuda.synchronize()
        assert pkg.h2_device_status(ops[0].handle) == 0
        for (mesh, m, leaf, prec, r), y, ref, single in zip(items, ys, refs, singles):
            y = y.cpu().numpy()
            tol = 1e-8 if prec == pkg.FP64 else (1e-4 if prec == pkg.BF16X3 else 1e-5)
            assert np.all(rel_err(y, ref) <= tol), (prec, rel_err(y, ref))
            # same segments and arithmetic, only the order of atomic additions
            # differs -- except for tensor-core tiles, which the batched launch
            # (r up to 5: the tensor cores) and the single product of r <= 4 (the
            # CUDA cores) multiply on different pipes: both within the budget
            if prec in (pkg.TF32X3, pkg.BF16X3) and r <= 4:
                assert np.all(rel_err(y, single) <= tol), (prec, rel_err(y, single))
            else:
                assert np.all(rel_err(y, single) <= (1e-13 if prec == pkg.FP64 else 1e-6)), (prec, rel_err(y, single))


def test_batched_eight_uneven_meshes():
    """The eight meshes of 5k-100k nodes (m = 5, leaf 64) in one launch, FP64 and BF16 hi+lo."""
    meshes = synth.workloads.multi_mesh_set()
    for prec, tol in ((pkg.FP64, 1e-12), (pkg.BF16X3, 1e-6)):
        ops, xs = [], []
        for i, mesh in enumerate(meshes):
            g = pkg.Geometry(mesh.xyz, mesh.tri)
            ops.append(pkg.Operator(g, m=5, leaf=64, precision=prec, max_rhs=1))
            xs.append(torch.from_numpy(synth.smooth_states(mesh, 1, 1811 + i)).cuda())
        singles = [op.matvec(x).cpu().numpy() for op, x in zip(ops, xs)]
        ys = pkg.matvec_batched(ops, xs)
        torch.cuda.synchronize()
        assert pkg.h2_device_status(ops[0].handle) == 0
        for y, single in zip(ys, singles):
            assert np.all(rel_err(y.cpu().numpy(), single) <= tol)
        del ops


def test_batched_argument_checks():
    mesh = synth.icosphere(2)
    g = pkg.Geometry(mesh.xyz, mesh.tri)
    op = pkg.Operator(g, m=2, leaf=16, max_rhs=1)
    x = torch.zeros((1, mesh.n_vertices), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(pkg.H2Error):   # the same operator twice shares one workspace
        pkg.h2_matvec_batched([op.handle, op.handle], [x.data_ptr()] * 2, [y.data_ptr()] * 2, [1, 1])
    with pytest.raises(pkg.H2Error):   # r above max_rhs
        pkg.h2_matvec_batched([op.handle], [x.data_ptr()], [y.data_ptr()], [2])
