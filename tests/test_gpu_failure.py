"""Failure detection without a GPU fault: a dependency that never completes
makes one bounded device-side wait (1 s) run out; the product stops, the
host reads H2_ERR_TIMEOUT, and the CUDA context stays usable."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1811_05731_gb300 as pkg  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

H2_ERR_TIMEOUT = -7


def test_stalled_dependency_times_out_and_context_recovers():
    m = synth.cube_surface(12)
    x = synth.gaussian_rhs(m.n_vertices, 1, 3)
    ref = oracle.H2Oracle(m.xyz, m.tri, 4, 64, 2.0).matvec(x)
    g = pkg.Geometry(m.xyz, m.tri)
    op = pkg.Operator(g, m=4, leaf=64)
    xd = torch.from_numpy(x).cuda()
    L = pkg.load()
    assert L.h2_fault_inject_stall(op.handle, 1) == 0
    t0 = time.perf_counter()
    op.matvec(xd)
    torch.cuda.synchronize()
    assert pkg.h2_device_status(op.handle) == H2_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert L.h2_fault_inject_stall(op.handle, 0) == 0
    y = op.matvec(xd).cpu().numpy()
    assert pkg.h2_device_status(op.handle) == 0
    assert np.linalg.norm(y - ref) <= 1e-8 * np.linalg.norm(ref)
