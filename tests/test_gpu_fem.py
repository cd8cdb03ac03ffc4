"""The finite-element half of the field evaluation on the GPU (h2_fem_create /
h2_fem_solve) against the oracle's pipeline (oracle/fem.py) and the physics.

Section "Basic Equations" of the paper: u1 from the Neumann problem, u2 on the
boundary from the boundary integral operator applied to u1 there, u2 inside
from the Dirichlet problem, and the energy (1/V) int M . grad(u1 + u2).

* With the exact operator (nothing admissible: every block an exact near
  block, the dense M of the oracle) the GPU's u1, u2 and energy equal the
  oracle's (sparse direct solves) to the conjugate-gradient tolerance, for a
  uniform and for a varying magnetisation.
* With the compressed operator: the cube's three factors are equal and
  converge to 1/3; the ball's to 1/3 at second order; a uniform M gives u1 =
  M.x up to a constant; the azimuthally magnetised 2:1 torus has an energy
  that vanishes under refinement while a uniform M on it gives an O(1) one.
"""
import numpy as np
import pytest

from oracle import fem
from synth import volume as vm

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_1811_05731_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    pkg.load()


def _setup(xyz, tets, eta=2.0, m=4, leaf=32):
    surf, nodes = vm.boundary_surface(xyz, tets)
    g = pkg.Geometry(surf.xyz, surf.tri)
    op = pkg.Operator(g, m=m, leaf=leaf, eta=eta)
    return surf, nodes, g, op, pkg.Fem(xyz, tets, nodes)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("gen,n", [(vm.cube_tets, 5), (vm.ball_tets, 6)])
def test_exact_operator_pipeline_matches_the_oracle(gen, n):
    xyz, tets = gen(n)
    surf, nodes, g, op, F = _setup(xyz, tets, eta=1e-9)
    assert op.stats()["n_far_blocks"] == 0
    c = xyz[tets].mean(axis=1)
    for M in (np.array([0.0, 0.0, 1.0]), np.array([0.6, -0.48, 0.64]),
              np.stack([np.cos(3 * c[:, 2]), np.sin(2 * c[:, 0]), 0.5 + 0.0 * c[:, 1]], axis=1)):
        u1_ref, u2_ref, e_ref = fem.pipeline(xyz, tets, M, surf, nodes)
        u1, u2, rep = F.solve(op, M, tol=1e-13)
        u1, u2 = u1.cpu().numpy(), u2.cpu().numpy()
        assert rep["resid_u1"] <= 1e-13 and rep["resid_u2"] <= 1e-13, rep
        assert _rel(u1, u1_ref) < 1e-9, _rel(u1, u1_ref)
        assert _rel(u2, u2_ref) < 1e-9, _rel(u2, u2_ref)
        assert abs(rep["energy"] - e_ref) < 1e-9 * max(1.0, abs(e_ref)), (rep["energy"], e_ref)
        assert abs(rep["volume"] - fem.p1_gradients(xyz, tets)[0].sum()) < 1e-12


def test_uniform_magnetisation_gives_a_linear_u1():
    xyz, tets = vm.ball_tets(6)
    _, _, _, op, F = _setup(xyz, tets)
    M = np.array([0.6, -0.48, 0.64])
    u1, _, rep = F.solve(op, M)
    d = u1.cpu().numpy() - xyz @ M
    assert np.ptp(d) < 1e-10, np.ptp(d)


def test_cube_factors_equal_and_converge_to_one_third():
    """The mesh is symmetric under axis permutations: with the exact operator
    the three factors agree to rounding; with the compressed one (whose
    cluster tree is not symmetric) to its approximation error, and they
    converge to 1/3."""
    errs = []
    for n in (3, 6, 12):
        xyz, tets = vm.cube_tets(n)
        if n <= 6:
            _, _, _, exact, Fx = _setup(xyz, tets, eta=1e-9)
            Nx = [Fx.solve(exact, np.eye(3)[d], tol=1e-13)[2]["energy"] for d in range(3)]
            assert max(Nx) - min(Nx) < 1e-11, Nx
        _, _, _, op, F = _setup(xyz, tets)
        Ns = [F.solve(op, np.eye(3)[d])[2]["energy"] for d in range(3)]
        assert max(Ns) - min(Ns) < 1e-3, Ns
        errs.append(abs(np.mean(Ns) - 1.0 / 3.0))
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5 and errs[2] < 4e-3, errs


def test_ball_factor_converges_at_second_order():
    errs = []
    for n in (4, 8, 16):
        xyz, tets = vm.ball_tets(n)
        _, _, _, op, F = _setup(xyz, tets)
        errs.append(abs(F.solve(op, [0.0, 0.0, 1.0])[2]["energy"] - 1.0 / 3.0))
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 2.5 and errs[2] < 1.5e-3, errs


def test_torus_azimuthal_energy_vanishes():
    es = []
    for nu, nc in ((12, 2), (24, 4), (36, 6)):
        xyz, tets = vm.torus_tets(nu, nc)
        _, _, _, op, F = _setup(xyz, tets, m=5)
        c = xyz[tets].mean(axis=1)
        phi = np.arctan2(c[:, 1], c[:, 0])
        M = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
        es.append(abs(F.solve(op, M)[2]["energy"]))
        if nc == 4:
            assert 0.3 < F.solve(op, [0.0, 0.0, 1.0])[2]["energy"] < 0.7
    assert es[1] < es[0] / 5 and es[2] < es[1] and es[2] < 1e-5, es


def test_fem_argument_checks():
    xyz, tets = vm.cube_tets(2)
    surf, nodes = vm.boundary_surface(xyz, tets)
    bad = tets.copy()
    bad[0, [1, 2]] = bad[0, [2, 1]]   # negative volume
    with pytest.raises(pkg.H2Error):
        pkg.Fem(xyz, bad, nodes)
    with pytest.raises(pkg.H2Error):
        pkg.Fem(xyz, tets, np.concatenate([nodes, nodes[:1]]))   # a repeated surface node
    F = pkg.Fem(xyz, tets, nodes)
    op = pkg.Operator(pkg.Geometry(surf.xyz, surf.tri), m=2, leaf=8)
    with pytest.raises(pkg.H2Error):   # tolerance must be positive
        F.solve(op, [0.0, 0.0, 1.0], tol=0.0)
    s3 = vm.boundary_surface(*vm.cube_tets(3))[0]
    op3 = pkg.Operator(pkg.Geometry(s3.xyz, s3.tri), m=2, leaf=8)
    with pytest.raises(pkg.H2Error):   # an operator on another surface
        F.solve(op3, [0.0, 0.0, 1.0])
