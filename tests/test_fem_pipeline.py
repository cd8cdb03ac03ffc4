"""The oracle's full FEM/BEM pipeline (oracle/fem.py) on small tetrahedral meshes.

Pins (what the mathematics fixes):
* P1 elements reproduce linear functions, and for a uniform M the Neumann
  problem is solved by u1 = M.x (+ const): the computed u1 is that, to rounding;
* for P1 fields the volume energy (1/V) int M.grad u equals the boundary form
  (1/V) oint u M.n dS exactly (the divergence theorem holds tet by tet), so the
  pipeline and ``oracle.demag_factor`` agree to rounding;
* the cube's three factors are equal on a mesh symmetric under axis
  permutations and converge to 1/3; the ball's converge to 1/3 at second order
  (Section "Sphere": N = 1/3), and inside the ball u2 tends to -2/3 M.x.
"""
import numpy as np
import pytest

import oracle
from oracle import fem
from synth import volume as vm


def _run(gen, n, M):
    xyz, tets = gen(n)
    surf, nodes = vm.boundary_surface(xyz, tets)
    u1, u2, e = fem.pipeline(xyz, tets, np.asarray(M, dtype=np.float64), surf, nodes)
    return xyz, tets, surf, nodes, u1, u2, e


@pytest.mark.parametrize("M", [(0.0, 0.0, 1.0), (0.6, -0.48, 0.64)])
def test_neumann_solution_is_linear_for_uniform_m(M):
    xyz, tets = vm.ball_tets(5)
    u1 = fem.solve_u1(xyz, tets, np.asarray(M))
    lin = xyz @ np.asarray(M)
    d = u1 - lin
    assert np.ptp(d) < 1e-13


def test_volume_energy_equals_boundary_form():
    for gen, n in ((vm.cube_tets, 5), (vm.ball_tets, 6)):
        for M in ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0)):
            xyz, tets, surf, nodes, u1, u2, e = _run(gen, n, M)
            eb = oracle.demag_factor(surf.xyz, surf.tri, (u1 + u2)[nodes], M)
            assert abs(e - eb) < 1e-13, (gen.__name__, M, e, eb)


def test_cube_factors_equal_and_converge_to_one_third():
    errs = []
    for n in (3, 6, 12):
        Ns = [_run(vm.cube_tets, n, np.eye(3)[d])[-1] for d in range(3)]
        assert max(Ns) - min(Ns) < 1e-12, Ns
        errs.append(abs(Ns[0] - 1.0 / 3.0))
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5 and errs[2] < 4e-3, errs


def test_ball_factor_converges_at_second_order_and_u2_inside():
    errs, u2errs = [], []
    for n in (4, 8):
        xyz, tets, surf, nodes, u1, u2, e = _run(vm.ball_tets, n, (0.0, 0.0, 1.0))
        errs.append(abs(e - 1.0 / 3.0))
        inner = np.linalg.norm(xyz, axis=1) < 0.5
        u2errs.append(np.max(np.abs(u2[inner] - (u2[inner].mean() - 2.0 / 3.0 * (xyz[inner, 2] - xyz[inner, 2].mean())))))
    assert errs[1] < errs[0] / 3.5 and errs[1] < 4e-3, errs
    assert u2errs[1] < u2errs[0] and u2errs[1] < 2e-2, u2errs


def test_torus_azimuthal_energy_vanishes():
    """Section "Torus": a 2:1 solid torus magnetised azimuthally has neither
    volume nor surface charges, so e_d = 0.  With M piecewise constant (the
    azimuthal direction at each tetrahedron's centroid) the computed energy is
    a discretisation error that falls quickly under refinement, while a uniform
    M on the same meshes gives an O(1) energy."""
    es = []
    for nu, nc in ((12, 2), (24, 4), (36, 6)):
        xyz, tets = vm.torus_tets(nu, nc)
        surf, nodes = vm.boundary_surface(xyz, tets)
        e_tri = np.unique(np.sort(np.concatenate([surf.tri[:, [0, 1]], surf.tri[:, [1, 2]], surf.tri[:, [2, 0]]]),
                                  axis=1), axis=0)
        assert surf.n_vertices - len(e_tri) + surf.n_triangles == 0   # genus 1
        c = xyz[tets].mean(axis=1)
        phi = np.arctan2(c[:, 1], c[:, 0])
        M = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
        es.append(abs(fem.pipeline(xyz, tets, M, surf, nodes)[-1]))
        if nc == 4:
            ez = fem.pipeline(xyz, tets, np.array([0.0, 0.0, 1.0]), surf, nodes)[-1]
            assert 0.3 < ez < 0.7
    assert es[1] < es[0] / 5 and es[2] < es[1] / 3 and es[2] < 1e-6, es
