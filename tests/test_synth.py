"""The synthetic input recipe: mesh sizes of the benchmark configurations,
closed outward surfaces, and seeded right-hand sides that repeat exactly."""
import numpy as np
import pytest

import oracle
import synth

SIZES = {   # nodes, triangles
    "ico3": (642, 1280),
    "cube64": (24578, 49152),
    "film": (209922, 419840),
    "ellipsoid": (163842, 327680),
    "ico8": (655362, 1310720),
}


def _edges(tri):
    e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    return np.unique(e, axis=0)


@pytest.mark.parametrize("name", sorted(SIZES))
def test_workload_sizes_and_closed_outward_surface(name):
    w = synth.make_workload(name)
    n, t = SIZES[name]
    assert (w.mesh.n_vertices, w.mesh.n_triangles) == (n, t)
    # a closed genus-0 surface: V - E + F = 2, every edge in two triangles
    e = _edges(w.mesh.tri)
    assert n - len(e) + t == 2
    assert 2 * len(e) == 3 * t
    assert oracle.enclosed_volume(w.mesh.xyz, w.mesh.tri) > 0.0   # outward orientation
    assert np.all(np.isfinite(w.u1)) and w.u1.shape[1] == n


@pytest.mark.parametrize("name", ["ico3", "cube64"])
def test_seeded_inputs_repeat_and_depend_on_the_seed(name):
    a, b = synth.make_workload(name), synth.make_workload(name)
    assert np.array_equal(a.u1, b.u1) and np.array_equal(a.mesh.xyz, b.mesh.xyz)
    c = synth.make_workload(name, seed=7)
    assert not np.array_equal(a.u1, c.u1)


def test_smooth_states_are_normal_components_of_unit_fields():
    m = synth.cube_surface(8)
    u = synth.smooth_states(m, 4, 5)
    assert u.shape == (4, m.n_vertices)
    assert np.all(np.abs(u) <= 1.0 + 1e-12)        # n . m with |n| = |m| = 1
    assert np.linalg.matrix_rank(u) == 4             # independent states


def test_eight_uneven_meshes():
    ms = synth.workloads.multi_mesh_set()
    sizes = [m.n_vertices for m in ms]
    assert len(ms) == 8 and sum(sizes) == 266742
    assert min(sizes) >= 5000 and max(sizes) <= 100000


def test_torus_is_a_closed_outward_genus_one_surface():
    """The torus used for the zero-energy pin: V - E + F = 0 (genus 1), every
    edge in two triangles, each directed edge once (consistent orientation),
    and an enclosed volume that converges to 2 pi^2 R r^2 from below."""
    vols = []
    for nu, nv in ((24, 12), (48, 24), (96, 48)):
        m = synth.torus_surface(nu, nv)
        e = _edges(m.tri)
        assert m.n_vertices - len(e) + m.n_triangles == 0
        assert 2 * len(e) == 3 * m.n_triangles
        d = np.concatenate([m.tri[:, [0, 1]], m.tri[:, [1, 2]], m.tri[:, [2, 0]]])
        assert len(np.unique(d, axis=0)) == len(d)
        vols.append(oracle.enclosed_volume(m.xyz, m.tri))
    exact = 2.0 * np.pi ** 2 * 2.0 * 1.0
    assert 0.0 < vols[0] < vols[1] < vols[2] < exact
    assert (exact - vols[2]) / exact < 5e-3


@pytest.mark.parametrize("which,n", [("cube", 4), ("ball", 6)])
def test_volume_meshes_and_their_boundaries(which, n):
    """Tetrahedral meshes of the full-pipeline checks: every tetrahedron
    positively oriented, volumes summing to the body's, and a boundary that is
    a closed genus-0 surface, outward, enclosing the same volume."""
    from synth import volume as vm
    xyz, tets = vm.cube_tets(n) if which == "cube" else vm.ball_tets(n)
    p = xyz[tets]
    vol = np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0])) / 6.0
    assert np.all(vol > 0)
    surf, nodes = vm.boundary_surface(xyz, tets)
    e = _edges(surf.tri)
    assert surf.n_vertices - len(e) + surf.n_triangles == 2 and 2 * len(e) == 3 * surf.n_triangles
    assert abs(oracle.enclosed_volume(surf.xyz, surf.tri) - vol.sum()) < 1e-12 * vol.sum()
    if which == "cube":
        assert abs(vol.sum() - 1.0) < 1e-12
    else:
        assert np.allclose(np.linalg.norm(surf.xyz, axis=1), 1.0)
