"""Named synthetic workloads: a mesh, H2 parameters and seeded right-hand sides.

Parameters per workload (Chebyshev order m, leaf size, admissibility eta, number
of right-hand sides r) follow the benchmark configurations of the matvec:
icosphere level 3 (m=3, leaf 32), the 64 x 64-per-face cube (m=4, leaf 64), the
1000 x 1000 x 10 thin film (m=5, leaf 64), the 3:2:1 ellipsoid with 32
right-hand sides and the level-8 icosphere with 16 right-hand sides.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fields, meshes


@dataclass
class Workload:
    name: str
    mesh: meshes.Mesh
    m: int
    leaf: int
    eta: float
    u1: np.ndarray            # (r, N) float64
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def r(self) -> int:
        return int(self.u1.shape[0])


def _ico3(seed):
    m = meshes.icosphere(3)
    u = np.vstack([fields.gaussian_rhs(m.n_vertices, 1, seed), np.ones((1, m.n_vertices))])
    return Workload("ico3", m, 3, 32, 2.0, u, "icosphere level 3; u1 ~ N(0,1) plus all-ones")


def _cube64(seed):
    m = meshes.cube_surface(64)
    return Workload("cube64", m, 4, 64, 2.0, fields.normal_dot_field(m, seed),
                    "unit cube 64x64 per face; u1 = n.m for a seeded smooth unit field")


def _film(seed):
    m = meshes.film_box(320, 4)
    return Workload("film", m, 5, 64, 2.0, fields.uniform_rhs(m.n_vertices, 1, seed),
                    "1000x1000x10 film, 320x320 faces, 4 layers on the sides; u1 ~ U(-1,1)")


def _ellipsoid(seed, r=32):
    m = meshes.ellipsoid(7)
    return Workload("ellipsoid", m, 5, 64, 2.0, fields.smooth_states(m, r, seed),
                    f"icosphere level 7 scaled 3:2:1; {r} smooth states")


def _ico8(seed, r=16):
    m = meshes.icosphere(8)
    u = np.vstack([fields.uniform_rhs_magnetisation(m), fields.smooth_states(m, r - 1, seed)])
    return Workload("ico8", m, 5, 64, 2.0, u, f"icosphere level 8; u1 = z plus {r - 1} smooth states")


def multi_mesh_set():
    """The eight uneven meshes of the multi-mesh batch (5k-100k nodes)."""
    return [meshes.cube_surface(29), meshes.cube_surface(40), meshes.cube_surface(64),
            meshes.cube_surface(90), meshes.cube_surface(128), meshes.icosphere(5),
            meshes.icosphere(6), meshes.cube_sphere(70)]


WORKLOADS = {
    "ico3": _ico3,
    "cube64": _cube64,
    "film": _film,
    "ellipsoid": _ellipsoid,
    "ico8": _ico8,
}


def make_workload(name: str, seed: int = 1811, **kw) -> Workload:
    return WORKLOADS[name](seed, **kw)
