"""Seeded synthetic inputs: closed triangle surface meshes and right-hand sides.

This package is shared by the CPU oracle, the tests and the benchmark. It holds
none of the boundary-operator arithmetic: only mesh generators (icosphere, box
surfaces, mapped spheres, ellipsoids, tori), tetrahedral volume meshes of a
cube and a ball (``synth.volume``) and seeded vectors u1 at the nodes.
"""
from .meshes import (  # noqa: F401
    Mesh, icosphere, box_surface, cube_surface, cube_sphere, ellipsoid, film_box, torus_surface,
    transformed,
)
from .fields import (  # noqa: F401
    gaussian_rhs, uniform_rhs, smooth_unit_field, vertex_normals, normal_dot_field,
    uniform_rhs_magnetisation,
    smooth_states,
)
from .workloads import WORKLOADS, make_workload  # noqa: F401
