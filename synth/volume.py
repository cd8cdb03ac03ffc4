"""Tetrahedral volume meshes for the full-pipeline checks (geometry only).

* ``cube_tets``: the cube [0, side]^3 on an n^3 grid, every cell split into the
  six tetrahedra around its main diagonal (Kuhn's split: one tetrahedron per
  ordering of the axes), so the mesh is conforming and symmetric under any
  permutation of the axes.
* ``ball_tets``: the same grid on [-1, 1]^3 mapped radially onto the unit
  ball (x -> x |x|_inf / |x|_2), which sends the cube's surface onto the sphere.
* ``torus_tets``: a solid torus of revolution, the same split of a
  (tube disc x angle) grid.
* ``boundary_surface``: the faces that belong to one tetrahedron only, oriented
  outward, as a surface ``Mesh`` plus the volume index of every surface node.

Nothing here evaluates an operator.
"""
from __future__ import annotations

import itertools

import numpy as np

from .meshes import Mesh


def _grid(n: int, lo: float, hi: float) -> np.ndarray:
    g = np.linspace(lo, hi, n + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X, Y, Z], axis=-1).reshape(-1, 3)


def _kuhn_tets(n: int) -> np.ndarray:
    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    tets = []
    for i, j, k in itertools.product(range(n), repeat=3):
        for perm in itertools.permutations(range(3)):
            p = [i, j, k]
            verts = [vid(*p)]
            for ax in perm:
                p[ax] += 1
                verts.append(vid(*p))
            tets.append(verts)
    tets = np.asarray(tets, dtype=np.int64)
    return tets


def _orient(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Every tetrahedron with a positive signed volume."""
    p = xyz[tets]
    vol = np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]))
    tets = tets.copy()
    neg = vol < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3], tets[neg, 2].copy()
    return tets


def cube_tets(n: int, side: float = 1.0):
    """(xyz (N, 3), tets (T, 4)) of the cube [0, side]^3, n cells per edge."""
    xyz = _grid(n, 0.0, side)
    return xyz, _orient(xyz, _kuhn_tets(n))


def ball_tets(n: int):
    """(xyz, tets) of the unit ball: the [-1, 1]^3 grid mapped radially."""
    xyz = _grid(n, -1.0, 1.0)
    r2 = np.linalg.norm(xyz, axis=1)
    rinf = np.max(np.abs(xyz), axis=1)
    scale = np.where(r2 > 0, rinf / np.where(r2 > 0, r2, 1.0), 0.0)
    xyz = xyz * scale[:, None]
    return xyz, _orient(xyz, _kuhn_tets(n))


def torus_tets(nu: int, nc: int, R: float = 2.0, r: float = 1.0):
    """(xyz, tets) of the solid torus of revolution about z (centre-line radius
    R, tube radius r): an nc x nc grid on [-1, 1]^2 mapped radially onto the
    tube's disc, swept over nu angles about z (periodic), each cell of the
    (disc, angle) grid split into six tetrahedra like ``cube_tets``."""
    g = np.linspace(-1.0, 1.0, nc + 1)
    A, B = np.meshgrid(g, g, indexing="ij")
    ab = np.stack([A.ravel(), B.ravel()], axis=1)
    r2 = np.linalg.norm(ab, axis=1)
    rinf = np.max(np.abs(ab), axis=1)
    ab = ab * np.where(r2 > 0, rinf / np.where(r2 > 0, r2, 1.0), 0.0)[:, None]
    u = 2.0 * np.pi * np.arange(nu) / nu
    rho = R + r * ab[:, 0]
    xyz = np.stack([np.outer(np.cos(u), rho), np.outer(np.sin(u), rho),
                    np.broadcast_to(r * ab[:, 1], (nu, ab.shape[0]))], axis=-1).reshape(-1, 3)
    m = nc + 1

    def vid(i, j, k):
        return (k % nu) * m * m + i * m + j

    tets = []
    for i, j, k in itertools.product(range(nc), range(nc), range(nu)):
        for perm in itertools.permutations(range(3)):
            p = [i, j, k]
            verts = [vid(*p)]
            for ax in perm:
                p[ax] += 1
                verts.append(vid(*p))
            tets.append(verts)
    return xyz, _orient(xyz, np.asarray(tets, dtype=np.int64))


def boundary_surface(xyz: np.ndarray, tets: np.ndarray):
    """(surface Mesh, volume index of each surface node) of a tetrahedral mesh."""
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 3, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 1]]])
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    outer = faces[cnt[inv.ravel()] == 1]
    # (a, b, c) above is ordered so that its normal points away from the
    # tetrahedron's fourth vertex for a positively oriented tetrahedron
    nodes = np.unique(outer)
    local = -np.ones(xyz.shape[0], dtype=np.int64)
    local[nodes] = np.arange(nodes.size)
    mesh = Mesh(xyz[nodes], local[outer].astype(np.int32), "boundary").contiguous()
    return mesh, nodes
