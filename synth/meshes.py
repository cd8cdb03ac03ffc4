"""Closed, outward-oriented triangle surface meshes used as seeded synthetic inputs.

Every mesh is a conforming, closed 2-manifold with counter-clockwise triangles
seen from outside, so that (r2 - r1) x (r3 - r1) points out of the body.  The
generators hold geometry only (vertex positions and connectivity); nothing in
this module evaluates the boundary operator.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    """Surface mesh: ``xyz`` (N, 3) float64 node positions, ``tri`` (T, 3) int32."""

    xyz: np.ndarray
    tri: np.ndarray
    name: str = ""

    @property
    def n_vertices(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_triangles(self) -> int:
        return int(self.tri.shape[0])

    def contiguous(self) -> "Mesh":
        return Mesh(np.ascontiguousarray(self.xyz, dtype=np.float64),
                    np.ascontiguousarray(self.tri, dtype=np.int32), self.name)


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def icosphere(level: int, radius: float = 1.0) -> Mesh:
    """Unit icosphere after ``level`` 4-way subdivisions (level 3: 642 nodes, 1280 triangles)."""
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(level):
        cache = {}
        new_f = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                p = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
                p = p / np.linalg.norm(p)
                verts.append(tuple(p))
                idx = len(verts) - 1
                cache[key] = idx
            return idx

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_f += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.asarray(new_f, dtype=np.int64)
    xyz = np.asarray(verts, dtype=np.float64) * radius
    return Mesh(xyz, f.astype(np.int32), f"icosphere{level}").contiguous()


def box_surface(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0,
                lz: float = 1.0, origin=(0.0, 0.0, 0.0)) -> Mesh:
    """Surface of an lx x ly x lz box with a structured nx x ny x nz grid on its faces.

    Each grid quad is split into two right triangles along the same diagonal.
    Nodes: 2(nx ny + ny nz + nz nx) + 2.
    """
    n = (nx, ny, nz)
    L = (lx, ly, lz)
    idx = -np.ones((nx + 1, ny + 1, nz + 1), dtype=np.int64)
    pts = []

    def node(i, j, k):
        if idx[i, j, k] < 0:
            idx[i, j, k] = len(pts)
            pts.append((origin[0] + lx * i / nx, origin[1] + ly * j / ny, origin[2] + lz * k / nz))
        return idx[i, j, k]

    tris = []
    for axis in range(3):
        u, v = [a for a in range(3) if a != axis]
        for side in (0, 1):
            # outward normal is +axis for side 1, -axis for side 0; e_u x e_v = +e_axis
            # for the cyclic pairs (x,y,z): (y,z)->x, (x,z)->-y, (x,y)->z.
            sign_uv = 1 if (axis, u, v) in ((0, 1, 2), (2, 0, 1)) else -1
            outward = 1 if side == 1 else -1
            flip = (sign_uv != outward)
            for a in range(n[u]):
                for b in range(n[v]):
                    def p(da, db):
                        c = [0, 0, 0]
                        c[axis] = n[axis] if side else 0
                        c[u] = a + da
                        c[v] = b + db
                        return node(*c)
                    p00, p10, p11, p01 = p(0, 0), p(1, 0), p(1, 1), p(0, 1)
                    if not flip:
                        tris += [[p00, p10, p11], [p00, p11, p01]]
                    else:
                        tris += [[p00, p11, p10], [p00, p01, p11]]
    del L
    return Mesh(np.asarray(pts, dtype=np.float64), np.asarray(tris, dtype=np.int32),
                f"box{nx}x{ny}x{nz}").contiguous()


def cube_surface(n: int, side: float = 1.0) -> Mesh:
    """Unit cube surface with an n x n grid per face (n = 64: 24,578 nodes)."""
    m = box_surface(n, n, n, side, side, side)
    m.name = f"cube{n}"
    return m


def film_box(nxy: int = 320, nz: int = 4, lxy: float = 1000.0, lz: float = 10.0) -> Mesh:
    """Thin-film box lxy x lxy x lz (default 1000 x 1000 x 10: 209,922 nodes)."""
    m = box_surface(nxy, nxy, nz, lxy, lxy, lz)
    m.name = f"film{nxy}x{nz}"
    return m


def cube_sphere(n: int, radius: float = 1.0) -> Mesh:
    """Cube surface (n x n per face, centred) projected radially onto a sphere."""
    m = box_surface(n, n, n, 2.0, 2.0, 2.0, origin=(-1.0, -1.0, -1.0))
    xyz = m.xyz / np.linalg.norm(m.xyz, axis=1, keepdims=True) * radius
    return Mesh(xyz, m.tri, f"cubesphere{n}").contiguous()


def ellipsoid(level: int, axes=(3.0, 2.0, 1.0)) -> Mesh:
    """Icosphere of the given level scaled to semi-axes ``axes``."""
    m = icosphere(level)
    xyz = m.xyz * np.asarray(axes, dtype=np.float64)[None, :]
    return Mesh(xyz, m.tri, f"ellipsoid{level}").contiguous()


def torus_surface(nu: int, nv: int, R: float = 2.0, r: float = 1.0) -> Mesh:
    """Torus of revolution about z (centre-line radius R, tube radius r; the
    default aspect ratio R : r = 2 : 1), an nu x nv grid in the angles u about
    z and v about the tube, each quad split into two triangles.  Genus 1, so
    it has saddle-shaped (non-convex) vertex fans on the inner side.
    Nodes: nu nv."""
    u = 2.0 * np.pi * np.arange(nu) / nu
    v = 2.0 * np.pi * np.arange(nv) / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    A = R + r * np.cos(V)
    xyz = np.stack([A * np.cos(U), A * np.sin(U), r * np.sin(V)], axis=-1).reshape(-1, 3)

    def node(i, j):
        return (i % nu) * nv + (j % nv)

    tris = []
    for i in range(nu):
        for j in range(nv):
            # d/du x d/dv points away from the tube's centre line (outward)
            p00, p10, p11, p01 = node(i, j), node(i + 1, j), node(i + 1, j + 1), node(i, j + 1)
            tris += [[p00, p10, p11], [p00, p11, p01]]
    return Mesh(xyz, np.asarray(tris, dtype=np.int32), f"torus{nu}x{nv}").contiguous()


def transformed(mesh: Mesh, rot: np.ndarray, shift, scale: float) -> Mesh:
    """Rigid motion plus uniform scaling x -> scale * rot @ x + shift (rot proper, det +1)."""
    xyz = scale * (mesh.xyz @ np.asarray(rot, dtype=np.float64).T) + np.asarray(shift)[None, :]
    return Mesh(xyz, mesh.tri.copy(), mesh.name + "_moved").contiguous()
