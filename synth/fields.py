"""Seeded right-hand sides u1 at the mesh nodes.

All randomness comes from numpy's PCG64 generator seeded explicitly, so the
oracle, the tests and the benchmark see identical inputs.
"""
from __future__ import annotations

import numpy as np

from .meshes import Mesh


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_rhs(n: int, r: int = 1, seed: int = 1811) -> np.ndarray:
    """u1 ~ N(0, 1) per node; shape (r, n)."""
    return rng(seed).standard_normal((r, n))


def uniform_rhs(n: int, r: int = 1, seed: int = 1811) -> np.ndarray:
    """u1 ~ U(-1, 1) per node; shape (r, n)."""
    return rng(seed).uniform(-1.0, 1.0, (r, n))


def vertex_normals(mesh: Mesh) -> np.ndarray:
    """Area-weighted mean of the adjacent triangle normals, normalised; shape (N, 3)."""
    p = mesh.xyz[mesh.tri]
    cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])  # 2 * area * unit normal
    vn = np.zeros_like(mesh.xyz)
    for a in range(3):
        np.add.at(vn, mesh.tri[:, a], cr)
    return vn / np.linalg.norm(vn, axis=1, keepdims=True)


def smooth_unit_field(xyz: np.ndarray, seed: int = 1811, n_modes: int = 8) -> np.ndarray:
    """Smooth unit vector field m(x) = normalise(sum_q a_q cos(2 pi f_q.x / L + phi_q)).

    a_q ~ N(0, I3), f_q ~ U[-2, 2]^3, phi_q ~ U[0, 2 pi), L = longest bounding-box side.
    """
    g = rng(seed)
    a = g.standard_normal((n_modes, 3))
    f = g.uniform(-2.0, 2.0, (n_modes, 3))
    ph = g.uniform(0.0, 2.0 * np.pi, n_modes)
    L = float(np.max(xyz.max(axis=0) - xyz.min(axis=0)))
    arg = 2.0 * np.pi * (xyz @ f.T) / L + ph[None, :]
    m = np.cos(arg) @ a
    nrm = np.linalg.norm(m, axis=1, keepdims=True)
    nrm[nrm == 0.0] = 1.0
    return m / nrm


def normal_dot_field(mesh: Mesh, seed: int = 1811) -> np.ndarray:
    """u1 = n . m at the nodes, for the vertex normal n and a seeded smooth unit field m; (1, N)."""
    n = vertex_normals(mesh)
    m = smooth_unit_field(mesh.xyz, seed)
    return np.sum(n * m, axis=1)[None, :]


def uniform_rhs_magnetisation(mesh: Mesh, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    """u1 = M . xi at the nodes for a uniform magnetisation M (the exact Neumann solution); (1, N)."""
    d = np.asarray(direction, dtype=np.float64)
    return (mesh.xyz @ d)[None, :]


def smooth_states(mesh: Mesh, r: int, seed: int = 1811) -> np.ndarray:
    """r right-hand sides u1 = n . m_c for r independently seeded smooth fields; (r, N)."""
    n = vertex_normals(mesh)
    out = np.empty((r, mesh.n_vertices))
    for c in range(r):
        out[c] = np.sum(n * smooth_unit_field(mesh.xyz, seed + 7919 * c), axis=1)
    return out
