"""The full FEM/BEM pipeline of the method on small tetrahedral meshes.

TEST INFRASTRUCTURE ONLY (part of the oracle): plain numpy / scipy.sparse in
FP64; nothing on the product path imports it.

Section "Fredkin-Koehler method" of the paper splits the magnetostatic
potential as u = u1 + u2:

* u1 solves the Poisson problem Delta u1 = div M in the body (Eq. u1Poiss)
  with the Neumann data du1/dn = M.n (Eq. u1Neumann).  With P1 elements the
  weak form is  int grad u1 . grad v = int M . grad v  for every P1 function v
  (partial integration of both sides; the boundary terms are the Neumann data
  and cancel), made unique by a zero mean (one Lagrange multiplier).
* u2 is harmonic (Eq. u2diri); its boundary values follow from u1 on the
  boundary through the boundary integral equation (Eq. mainInt), i.e. the
  double-layer matrix M = K + D of ``dense_matrix`` applied to u1|boundary.
  The interior values solve the P1 Dirichlet problem with those values.
* H = -grad u, and the energy density in units of K_d = mu0 Ms^2 / 2 is
  e_d / K_d = (1/V) int M . grad u  (Section "Magnetostatic field and
  energy"); for a uniform unit M it is the demagnetising factor along M.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dense_matrix


def p1_gradients(xyz, tets):
    """Volumes (T,) and gradients (T, 4, 3) of the four barycentric functions."""
    p = np.asarray(xyz)[np.asarray(tets)]
    J = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=1)   # rows: edge vectors
    vol = np.linalg.det(J) / 6.0
    Jinv = np.linalg.inv(J)                     # columns: gradients of lambda_1..3
    g123 = np.transpose(Jinv, (0, 2, 1))
    g0 = -g123.sum(axis=1, keepdims=True)
    return vol, np.concatenate([g0, g123], axis=1)


def stiffness(xyz, tets):
    """Sparse P1 stiffness matrix  K_ab = int grad phi_a . grad phi_b."""
    vol, g = p1_gradients(xyz, tets)
    loc = vol[:, None, None] * np.einsum("tad,tbd->tab", g, g)
    rows = np.repeat(tets, 4, axis=1)
    cols = np.tile(tets, (1, 4))
    n = np.asarray(xyz).shape[0]
    return sp.csr_matrix((loc.reshape(-1), (rows.reshape(-1), cols.reshape(-1))), shape=(n, n)), vol, g


def solve_u1(xyz, tets, M):
    """P1 solution of the Neumann problem (zero mean); M: (3,) or (T, 3)."""
    K, vol, g = stiffness(xyz, tets)
    n = K.shape[0]
    Mt = np.broadcast_to(np.asarray(M, dtype=np.float64), (len(tets), 3))
    f = np.zeros(n)
    np.add.at(f, np.asarray(tets), vol[:, None] * np.einsum("tad,td->ta", g, Mt))
    c = np.zeros(n)
    np.add.at(c, np.asarray(tets), np.repeat(vol[:, None] / 4.0, 4, axis=1))
    A = sp.bmat([[K, sp.csr_matrix(c[:, None])], [sp.csr_matrix(c[None, :]), None]], format="csc")
    sol = spla.spsolve(A, np.concatenate([f, [0.0]]))
    return sol[:n]


def pipeline(xyz, tets, M, surface, surf_nodes):
    """u1, u2 and e_d / K_d for magnetisation M (uniform (3,) or per tet (T, 3)).

    ``surface``: the boundary as an outward surface mesh, ``surf_nodes``: the
    volume index of each of its nodes (``synth.volume.boundary_surface``)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets)
    u1 = solve_u1(xyz, tets, M)
    B = dense_matrix(surface.xyz, surface.tri)
    u2b = B @ u1[surf_nodes]
    K, vol, g = stiffness(xyz, tets)
    n = xyz.shape[0]
    interior = np.setdiff1d(np.arange(n), surf_nodes)
    u2 = np.zeros(n)
    u2[surf_nodes] = u2b
    KII = K[interior][:, interior].tocsc()
    KIB = K[interior][:, surf_nodes]
    u2[interior] = spla.spsolve(KII, -KIB @ u2b)
    u = u1 + u2
    Mt = np.broadcast_to(np.asarray(M, dtype=np.float64), (len(tets), 3))
    grad_u = np.einsum("ta,tad->td", u[tets], g)
    e = float(np.sum(vol * np.einsum("td,td->t", Mt, grad_u)) / np.sum(vol))
    return u1, u2, e
