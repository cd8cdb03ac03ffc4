"""CPU oracle for the boundary double-layer operator and its H2 approximation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package.

The arithmetic lives in ``h2_oracle.c`` (plain C, FP64, OpenMP over rows),
compiled with gcc into ``oracle/_build``; this module marshals numpy arrays.
Equation names refer to arXiv:1811.05731.

* ``psi``: interior solid angle Psi at each node (Eq. mainInt); ``psi_at``
  at selected nodes only.
* ``lindholm``: corner weights of one triangle seen from one point (K entries,
  Eq. matrix_definition, Lindholm's closed form).
* ``dense_matrix`` / ``dense_matvec`` / ``dense_rows``: M = K + D (Eq. denseMat).
* ``H2Oracle``: cluster tree, block partition and the direct (non-nested)
  Chebyshev-interpolation H2 product (Section "H2-Matrix Compression").
* ``demag_factor``: e_d / K_d from boundary values of u = u1 + u2 for a
  uniform magnetisation (Section "Sphere": e_d = mu0 N Ms^2 / 2).
* ``recompress`` (module, numpy): algebraic recompression of the H2 far field
  (orthogonalised nested bases truncated with total cluster-basis weights),
  the reference for a recompressed product.
* ``fem`` (module, numpy / scipy.sparse): the full FEM/BEM pipeline on small
  tetrahedral meshes (P1 Neumann solve for u1, u2 on the boundary through the
  dense operator, P1 Dirichlet solve, volume energy).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h2_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march flags; the same source builds on x86 and Arm)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            L.o_solid_angle.restype = ctypes.c_double
            L.o_solid_angle.argtypes = [_d, _d, _d, _d]
            L.o_lindholm.argtypes = [_d, _d, _d, _d, _d]
            L.o_psi.argtypes = [ctypes.c_int64, _d, ctypes.c_int64, _i32, _d]
            L.o_psi_nodes.argtypes = [_d, ctypes.c_int64, _i32, ctypes.c_int64, _i64, _d]
            L.o_dense_matrix.argtypes = [ctypes.c_int64, _d, ctypes.c_int64, _i32, _d, _d]
            L.o_dense_rows.argtypes = [ctypes.c_int64, _d, ctypes.c_int64, _i32, _d,
                                       ctypes.c_int64, _i64, _d]
            L.o_dense_matvec.argtypes = [ctypes.c_int64, _d, ctypes.c_int64, _i32, _d,
                                         ctypes.c_int32, _d, _d]
            L.o_gauss_legendre01.argtypes = [ctypes.c_int, _d, _d]
            L.o_cheb_points.argtypes = [_d, ctypes.c_int, _d]
            L.o_lagrange3.argtypes = [_d, ctypes.c_int, _d, _d, _d]
            L.o_admissible.restype = ctypes.c_int
            L.o_admissible.argtypes = [_d, _d, ctypes.c_double]
            L.o2_create.restype = ctypes.c_void_p
            L.o2_create.argtypes = [ctypes.c_int64, _d, ctypes.c_int64, _i32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_int32]
            L.o2_info.argtypes = [ctypes.c_void_p, _i64]
            L.o2_get_tree.argtypes = [ctypes.c_void_p, _i32, _i32, _i32, _i32, _i32, _i32, _i32, _d]
            L.o2_get_blocks.argtypes = [ctypes.c_void_p, _i32, _i32, _i32, _i32]
            L.o2_get_psi.argtypes = [ctypes.c_void_p, _d]
            L.o2_cluster_bases.argtypes = [ctypes.c_void_p, ctypes.c_int32, _d, _d]
            L.o2_coupling.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _d]
            L.o2_matvec.argtypes = [ctypes.c_void_p, ctypes.c_int32, _d, _d]
            L.o2_rows.argtypes = [ctypes.c_void_p, ctypes.c_int32, _d, ctypes.c_int64, _i64, _d]
            L.o2_destroy.argtypes = [ctypes.c_void_p]
            L.o_num_threads.restype = ctypes.c_int
            _LIB = L
    return _LIB


def _pd(a):
    return a.ctypes.data_as(_d)


def _pi32(a):
    return a.ctypes.data_as(_i32)


def _pi64(a):
    return a.ctypes.data_as(_i64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_lib().o_num_threads())


def solid_angle(x, a, b, c) -> float:
    """Signed solid angle of triangle (a, b, c) seen from x (Van Oosterom-Strackee)."""
    x, a, b, c = (_f64(v) for v in (x, a, b, c))
    return float(_lib().o_solid_angle(_pd(x), _pd(a), _pd(b), _pd(c)))


def lindholm(x, r0, r1, r2) -> np.ndarray:
    """(1/4pi) int_T phi_a n.(x-y)/|x-y|^3 dS for the three corners a of T = (r0, r1, r2)."""
    out = np.zeros(3)
    x, r0, r1, r2 = (_f64(v) for v in (x, r0, r1, r2))
    _lib().o_lindholm(_pd(x), _pd(r0), _pd(r1), _pd(r2), _pd(out))
    return out


def psi(xyz, tri) -> np.ndarray:
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    out = np.zeros(xyz.shape[0])
    _lib().o_psi(xyz.shape[0], _pd(xyz), tri.shape[0], _pi32(tri), _pd(out))
    return out


def psi_at(xyz, tri, nodes) -> np.ndarray:
    """Psi at the given nodes only (NaN elsewhere): O(T) per node, for sampled rows of large meshes."""
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.full(xyz.shape[0], np.nan)
    _lib().o_psi_nodes(_pd(xyz), tri.shape[0], _pi32(tri), nodes.size, _pi64(nodes), _pd(out))
    return out


def dense_matrix(xyz, tri, psi_v=None) -> np.ndarray:
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    ps = psi(xyz, tri) if psi_v is None else _f64(psi_v)
    n = xyz.shape[0]
    M = np.zeros((n, n))
    _lib().o_dense_matrix(n, _pd(xyz), tri.shape[0], _pi32(tri), _pd(ps), _pd(M))
    return M


def dense_rows(xyz, tri, rows, psi_v=None) -> np.ndarray:
    """Rows of M at the given nodes (Psi is needed at those nodes only)."""
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    ps = psi_at(xyz, tri, rows) if psi_v is None else _f64(psi_v)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((rows.size, xyz.shape[0]))
    _lib().o_dense_rows(xyz.shape[0], _pd(xyz), tri.shape[0], _pi32(tri), _pd(ps),
                        rows.size, _pi64(rows), _pd(out))
    return out


def dense_matvec(xyz, tri, x, psi_v=None) -> np.ndarray:
    """y = M x with x of shape (r, N) (rows of M rebuilt on the fly)."""
    xyz = _f64(xyz)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    ps = psi(xyz, tri) if psi_v is None else _f64(psi_v)
    x = _f64(np.atleast_2d(x))
    y = np.zeros_like(x)
    _lib().o_dense_matvec(xyz.shape[0], _pd(xyz), tri.shape[0], _pi32(tri), _pd(ps),
                          x.shape[0], _pd(x), _pd(y))
    return y


def gauss_legendre01(q: int):
    x = np.zeros(q)
    w = np.zeros(q)
    _lib().o_gauss_legendre01(q, _pd(x), _pd(w))
    return x, w


def cheb_points(box, m: int) -> np.ndarray:
    box = _f64(box)
    out = np.zeros((m ** 3, 3))
    _lib().o_cheb_points(_pd(box), m, _pd(out))
    return out


def lagrange3(box, m: int, x):
    """(L_nu(x), grad L_nu(x)) for the tensor Chebyshev basis of ``box``."""
    box, x = _f64(box), _f64(x)
    v = np.zeros(m ** 3)
    g = np.zeros((m ** 3, 3))
    _lib().o_lagrange3(_pd(box), m, _pd(x), _pd(v), _pd(g))
    return v, g


def admissible(box_t, box_s, eta: float) -> bool:
    return bool(_lib().o_admissible(_pd(_f64(box_t)), _pd(_f64(box_s)), float(eta)))


class H2Oracle:
    """Direct interpolation H2 approximation of M (cluster tree, blocks, V_t S_ts W_s^T).

    ``store=True`` keeps near blocks and direct bases for repeated products;
    ``store=False`` is for sampled rows of large meshes (``rows``).
    """

    def __init__(self, xyz, tri, m: int, leaf: int, eta: float = 2.0, rho: float = 0.25,
                 q: int = 0, store: bool = True):
        L = _lib()
        self.xyz = _f64(xyz)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.N = self.xyz.shape[0]
        self.m, self.leaf, self.eta, self.rho = m, leaf, eta, rho
        self._h = L.o2_create(self.N, _pd(self.xyz), self.tri.shape[0], _pi32(self.tri), m, leaf,
                              float(eta), float(rho), q, 1 if store else 0)
        info = np.zeros(8, dtype=np.int64)
        L.o2_info(self._h, _pi64(info))
        (self.n_clusters, self.n_levels, self.n_far, self.n_near, self.near_entries,
         self.far_coefficients, self.k, self.q) = (int(v) for v in info)

    def close(self):
        if getattr(self, "_h", None):
            _lib().o2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tree(self) -> dict:
        nc = self.n_clusters
        out = {k: np.zeros(nc, dtype=np.int32) for k in
               ("start", "size", "parent", "child0", "child1", "level")}
        perm = np.zeros(self.N, dtype=np.int32)
        box = np.zeros((nc, 6))
        _lib().o2_get_tree(self._h, _pi32(perm), _pi32(out["start"]), _pi32(out["size"]),
                           _pi32(out["parent"]), _pi32(out["child0"]), _pi32(out["child1"]),
                           _pi32(out["level"]), _pd(box))
        out["perm"] = perm
        out["box"] = box
        return out

    def blocks(self) -> dict:
        ft = np.zeros(self.n_far, dtype=np.int32)
        fs = np.zeros(self.n_far, dtype=np.int32)
        nt = np.zeros(self.n_near, dtype=np.int32)
        ns = np.zeros(self.n_near, dtype=np.int32)
        _lib().o2_get_blocks(self._h, _pi32(ft), _pi32(fs), _pi32(nt), _pi32(ns))
        return {"far_t": ft, "far_s": fs, "near_t": nt, "near_s": ns}

    def psi(self) -> np.ndarray:
        """Psi at every node (``store=False``: only at nodes already sampled by ``rows``, NaN elsewhere)."""
        out = np.zeros(self.N)
        _lib().o2_get_psi(self._h, _pd(out))
        return out

    def cluster_bases(self, c: int, size: int):
        V = np.zeros((size, self.k))
        W = np.zeros((size, self.k))
        _lib().o2_cluster_bases(self._h, int(c), _pd(V), _pd(W))
        return V, W

    def coupling(self, t: int, s: int) -> np.ndarray:
        S = np.zeros((self.k, self.k))
        _lib().o2_coupling(self._h, int(t), int(s), _pd(S))
        return S

    def matvec(self, x) -> np.ndarray:
        x = _f64(np.atleast_2d(x))
        y = np.zeros_like(x)
        _lib().o2_matvec(self._h, x.shape[0], _pd(x), _pd(y))
        return y

    def rows(self, x, rows) -> np.ndarray:
        """(H2 x)[:, rows] for x of shape (r, N); near entries and bases built on the fly."""
        x = _f64(np.atleast_2d(x))
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((x.shape[0], rows.size))
        _lib().o2_rows(self._h, x.shape[0], _pd(x), rows.size, _pi64(rows), _pd(out))
        return out


def triangle_normals_areas(xyz, tri):
    p = np.asarray(xyz)[np.asarray(tri)]
    cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    a2 = np.linalg.norm(cr, axis=1)
    return cr / a2[:, None], 0.5 * a2


def enclosed_volume(xyz, tri) -> float:
    """V = sum_T r_a . (r_b x r_c) / 6 (divergence theorem on the closed polyhedron)."""
    p = np.asarray(xyz)[np.asarray(tri)]
    return float(np.sum(np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2]))) / 6.0)


def demag_factor(xyz, tri, u, direction=(0.0, 0.0, 1.0)) -> float:
    """e_d / K_d = (1/V) oint u (M.n) dS for unit uniform magnetisation M along ``direction``.

    E = (mu0/2) int M.grad u dV = (mu0/2) oint u M.n dS for uniform M, so with
    K_d = mu0 Ms^2/2 the ratio is the demagnetising factor N (1/3 for a sphere).
    u is linear on each flat triangle, so its integral is A (u_a + u_b + u_c)/3.
    """
    n, A = triangle_normals_areas(xyz, tri)
    mn = n @ np.asarray(direction, dtype=np.float64)
    uu = np.asarray(u)[np.asarray(tri)].sum(axis=1) / 3.0
    return float(np.sum(mn * A * uu) / enclosed_volume(xyz, tri))
