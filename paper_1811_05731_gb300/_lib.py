"""ctypes binding of libh2bem (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import lib_path

FP64 = 0
FP32 = 1
TF32X3 = 2
BF16X3 = 3
SCHEDULE_FLOW = 0
SCHEDULE_LEVELS = 1
COUPLING_STORED = 0
COUPLING_ON_THE_FLY = 1
NEAR_FP64 = 0
NEAR_F32PAIR = 1

_LIB = None
_LOCK = threading.Lock()
_c_d = ctypes.POINTER(ctypes.c_double)
_c_i32 = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


class H2Error(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {h2_error_string(code)} ({code})"
        try:
            extra = lib().h2_last_error_message().decode()
            if extra:
                msg += f": {extra}"
        except Exception:
            pass
        super().__init__(msg)


class Params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("leaf", ctypes.c_int32), ("eta", ctypes.c_double),
                ("box_inflation", ctypes.c_double), ("precision", ctypes.c_int32),
                ("max_rhs", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("coupling", ctypes.c_int32), ("near_field", ctypes.c_int32),
                ("recompress_eps", ctypes.c_double)]


class PlanReport(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("n_far_blocks", ctypes.c_int64), ("n_near_blocks", ctypes.c_int64),
                ("n_segments", ctypes.c_int64), ("n_chunks", ctypes.c_int64),
                ("n_split_segments", ctypes.c_int64), ("n_regions", ctypes.c_int32),
                ("violations", ctypes.c_int32), ("bytes_streamed", ctypes.c_int64),
                ("makespan_us", ctypes.c_double), ("split_makespan_us", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("stages", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("n_candidates", ctypes.c_int32), ("ms_best", ctypes.c_double), ("ms_default", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("n_clusters", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("n_leaves", ctypes.c_int32), ("k", ctypes.c_int32),
                ("n_far_blocks", ctypes.c_int64), ("n_near_blocks", ctypes.c_int64),
                ("near_entries", ctypes.c_int64), ("far_coefficients", ctypes.c_int64),
                ("basis_coefficients", ctypes.c_int64), ("bytes_far", ctypes.c_int64),
                ("bytes_near", ctypes.c_int64), ("bytes_streamed", ctypes.c_int64),
                ("macs_per_rhs", ctypes.c_int64), ("compression_ratio", ctypes.c_double),
                ("assemble_seconds", ctypes.c_double), ("precision", ctypes.c_int32),
                ("max_rhs", ctypes.c_int32), ("n_launches_matvec", ctypes.c_int32),
                ("n_passes", ctypes.c_int32), ("bytes_near_pair", ctypes.c_int64),
                ("near_field", ctypes.c_int32), ("coupling", ctypes.c_int32),
                ("recompress_eps", ctypes.c_double), ("mean_rank_row", ctypes.c_double),
                ("mean_rank_col", ctypes.c_double), ("max_rank", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def load(path: str | None = None):
    """Load libh2bem (built by :func:`paper_1811_05731_gb300.build`); raises if absent."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        p = path or lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"libh2bem is not built ({p}); run paper_1811_05731_gb300.build()")
        L = ctypes.CDLL(p)
        L.h2_default_params.argtypes = [ctypes.POINTER(Params)]
        L.h2_default_params.restype = None
        L.h2_error_string.argtypes = [ctypes.c_int]
        L.h2_error_string.restype = ctypes.c_char_p
        L.h2_last_error_message.argtypes = []
        L.h2_last_error_message.restype = ctypes.c_char_p
        L.h2_build_geometry.argtypes = [_c_d, ctypes.c_int64, _c_i32, ctypes.c_int64, _vp,
                                        ctypes.POINTER(_vp)]
        L.h2_assemble.argtypes = [_vp, ctypes.POINTER(Params), ctypes.POINTER(_vp)]
        L.h2_matvec.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _vp]
        L.h2_matvec_noalloc.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _vp]
        L.h2_matvec_batched.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp),
                                        ctypes.POINTER(_vp), _c_i32, _vp]
        L.h2_autotune.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.POINTER(Tuning)]
        L.h2_fault_inject_stall.argtypes = [_vp, ctypes.c_int32]
        L.h2_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
        L.h2_get_tree.argtypes = [_vp] + [_c_i32] * 7 + [_c_d]
        L.h2_get_blocks.argtypes = [_vp] + [_c_i32] * 4
        L.h2_get_psi.argtypes = [_vp, _c_d]
        L.h2_device_status.argtypes = [_vp]
        L.h2_free.argtypes = [_vp]
        L.h2_plan_check.argtypes = [_c_d, ctypes.c_int64, _c_i32, ctypes.c_int64, ctypes.POINTER(Params),
                                    ctypes.c_int32, ctypes.POINTER(PlanReport)]
        L.h2_fem_create.argtypes = [_c_d, ctypes.c_int64, _c_i32, ctypes.c_int64, _c_i32, ctypes.c_int64,
                                    ctypes.POINTER(_vp)]
        L.h2_fem_solve.argtypes = [_vp] * 5 + [ctypes.c_double, ctypes.c_int32, _vp, ctypes.c_void_p]
        for f in ("h2_build_geometry", "h2_assemble", "h2_matvec", "h2_matvec_noalloc", "h2_matvec_batched",
                  "h2_autotune", "h2_fault_inject_stall",
                  "h2_stats", "h2_get_tree",
                  "h2_get_blocks", "h2_get_psi", "h2_device_status", "h2_free", "h2_plan_check",
                  "h2_fem_create", "h2_fem_solve"):
            getattr(L, f).restype = ctypes.c_int
        _LIB = L
        return L


def lib():
    return load()


def h2_error_string(code: int) -> str:
    return lib().h2_error_string(int(code)).decode()


def _check(code: int, where: str):
    if code != 0:
        raise H2Error(code, where)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def h2_default_params(**kw) -> Params:
    p = Params()
    lib().h2_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "rho":
            k = "box_inflation"
        setattr(p, k, v)
    return p


def h2_build_geometry(xyz, tri, stream=None) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    h = _vp()
    _check(lib().h2_build_geometry(xyz.ctypes.data_as(_c_d), xyz.shape[0], tri.ctypes.data_as(_c_i32),
                                   tri.shape[0], _stream_ptr(stream), ctypes.byref(h)),
           "h2_build_geometry")
    return h.value


def h2_assemble(geom: int, params: Params | None = None) -> int:
    h = _vp()
    _check(lib().h2_assemble(geom, ctypes.byref(params) if params is not None else None,
                             ctypes.byref(h)), "h2_assemble")
    return h.value


def h2_matvec(op: int, u1_ptr: int, u2_ptr: int, r: int, stream=None) -> None:
    """u2 = M u1 on raw pointers (both device or both host), r x N row-major FP64."""
    _check(lib().h2_matvec(op, u1_ptr, u2_ptr, int(r), _stream_ptr(stream) if stream != 0 else 0),
           "h2_matvec")


def h2_matvec_noalloc(op: int, u1_ptr: int, u2_ptr: int, r: int, stream=None) -> None:
    """u2 = M u1 on device pointers with the library's fixed scratch (no device allocation)."""
    _check(lib().h2_matvec_noalloc(op, u1_ptr, u2_ptr, int(r), _stream_ptr(stream)),
           "h2_matvec_noalloc")


def h2_autotune(op: int, r: int, stream=None) -> dict:
    """Times the launch configurations of an operator's product and keeps the fastest."""
    t = Tuning()
    _check(lib().h2_autotune(op, int(r), _stream_ptr(stream), ctypes.byref(t)), "h2_autotune")
    return t.as_dict()


def h2_matvec_batched(ops, u1_ptrs, u2_ptrs, rs, stream=None) -> None:
    """u2_i = M_i u1_i for several operators in one persistent launch (device pointers)."""
    n = len(ops)
    arr = lambda xs: (_vp * n)(*[_vp(int(x)) for x in xs])
    rr = (ctypes.c_int32 * n)(*[int(x) for x in rs])
    _check(lib().h2_matvec_batched(arr(ops), n, arr(u1_ptrs), arr(u2_ptrs), rr, _stream_ptr(stream)),
           "h2_matvec_batched")


def matvec_batched(operators, xs, ys=None, stream=None):
    """Batched product of ``Operator`` objects on torch CUDA tensors ``xs`` (each (r_i, N_i))."""
    import torch
    xs = [x if x.dim() == 2 else x.unsqueeze(0) for x in xs]
    ys = ys if ys is not None else [torch.empty_like(x) for x in xs]
    h2_matvec_batched([o.handle for o in operators], [x.data_ptr() for x in xs], [y.data_ptr() for y in ys],
                      [x.shape[0] for x in xs], stream)
    return ys


def h2_plan_check(xyz, tri, workers: int = 456, **params) -> dict:
    """Host-only build and check of the execution plan (no GPU needed); see
    h2_plan_check in h2bem.h.  ``params`` as for :func:`h2_default_params`."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    p = h2_default_params(**params)
    rep = PlanReport()
    _check(lib().h2_plan_check(xyz.ctypes.data_as(_c_d), xyz.shape[0], tri.ctypes.data_as(_c_i32), tri.shape[0],
                               ctypes.byref(p), int(workers), ctypes.byref(rep)), "h2_plan_check")
    return rep.as_dict()


def h2_stats(op: int) -> dict:
    s = Stats()
    _check(lib().h2_stats(op, ctypes.byref(s)), "h2_stats")
    return s.as_dict()


def h2_get_tree(op: int) -> dict:
    st = h2_stats(op)
    nc, N = st["n_clusters"], st["n_vertices"]
    out = {k: np.zeros(nc, dtype=np.int32) for k in ("start", "size", "parent", "child0", "child1", "level")}
    perm = np.zeros(N, dtype=np.int32)
    box = np.zeros((nc, 6))
    p = lambda a: a.ctypes.data_as(_c_i32)  # noqa: E731
    _check(lib().h2_get_tree(op, p(perm), p(out["start"]), p(out["size"]), p(out["parent"]),
                             p(out["child0"]), p(out["child1"]), p(out["level"]),
                             box.ctypes.data_as(_c_d)), "h2_get_tree")
    out["perm"] = perm
    out["box"] = box
    return out


def h2_get_blocks(op: int) -> dict:
    st = h2_stats(op)
    nf, nn = st["n_far_blocks"], st["n_near_blocks"]
    out = {"far_t": np.zeros(nf, np.int32), "far_s": np.zeros(nf, np.int32),
           "near_t": np.zeros(nn, np.int32), "near_s": np.zeros(nn, np.int32)}
    p = lambda a: a.ctypes.data_as(_c_i32)  # noqa: E731
    _check(lib().h2_get_blocks(op, p(out["far_t"]), p(out["far_s"]), p(out["near_t"]),
                               p(out["near_s"])), "h2_get_blocks")
    return out


def h2_get_psi(h: int, n: int) -> np.ndarray:
    out = np.zeros(n)
    _check(lib().h2_get_psi(h, out.ctypes.data_as(_c_d)), "h2_get_psi")
    return out


def h2_device_status(op: int) -> int:
    return int(lib().h2_device_status(op))


def h2_free(h: int) -> None:
    if h:
        _check(lib().h2_free(h), "h2_free")


class Geometry:
    """Closed, outward-oriented triangle surface mesh on the GPU."""

    def __init__(self, xyz, tri, stream=None):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.N = int(self.xyz.shape[0])
        self.handle = h2_build_geometry(self.xyz, self.tri, stream)

    def psi(self) -> np.ndarray:
        return h2_get_psi(self.handle, self.N)

    def close(self):
        if getattr(self, "handle", None):
            h2_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """H2 approximation of M = K + D on one GPU."""

    def __init__(self, geom: Geometry, m: int = 4, leaf: int = 64, eta: float = 2.0,
                 rho: float = 0.25, precision: int = FP64, max_rhs: int = 1,
                 schedule: int = SCHEDULE_FLOW, autotune: bool = False,
                 coupling: int = COUPLING_STORED, near_field: int = NEAR_FP64, recompress_eps: float = 0.0):
        self.geom = geom
        self.N = geom.N
        self.params = h2_default_params(m=m, leaf=leaf, eta=eta, box_inflation=rho,
                                        precision=precision, max_rhs=max_rhs, schedule=schedule,
                                        autotune=1 if autotune else 0, coupling=coupling,
                                        near_field=near_field, recompress_eps=float(recompress_eps))
        self.handle = h2_assemble(geom.handle, self.params)

    def autotune(self, r: int | None = None, stream=None) -> dict:
        """Picks the fastest launch configuration for products of r right-hand sides."""
        return h2_autotune(self.handle, r or self.params.max_rhs, stream)

    def stats(self) -> dict:
        return h2_stats(self.handle)

    def tree(self) -> dict:
        return h2_get_tree(self.handle)

    def blocks(self) -> dict:
        return h2_get_blocks(self.handle)

    def matvec(self, u1, u2=None, stream=None):
        """u2 = M u1.  ``u1`` is a (r, N) or (N,) FP64 torch CUDA tensor or numpy array.

        Torch tensors stay on the device (asynchronous on ``stream``); numpy
        arrays go through the library's synchronous host-pointer path.
        """
        if isinstance(u1, np.ndarray):
            x = np.ascontiguousarray(np.atleast_2d(u1), dtype=np.float64)
            y = np.empty_like(x) if u2 is None else u2
            h2_matvec(self.handle, x.ctypes.data, y.ctypes.data, x.shape[0], stream)
            return y if u1.ndim == 2 else y[0]
        import torch
        if u1.dtype != torch.float64 or not u1.is_cuda or not u1.is_contiguous():
            raise ValueError("u1 must be a contiguous float64 CUDA tensor")
        x = u1 if u1.dim() == 2 else u1.view(1, -1)
        if x.shape[1] != self.N:
            raise ValueError(f"u1 has {x.shape[1]} columns, the mesh has {self.N} nodes")
        y = torch.empty_like(x) if u2 is None else u2.view(x.shape)
        h2_matvec(self.handle, x.data_ptr(), y.data_ptr(), x.shape[0], stream)
        return y if u1.dim() == 2 else y.view(-1)

    def close(self):
        if getattr(self, "handle", None):
            h2_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FemReport(ctypes.Structure):
    _fields_ = [("iters_u1", ctypes.c_int32), ("iters_u2", ctypes.c_int32), ("resid_u1", ctypes.c_double),
                ("resid_u2", ctypes.c_double), ("energy", ctypes.c_double), ("volume", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def h2_fem_create(xyz, tets, surf_nodes) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    surf = np.ascontiguousarray(surf_nodes, dtype=np.int32)
    h = _vp()
    _check(lib().h2_fem_create(xyz.ctypes.data_as(_c_d), xyz.shape[0], tets.ctypes.data_as(_c_i32), tets.shape[0],
                               surf.ctypes.data_as(_c_i32), surf.shape[0], ctypes.byref(h)), "h2_fem_create")
    return h.value


def h2_fem_solve(fem: int, op: int, M_ptr: int, u1_ptr: int, u2_ptr: int, tol: float, max_iter: int,
                 stream=None) -> dict:
    rep = FemReport()
    _check(lib().h2_fem_solve(fem, op, M_ptr, u1_ptr, u2_ptr, float(tol), int(max_iter), _stream_ptr(stream),
                              ctypes.byref(rep)), "h2_fem_solve")
    return rep.as_dict()


class Fem:
    """Tetrahedral mesh of the magnetic body (P1 elements) on the GPU, with its
    boundary surface given as the volume index of every surface node."""

    def __init__(self, xyz, tets, surf_nodes):
        self.nv = int(np.asarray(xyz).shape[0])
        self.nt = int(np.asarray(tets).shape[0])
        self.handle = h2_fem_create(xyz, tets, surf_nodes)

    def solve(self, op: "Operator", M, tol: float = 1e-12, max_iter: int = 5000, stream=None):
        """(u1, u2, report) for the magnetisation M: a (3,) vector (uniform) or
        an (n_tets, 3) array, numpy or a torch CUDA tensor."""
        import torch
        Mt = torch.as_tensor(np.broadcast_to(np.asarray(M, dtype=np.float64), (self.nt, 3)).copy()
                             if not isinstance(M, torch.Tensor) else M, dtype=torch.float64).cuda().contiguous()
        u1 = torch.empty(self.nv, dtype=torch.float64, device="cuda")
        u2 = torch.empty_like(u1)
        rep = h2_fem_solve(self.handle, op.handle, Mt.data_ptr(), u1.data_ptr(), u2.data_ptr(), tol, max_iter,
                           stream)
        return u1, u2, rep

    def close(self):
        if getattr(self, "handle", None):
            h2_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
