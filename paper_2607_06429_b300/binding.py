"""Thin ctypes binding of libvsie (argument marshalling only; every step of the operator
runs in the library's CUDA kernels).  Names follow the C ABI in include/vsie.h.

Device vectors are torch.complex128 CUDA tensors; a block of right-hand sides has shape
(nrhs, n), which in memory is the column-major n x nrhs layout the library expects.
There is no CPU fallback: if the library or a CUDA device is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvsie.so")

STATUS = {
    0: "VSIE_OK", 1: "VSIE_ERR_ARG", 2: "VSIE_ERR_MESH", 3: "VSIE_ERR_CUDA", 4: "VSIE_ERR_OOM",
    5: "VSIE_ERR_NOT_CONVERGED", 6: "VSIE_ERR_BREAKDOWN", 7: "VSIE_ERR_NAN",
}
VSIE_ERR_NOT_CONVERGED = 5

EXPORTS = ("vsie_create", "vsie_destroy", "vsie_sizes", "vsie_apply", "vsie_apply_host",
           "vsie_apply_timed", "vsie_apply_noalloc", "vsie_apply_batched",
           "vsie_adjoint_apply", "vsie_plane_wave_rhs", "vsie_far_field", "vsie_solve",
           "vsie_far_field_adjoint", "vsie_solve_batched", "vsie_apply_batched_multi",
           "vsie_graph_create_batched", "vsie_graph_launch", "vsie_graph_nodes", "vsie_graph_destroy",
           "vsie_autotune", "vsie_get_tuning", "vsie_set_tuning", "vsie_gradient_channels", "vsie_source_points",
           "vsie_lsq_grad_alpha", "vsie_lsq_grad_alpha_adjoint", "vsie_scattered_field",
           "vsie_create_cuboid", "vsie_set_frequency", "vsie_cuboid_faces", "vsie_apply_rows",
           "vsie_pipe_probe", "vsie_last_error", "vsie_bem_create", "vsie_bem_destroy", "vsie_bem_sizes",
           "vsie_bem_apply", "vsie_bem_rhs", "vsie_bem_solve", "vsie_bem_far_field")


class VsieError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Mesh(ctypes.Structure):
    _fields_ = [("n_vert", ctypes.c_int64), ("vert", ctypes.c_void_p),
                ("n_tet", ctypes.c_int64), ("tet", ctypes.c_void_p),
                ("n_tri", ctypes.c_int64), ("tri", ctypes.c_void_p)]


class _Material(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("c0", ctypes.c_double),
                ("rho", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("grad_alpha", ctypes.c_void_p), ("tri_rho_in", ctypes.c_void_p),
                ("tri_rho_out", ctypes.c_void_p)]


class _CuboidGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("x_edges", ctypes.c_void_p), ("y_edges", ctypes.c_void_p), ("z_edges", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("tet_far_points", ctypes.c_int32), ("near_radius", ctypes.c_double),
                ("tri_near_radius", ctypes.c_double), ("tile_override", ctypes.c_int32),
                ("debug_flags", ctypes.c_int32)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("max_refinements", ctypes.c_int32),
                ("adjoint", ctypes.c_int32), ("initial_guess", ctypes.c_int32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("far_chunk", ctypes.c_int32 * 3), ("far_blocks_per_sm", ctypes.c_int32 * 3),
                ("far_ms", ctypes.c_double * 3), ("far_default_ms", ctypes.c_double * 3),
                ("batch_chunk_tiles", ctypes.c_int32), ("batch_ms", ctypes.c_double),
                ("batch_default_ms", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("gk_blocks_per_sm", ctypes.c_int32 * 2), ("gk_ms", ctypes.c_double),
                ("gk_sequential_ms", ctypes.c_double)]


class _BemDesc(ctypes.Structure):
    _fields_ = [("n_interfaces", ctypes.c_int32), ("h_vert", ctypes.c_void_p * 2), ("h_tri", ctypes.c_void_p * 2),
                ("n_vert", ctypes.c_int64 * 2), ("n_tri", ctypes.c_int64 * 2), ("k0", ctypes.c_double),
                ("rho0", ctypes.c_double), ("c0", ctypes.c_double), ("rho", ctypes.c_double * 2),
                ("c", ctypes.c_double * 2), ("far_order", ctypes.c_int32), ("near_order", ctypes.c_int32),
                ("near_factor", ctypes.c_double)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("fp64_applies", ctypes.c_int32),
                ("fp32_applies", ctypes.c_int32)]


@dataclass
class SolveInfo:
    status: int
    iterations: int
    refinements: int
    rel_residual: float
    fp64_applies: int
    fp32_applies: int


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libvsie.so (built in-tree by ``paper_2607_06429_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libvsie.so not found at {path}; run paper_2607_06429_b300/build.py")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.vsie_create.argtypes = [ctypes.POINTER(_Mesh), ctypes.POINTER(_Material), D,
                                ctypes.POINTER(_Options), ctypes.POINTER(P)]
    lib.vsie_destroy.argtypes = [P]
    lib.vsie_destroy.restype = None
    lib.vsie_sizes.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.vsie_apply.argtypes = [P, P, P, I32, I32, P]
    lib.vsie_apply_host.argtypes = [P, P, P, I32, I32, P]
    lib.vsie_apply_rows.argtypes = [P, P, P, I64, I64, I32, P]
    lib.vsie_pipe_probe.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P]
    lib.vsie_apply_noalloc.argtypes = [P, P, P, I32, I32, P]
    lib.vsie_apply_batched.argtypes = [P, P, P, I32, I32, P]
    lib.vsie_adjoint_apply.argtypes = [P, P, P, I32, I32, P]
    lib.vsie_apply_timed.argtypes = [P, P, P, I32, P, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(I32)]
    lib.vsie_plane_wave_rhs.argtypes = [P, P, I32, P, P]
    lib.vsie_far_field.argtypes = [P, P, I32, P, I32, P, P]
    lib.vsie_far_field_adjoint.argtypes = [P, P, I32, P, I32, P, P]
    lib.vsie_scattered_field.argtypes = [P, P, I32, P, I64, I32, P, P]
    lib.vsie_create_cuboid.argtypes = [ctypes.POINTER(_CuboidGrid), P, P, D, D, D, ctypes.POINTER(P)]
    lib.vsie_set_frequency.argtypes = [P, D]
    lib.vsie_cuboid_faces.argtypes = [ctypes.POINTER(_CuboidGrid), P, D, I64, ctypes.POINTER(I64), P, P, P, P, P]
    lib.vsie_solve.argtypes = [P, P, P, ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveInfo), P]
    lib.vsie_solve_batched.argtypes = [P, P, P, ctypes.c_int32, ctypes.POINTER(_SolveOpts),
                                       ctypes.POINTER(_SolveInfo), P]
    lib.vsie_apply_batched_multi.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(P), ctypes.POINTER(P),
                                             I32, P]
    lib.vsie_graph_create_batched.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(P), ctypes.POINTER(P),
                                              I32, ctypes.POINTER(P)]
    lib.vsie_graph_launch.argtypes = [P, P]
    lib.vsie_autotune.argtypes = [P, I32, ctypes.POINTER(_Tuning), P]
    lib.vsie_get_tuning.argtypes = [P, ctypes.POINTER(_Tuning)]
    lib.vsie_set_tuning.argtypes = [P, ctypes.POINTER(_Tuning)]
    lib.vsie_gradient_channels.argtypes = [P, P, I32, P, P, P]
    lib.vsie_source_points.argtypes = [P, P, P, P]
    lib.vsie_lsq_grad_alpha.argtypes = [ctypes.POINTER(_Mesh), P, P, P]
    lib.vsie_lsq_grad_alpha_adjoint.argtypes = [ctypes.POINTER(_Mesh), P, P, P]
    lib.vsie_graph_nodes.argtypes = [P, ctypes.POINTER(I64)]
    lib.vsie_graph_destroy.argtypes = [P]
    lib.vsie_graph_destroy.restype = None
    lib.vsie_bem_create.argtypes = [ctypes.POINTER(_BemDesc), ctypes.POINTER(P)]
    lib.vsie_bem_destroy.argtypes = [P]
    lib.vsie_bem_destroy.restype = None
    lib.vsie_bem_sizes.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.vsie_bem_apply.argtypes = [P, P, P, I32, P]
    lib.vsie_bem_rhs.argtypes = [P, P, P, P]
    lib.vsie_bem_solve.argtypes = [P, P, P, ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveInfo), P]
    lib.vsie_bem_far_field.argtypes = [P, P, P, I32, P, P]
    lib.vsie_last_error.argtypes = []
    lib.vsie_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("vsie_destroy", "vsie_last_error", "vsie_graph_destroy", "vsie_bem_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, allow=()):
    if status != 0 and status not in allow:
        raise VsieError(status, _lib.vsie_last_error().decode())
    return status


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a CUDA complex128 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Operator:
    """The discretised nested VSIE operator on the current CUDA device (vsie_create)."""

    def __init__(self, vert, tet, tri, rho, c, tri_rho_in, tri_rho_out, k0, rho0=1.0, c0=1.0,
                 grad_alpha=None, tet_far_points=1, near_radius=0.0, tri_near_radius=0.0,
                 tile_override=0, debug_flags=0):
        lib = load_library()
        self._keep = dict(vert=_f64(vert).reshape(-1), tet=_i32(tet).reshape(-1),
                          tri=_i32(tri).reshape(-1), rho=_f64(rho), c=_f64(c),
                          ga=None if grad_alpha is None else _f64(grad_alpha).reshape(-1),
                          rin=_f64(tri_rho_in), rout=_f64(tri_rho_out))
        k = self._keep
        mesh = _Mesh(k["vert"].shape[0] // 3, _ptr(k["vert"]), k["tet"].shape[0] // 4,
                     _ptr(k["tet"]), k["tri"].shape[0] // 3, _ptr(k["tri"]))
        mat = _Material(float(rho0), float(c0), _ptr(k["rho"]), _ptr(k["c"]), _ptr(k["ga"]),
                        _ptr(k["rin"]), _ptr(k["rout"]))
        opt = _Options(int(tet_far_points), float(near_radius), float(tri_near_radius),
                       int(tile_override), int(debug_flags))
        h = ctypes.c_void_p()
        _check(lib.vsie_create(ctypes.byref(mesh), ctypes.byref(mat), float(k0),
                               ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self._keep = None
        n, nf, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.vsie_sizes(h, ctypes.byref(n), ctypes.byref(nf), ctypes.byref(nnz)))
        self.n, self.n_far_sources, self.nnz = n.value, nf.value, nnz.value
        self.k0 = float(k0)

    @classmethod
    def from_workload(cls, w, **kw):
        ga = w.grad_alpha
        if getattr(w, "grad_alpha_lsq", False):
            ga = lsq_grad_alpha(w.vert, w.tet, w.tet_domain, w.rho0 / np.asarray(w.rho) - 1.0)
        return cls(w.vert, w.tet, w.tri, w.rho, w.c, w.tri_rho_in, w.tri_rho_out, w.k0,
                   w.rho0, w.c0, ga, w.tet_far_points, w.near_radius,
                   w.tri_near_radius, **kw)

    @classmethod
    def from_cuboid(cls, w):
        """The paper's cuboid discretisation of a CuboidWorkload (vsie_create_cuboid)."""
        lib = load_library()
        ex, ey, ez = (_f64(e) for e in (w.x_edges, w.y_edges, w.z_edges))
        rho, c = _f64(np.asarray(w.rho).reshape(-1)), _f64(np.asarray(w.c).reshape(-1))
        grid = _CuboidGrid(ex.shape[0] - 1, ey.shape[0] - 1, ez.shape[0] - 1, _ptr(ex), _ptr(ey), _ptr(ez))
        h = ctypes.c_void_p()
        _check(lib.vsie_create_cuboid(ctypes.byref(grid), _ptr(rho), _ptr(c), float(w.rho0), float(w.c0),
                                      float(w.k0), ctypes.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        self._keep = None
        n, nf, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.vsie_sizes(h, ctypes.byref(n), ctypes.byref(nf), ctypes.byref(nnz)))
        self.n, self.n_far_sources, self.nnz = n.value, nf.value, nnz.value
        self.k0 = float(w.k0)
        return self

    def set_frequency(self, k0):
        """Rebuild the operator for a new k0 (vsie_set_frequency)."""
        _check(_lib.vsie_set_frequency(self._h, float(k0)))
        self.k0 = float(k0)

    def close(self):
        if getattr(self, "_h", None):
            _lib.vsie_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def _nrhs(self, x):
        if x.dim() == 1:
            if x.shape[0] != self.n:
                raise ValueError("vector length must equal n")
            return 1
        if x.dim() != 2 or x.shape[1] != self.n:
            raise ValueError("blocks must have shape (nrhs, n)")
        return x.shape[0]

    def apply(self, x, y=None, precision=32, stream=None):
        """y = A x  (vsie_apply)."""
        import torch
        nrhs = self._nrhs(x)
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.vsie_apply(self._h, _dev(x, "x"), _dev(y, "y"), nrhs, int(precision),
                               _stream(stream)))
        return y

    def apply_rows(self, x, row_begin, row_end, y=None, precision=32, stream=None):
        """Rows row_begin .. row_end-1 of A x (vsie_apply_rows): x has all n unknowns, y the
        (row_end - row_begin) rows."""
        import torch
        if x.dim() != 1 or x.shape[0] != self.n:
            raise ValueError("x must have shape (n,)")
        m = int(row_end) - int(row_begin)
        if y is None:
            y = torch.empty(max(m, 0), dtype=x.dtype, device=x.device)
        elif y.dim() != 1 or y.shape[0] != m:
            raise ValueError("y must have shape (row_end - row_begin,)")
        if m == 0 and 0 <= int(row_begin) <= self.n:
            return y  # nothing to compute (an empty tensor has no device address to pass)
        _check(_lib.vsie_apply_rows(self._h, _dev(x, "x"), _dev(y, "y"), int(row_begin), int(row_end),
                                    int(precision), _stream(stream)))
        return y

    def apply_batched(self, x, y=None, precision=32, stream=None):
        """Y = A X for a block (nrhs, n) with the multi-RHS far field (vsie_apply_batched):
        precision 32 on the tensor cores, 64 in FP64 on the CUDA cores."""
        import torch
        nrhs = self._nrhs(x)
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.vsie_apply_batched(self._h, _dev(x, "x"), _dev(y, "y"), nrhs, int(precision),
                                       _stream(stream)))
        return y

    def source_points(self):
        """(positions (n_far, 3), owners (n_far,), classes (n_far,)) of the far-field source
        points in the library's order (vsie_source_points)."""
        xyz = np.empty((self.n_far_sources, 3), dtype=np.float64)
        own = np.empty(self.n_far_sources, dtype=np.int32)
        cls = np.empty(self.n_far_sources, dtype=np.int32)
        _check(_lib.vsie_source_points(self._h, _ptr(xyz), _ptr(own), _ptr(cls)))
        return xyz, own, cls

    def gradient_channels(self, lam, precision=64, stream=None):
        """(phi (n_far,), psi (n_far, 3)) of an adjoint state lam (vsie_gradient_channels)."""
        import torch
        if lam.dim() != 1 or lam.shape[0] != self.n:
            raise ValueError("lam must have shape (n,)")
        phi = torch.empty(self.n_far_sources, dtype=torch.complex128, device=lam.device)
        psi = torch.empty((self.n_far_sources, 3), dtype=torch.complex128, device=lam.device)
        _check(_lib.vsie_gradient_channels(self._h, _dev(lam, "lam"), int(precision), _dev(phi, "phi"),
                                           _dev(psi, "psi"), _stream(stream)))
        return phi, psi

    def get_tuning(self):
        """The work shapes in use (vsie_get_tuning), 0 where the built-in default applies."""
        t = _Tuning()
        _check(_lib.vsie_get_tuning(self._h, ctypes.byref(t)))
        return {"far_chunk": list(t.far_chunk), "far_blocks_per_sm": list(t.far_blocks_per_sm),
                "batch_chunk_tiles": t.batch_chunk_tiles, "gk_blocks_per_sm": list(t.gk_blocks_per_sm)}

    def set_tuning(self, far_chunk=(0, 0, 0), far_blocks_per_sm=(0, 0, 0), batch_chunk_tiles=0,
                   gk_blocks_per_sm=(0, 0)):
        """Set the work shapes without timing them (vsie_set_tuning); takes get_tuning()'s
        keys."""
        t = _Tuning()
        for i in range(3):
            t.far_chunk[i] = int(far_chunk[i])
            t.far_blocks_per_sm[i] = int(far_blocks_per_sm[i])
        t.batch_chunk_tiles = int(batch_chunk_tiles)
        t.gk_blocks_per_sm[0], t.gk_blocks_per_sm[1] = (int(v) for v in gk_blocks_per_sm)
        _check(_lib.vsie_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, far=True, batched=True, stream=None):
        """Time candidate work shapes on this operator and keep the fastest (vsie_autotune);
        returns the report as a dict."""
        flags = (1 if far else 0) | (2 if batched else 0)
        t = _Tuning()
        _check(_lib.vsie_autotune(self._h, flags, ctypes.byref(t), _stream(stream)))
        cls = ("G", "K", "F")
        return {"far": {c: {"chunk": t.far_chunk[i], "blocks_per_sm": t.far_blocks_per_sm[i],
                            "ms": t.far_ms[i], "default_ms": t.far_default_ms[i]}
                        for i, c in enumerate(cls) if t.far_chunk[i]} if far else None,
                "concurrent_gk": {"blocks_per_sm": list(t.gk_blocks_per_sm), "ms": t.gk_ms,
                                  "sequential_ms": t.gk_sequential_ms} if far else None,
                "batched": {"chunk_tiles": t.batch_chunk_tiles, "ms": t.batch_ms,
                            "default_ms": t.batch_default_ms} if batched else None,
                "candidates": t.candidates}

    def apply_noalloc(self, x, y, precision=32, stream=None):
        """y = A x without any device allocation in the call (vsie_apply_noalloc); the
        caller provides y."""
        nrhs = self._nrhs(x)
        _check(_lib.vsie_apply_noalloc(self._h, _dev(x, "x"), _dev(y, "y"), nrhs,
                                       int(precision), _stream(stream)))
        return y

    def apply_timed(self, x, y, precision=32, stream=None):
        """One apply with per-phase device times (vsie_apply_timed).  Returns
        (dict of ms per phase, number of kernel launches)."""
        ms = (ctypes.c_double * 4)()
        nl = ctypes.c_int32()
        _check(_lib.vsie_apply_timed(self._h, _dev(x, "x"), _dev(y, "y"), int(precision),
                                     _stream(stream), ms, ctypes.byref(nl)))
        names = ("prescale", "far_volume", "far_vector", "correction")
        return dict(zip(names, list(ms))), nl.value

    def apply_host(self, x: np.ndarray, precision=32, stream=None) -> np.ndarray:
        """y = A x with host buffers (vsie_apply_host); x complex128 (n,) or (nrhs, n)."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        nrhs = 1 if x.ndim == 1 else x.shape[0]
        y = np.empty_like(x)
        _check(_lib.vsie_apply_host(self._h, _ptr(x), _ptr(y), nrhs, int(precision),
                                    _stream(stream)))
        return y

    def apply_host_ptr(self, x_ptr: int, y_ptr: int, nrhs=1, precision=32, stream=None):
        """vsie_apply_host on raw (e.g. pinned) host pointers."""
        _check(_lib.vsie_apply_host(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                    int(nrhs), int(precision), _stream(stream)))

    def adjoint_apply(self, y, x=None, precision=32, stream=None):
        """x = A^H y  (vsie_adjoint_apply)."""
        import torch
        nrhs = self._nrhs(y)
        if x is None:
            x = torch.empty_like(y)
        _check(_lib.vsie_adjoint_apply(self._h, _dev(y, "y"), _dev(x, "x"), nrhs,
                                       int(precision), _stream(stream)))
        return x

    def plane_wave_rhs(self, dirs, stream=None):
        """b[d] = exp(i k0 x . d)  (vsie_plane_wave_rhs); returns (ndir, n)."""
        import torch
        d = _f64(dirs).reshape(-1, 3)
        b = torch.empty((d.shape[0], self.n), dtype=torch.complex128, device="cuda")
        _check(_lib.vsie_plane_wave_rhs(self._h, _ptr(d), d.shape[0], _dev(b, "b"),
                                        _stream(stream)))
        return b

    def far_field(self, p, dirs, stream=None):
        """Far-field pattern (vsie_far_field); returns (nrhs, ndir) or (ndir,)."""
        import torch
        nrhs = self._nrhs(p)
        d = _f64(dirs).reshape(-1, 3)
        out = torch.empty((nrhs, d.shape[0]), dtype=torch.complex128, device="cuda")
        _check(_lib.vsie_far_field(self._h, _dev(p, "p"), nrhs, _ptr(d), d.shape[0],
                                   _dev(out, "out"), _stream(stream)))
        return out[0] if p.dim() == 1 else out

    def scattered_field(self, p, points, precision=64, stream=None):
        """Scattered field p_s = p - p_inc at points outside the scatterer
        (vsie_scattered_field); p: (n,) or (nrhs, n), points: (m, 3); returns (m,) or
        (nrhs, m)."""
        import torch
        nrhs = self._nrhs(p)
        X = _f64(points).reshape(-1, 3)
        out = torch.empty((nrhs, X.shape[0]), dtype=torch.complex128, device="cuda")
        _check(_lib.vsie_scattered_field(self._h, _dev(p, "p"), nrhs, _ptr(X), X.shape[0], int(precision),
                                         _dev(out, "out"), _stream(stream)))
        return out[0] if p.dim() == 1 else out

    def far_field_adjoint(self, r, dirs, stream=None):
        """x = F^H r for the far-field map F (vsie_far_field_adjoint); r: (ndir,) or
        (nrhs, ndir); returns (n,) or (nrhs, n)."""
        import torch
        d = _f64(dirs).reshape(-1, 3)
        rr = r if r.dim() == 2 else r[None]
        if rr.shape[1] != d.shape[0]:
            raise ValueError("r must have one entry per direction")
        x = torch.empty((rr.shape[0], self.n), dtype=torch.complex128, device="cuda")
        _check(_lib.vsie_far_field_adjoint(self._h, _dev(rr.contiguous(), "r"), rr.shape[0], _ptr(d),
                                           d.shape[0], _dev(x, "x"), _stream(stream)))
        return x[0] if r.dim() == 1 else x

    def solve_batched(self, b, mode=32, tol=1e-8, max_iters=1000, restart=0, inner_tol=1e-4,
                      max_refinements=20, stream=None, raise_on_fail=True):
        """X with A X[c] = B[c] for a block B (nrhs, n), every column its own GMRES, the
        operator applications shared (vsie_solve_batched); returns (X, [SolveInfo])."""
        import torch
        nrhs = self._nrhs(b)
        x = torch.empty_like(b)
        o = _SolveOpts(int(mode), float(tol), int(max_iters), int(restart), float(inner_tol),
                       int(max_refinements), 0)
        infos = (_SolveInfo * nrhs)()
        st = _lib.vsie_solve_batched(self._h, _dev(b, "b"), _dev(x, "x"), nrhs, ctypes.byref(o),
                                     infos, _stream(stream))
        if raise_on_fail:
            _check(st)
        return x, [SolveInfo(st, i.iterations, i.refinements, i.rel_residual, i.fp64_applies,
                             i.fp32_applies) for i in infos]

    def solve(self, b, mode=32, tol=1e-8, max_iters=1000, restart=0, inner_tol=1e-4,
              max_refinements=20, stream=None, raise_on_fail=True, adjoint=False, x0=None):
        """x with A x = b, or A^H x = b if adjoint (vsie_solve); returns (x, SolveInfo).
        x0: a starting iterate (resume from a saved solution), copied, not modified."""
        import torch
        if b.dim() != 1:
            raise ValueError("vsie_solve takes one right-hand side")
        if x0 is not None:
            if tuple(x0.shape) != tuple(b.shape):
                raise ValueError("x0 must have the shape of b")
            x = x0.to(device=b.device, dtype=torch.complex128).clone()
        else:
            x = torch.empty_like(b)
        o = _SolveOpts(int(mode), float(tol), int(max_iters), int(restart), float(inner_tol),
                       int(max_refinements), 1 if adjoint else 0, 0 if x0 is None else 1)
        info = _SolveInfo()
        st = _lib.vsie_solve(self._h, _dev(b, "b"), _dev(x, "x"), ctypes.byref(o),
                             ctypes.byref(info), _stream(stream))
        if raise_on_fail:
            _check(st)
        return x, SolveInfo(st, info.iterations, info.refinements, info.rel_residual,
                            info.fp64_applies, info.fp32_applies)


class BemOperator:
    """The nested PMCHWT boundary element operator (vsie_bem_*): P1 Galerkin on one or two
    nested closed triangulated interfaces (outermost first), unknowns [u_1, v_1, u_2, v_2]
    at the vertices, rows scaled by the lumped mass."""

    def __init__(self, surfaces, k0, rho, c, rho0=1.0, c0=1.0, far_order=3, near_order=4, near_factor=2.0):
        load_library()
        if len(surfaces) not in (1, 2) or len(rho) != len(surfaces) or len(c) != len(surfaces):
            raise ValueError("one or two interfaces, with one (rho, c) per layer")
        self._keep = []
        d = _BemDesc()
        d.n_interfaces = len(surfaces)
        for m, (v, t) in enumerate(surfaces):
            v, t = _f64(v), _i32(t)
            self._keep += [v, t]
            d.h_vert[m] = v.ctypes.data
            d.h_tri[m] = t.ctypes.data
            d.n_vert[m] = v.shape[0]
            d.n_tri[m] = t.shape[0]
            d.rho[m] = float(rho[m])
            d.c[m] = float(c[m])
        d.k0, d.rho0, d.c0 = float(k0), float(rho0), float(c0)
        d.far_order, d.near_order, d.near_factor = int(far_order), int(near_order), float(near_factor)
        self._h = ctypes.c_void_p()
        _check(_lib.vsie_bem_create(ctypes.byref(d), ctypes.byref(self._h)))
        self._keep = None
        n, q, nn = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.vsie_bem_sizes(self._h, ctypes.byref(n), ctypes.byref(q), ctypes.byref(nn)))
        self.n, self.n_points, self.n_near_pairs = n.value, q.value, nn.value

    @classmethod
    def nested_spheres(cls, subdiv, radii, k0, rho, c, rho0=1.0, c0=1.0, **kw):
        """Concentric icosphere interfaces (workloads.icosphere)."""
        from .workloads import icosphere
        subdiv = [subdiv] * len(radii) if np.isscalar(subdiv) else list(subdiv)
        return cls([icosphere(sd, R) for sd, R in zip(subdiv, radii)], k0, rho, c, rho0, c0, **kw)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.vsie_bem_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x, y=None, precision=32, stream=None):
        """y = P A x (vsie_bem_apply); x: CUDA complex128 (n,); precision 32, 48 (double-float)
        or 64."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.vsie_bem_apply(self._h, _dev(x, "x"), _dev(y, "y"), int(precision), _stream(stream)))
        return y

    def rhs(self, direction, device="cuda", stream=None):
        """P (int phi p_inc, int phi (1/rho0) dp_inc/dn) for the plane wave along direction."""
        import torch
        b = torch.empty(self.n, dtype=torch.complex128, device=device)
        d = _f64(direction)
        _check(_lib.vsie_bem_rhs(self._h, _ptr(d), _dev(b, "b"), _stream(stream)))
        return b

    def solve(self, b, mode=32, tol=1e-8, max_iters=1000, restart=0, inner_tol=1e-4, max_refinements=20,
              stream=None, raise_on_fail=True):
        """x with P A x = P b (vsie_bem_solve); returns (x, SolveInfo)."""
        import torch
        x = torch.empty_like(b)
        o = _SolveOpts(int(mode), float(tol), int(max_iters), int(restart), float(inner_tol),
                       int(max_refinements), 0, 0)
        info = _SolveInfo()
        st = _lib.vsie_bem_solve(self._h, _dev(b, "b"), _dev(x, "x"), ctypes.byref(o), ctypes.byref(info),
                                 _stream(stream))
        if raise_on_fail:
            _check(st)
        return x, SolveInfo(st, info.iterations, info.refinements, info.rel_residual, info.fp64_applies,
                            info.fp32_applies)

    def far_field(self, x, dirs, stream=None):
        """Far-field pattern on the unit directions dirs (m, 3) (vsie_bem_far_field)."""
        import torch
        dirs = _f64(dirs).reshape(-1, 3)
        out = torch.empty(dirs.shape[0], dtype=torch.complex128, device=x.device)
        _check(_lib.vsie_bem_far_field(self._h, _dev(x, "x"), _ptr(dirs), dirs.shape[0], _dev(out, "out"),
                                       _stream(stream)))
        return out


def pipe_probe(stream=None):
    """Sustained issue rates per clock and per SM of the pipes the far-field sums use
    (vsie_pipe_probe), measured on the current device, with the SM clock seen."""
    load_library()
    r = (ctypes.c_double * 5)()
    mhz = ctypes.c_double()
    _check(_lib.vsie_pipe_probe(r, ctypes.byref(mhz), _stream(stream)))
    names = ("mufu_rsqrt", "mufu_sin", "ffma", "ffma2_fma_ops", "dfma")
    out = {k: float(v) for k, v in zip(names, r)}
    out["sm_mhz"] = float(mhz.value)
    return out


def _multi_arrays(ops, xs, ys):
    if len(ops) != len(xs) or len(ops) != len(ys) or not ops:
        raise ValueError("one input and one output block per operator")
    nrhs = ops[0]._nrhs(xs[0])
    for op, x, y in zip(ops, xs, ys):
        if op._nrhs(x) != nrhs or tuple(y.shape) != tuple(x.shape):
            raise ValueError("every block must have shape (nrhs, n) with the same nrhs")
    P = ctypes.c_void_p
    hs = (P * len(ops))(*[op._h for op in ops])
    xa = (P * len(ops))(*[_dev(x, "x") for x in xs])
    ya = (P * len(ops))(*[_dev(y, "y") for y in ys])
    return hs, xa, ya, nrhs


def apply_batched_multi(ops, xs, ys=None, stream=None):
    """ys[p] = A_p xs[p] for operators of one mesh (e.g. several frequencies), with one
    persistent tensor-core launch per source class for all of them (vsie_apply_batched_multi)."""
    import torch
    if ys is None:
        ys = [torch.empty_like(x) for x in xs]
    hs, xa, ya, nrhs = _multi_arrays(ops, xs, ys)
    _check(_lib.vsie_apply_batched_multi(hs, len(ops), xa, ya, nrhs, _stream(stream)))
    return ys


class BatchedGraph:
    """A CUDA-graph plan of apply_batched_multi for fixed operators and blocks
    (vsie_graph_create_batched); ``launch()`` replays it (vsie_graph_launch)."""

    def __init__(self, ops, xs, ys):
        hs, xa, ya, nrhs = _multi_arrays(ops, xs, ys)
        self._keep = (list(ops), list(xs), list(ys))  # the plan holds their device pointers
        g = ctypes.c_void_p()
        _check(_lib.vsie_graph_create_batched(hs, len(ops), xa, ya, nrhs, ctypes.byref(g)))
        self._g = g

    @property
    def nodes(self) -> int:
        n = ctypes.c_int64()
        _check(_lib.vsie_graph_nodes(self._g, ctypes.byref(n)))
        return n.value

    def launch(self, stream=None):
        _check(_lib.vsie_graph_launch(self._g, _stream(stream)))

    def close(self):
        if getattr(self, "_g", None) is not None and self._g.value:
            _lib.vsie_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tet_mesh(vert, tet):
    v = _f64(vert).reshape(-1)
    t = _i32(tet).reshape(-1)
    return _Mesh(v.shape[0] // 3, _ptr(v), t.shape[0] // 4, _ptr(t), 0, None), (v, t)


def cuboid_faces(w):
    """The interface unknowns of a CuboidWorkload in their unknown order (vsie_cuboid_faces):
    dict of centres (m, 3), axis (m,), area, omega and mass (m,)."""
    lib = load_library()
    ex, ey, ez = (_f64(e) for e in (w.x_edges, w.y_edges, w.z_edges))
    rho = _f64(np.asarray(w.rho).reshape(-1))
    grid = _CuboidGrid(ex.shape[0] - 1, ey.shape[0] - 1, ez.shape[0] - 1, _ptr(ex), _ptr(ey), _ptr(ez))
    cnt = ctypes.c_int64()
    _check(lib.vsie_cuboid_faces(ctypes.byref(grid), _ptr(rho), float(w.rho0), 0, ctypes.byref(cnt),
                                 None, None, None, None, None))
    m = cnt.value
    out = dict(centres=np.empty((m, 3)), axis=np.empty(m, dtype=np.int32), area=np.empty(m),
               omega=np.empty(m), mass=np.empty(m))
    _check(lib.vsie_cuboid_faces(ctypes.byref(grid), _ptr(rho), float(w.rho0), m, ctypes.byref(cnt),
                                 _ptr(out["centres"]), _ptr(out["axis"]), _ptr(out["area"]),
                                 _ptr(out["omega"]), _ptr(out["mass"])))
    return out


def lsq_grad_alpha(vert, tet, tet_domain, alpha):
    """grad(alpha) (n_tet, 3) of an element-wise alpha by the library's least-squares
    stencil over same-subdomain face neighbours (vsie_lsq_grad_alpha)."""
    lib = load_library()
    mesh, keep = _tet_mesh(vert, tet)
    dom = None if tet_domain is None else np.ascontiguousarray(tet_domain, dtype=np.int8)
    a = _f64(alpha)
    out = np.empty((a.shape[0], 3), dtype=np.float64)
    _check(lib.vsie_lsq_grad_alpha(ctypes.byref(mesh), _ptr(dom), _ptr(a), _ptr(out)))
    return out


def lsq_grad_alpha_adjoint(vert, tet, tet_domain, d_grad):
    """W^T d_grad for grad(alpha) = W alpha (vsie_lsq_grad_alpha_adjoint); d_grad (n_tet, 3)."""
    lib = load_library()
    mesh, keep = _tet_mesh(vert, tet)
    dom = None if tet_domain is None else np.ascontiguousarray(tet_domain, dtype=np.int8)
    g = _f64(d_grad).reshape(-1)
    out = np.empty(g.shape[0] // 3, dtype=np.float64)
    _check(lib.vsie_lsq_grad_alpha_adjoint(ctypes.byref(mesh), _ptr(dom), _ptr(g), _ptr(out)))
    return out
