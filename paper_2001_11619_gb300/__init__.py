"""GB300 recursive-skeletonization solver for 2-D Stokes flow in
multiply-connected domains (Ryan & Damle's bordered skeletonization with
fast updating).

This module is a thin ctypes binding over the C ABI of ``include/skel.h``:
it marshals arrays (PyTorch tensors on the GPU or CPU, or numpy arrays) to
plain pointers and calls the library.  Every step of the method runs in the
library's CUDA kernels; there is no CPU fallback, and importing this module
raises if the library is missing.

Array conventions (matching the oracle): a right-hand side or solution is a
vector of length 2N+3p or a matrix (2N+3p, nrhs); node j's density is at
rows 2j, 2j+1; lambda follows hole-major (alpha_i1, alpha_i2, beta_i).
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np

from . import _build

__all__ = ["Solver", "load_library", "SkelError", "FP64", "MIXED",
           "library_path", "kernel_launches", "release_cached_memory"]

FP64, MIXED = 0, 1
STOKES, LAPLACE = 0, 1   # kernel families (skel_params.kernel)
_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECAPACITY", -4: "ESINGULAR",
           -5: "ENOCONV", -6: "ETIMEOUT", -7: "ECUDA", -8: "ESTATE"}


class SkelError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"skel error {code} ({_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("n_proxy", C.c_int32),
                ("proxy_ratio", C.c_double), ("id_tol", C.c_double),
                ("precision", C.c_int32), ("gmres_tol", C.c_double),
                ("gmres_maxit", C.c_int32), ("kernel", C.c_int32)]


class _Geom(C.Structure):
    _fields_ = [("N", C.c_int64), ("p", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p),
                ("dx", C.c_void_p), ("dy", C.c_void_p),
                ("ddx", C.c_void_p), ("ddy", C.c_void_p),
                ("dt", C.c_void_p), ("comp", C.c_void_p),
                ("centers", C.c_void_p)]


_lib = None


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load_library().skel_kernel_launches())


def release_cached_memory() -> None:
    """Return the device blocks cached by the library to the driver
    (skel_release_cached_memory)."""
    rc = load_library().skel_release_cached_memory()
    if rc != 0:
        raise SkelError(rc, "skel_release_cached_memory failed")


def measure_alu_peaks() -> dict:
    """FP64 and FP32 FMA throughput of the current device in TFLOP/s
    (skel_measure_alu_peaks)."""
    out = (C.c_double * 2)()
    rc = load_library().skel_measure_alu_peaks(out)
    if rc != 0:
        raise SkelError(rc, "skel_measure_alu_peaks failed")
    return {"fp64_tflops": out[0], "fp32_tflops": out[1]}


def gemm_tf32x3(A, B, C):
    """C <- C - A @ B on the tensor cores in 3xTF32 (skel_gemm_tf32x3), the
    building block of the mixed form's large-box products.  A (M, K),
    B (K, N) and C (M, N) are float64 CUDA tensors stored column-major
    (stride (1, rows), as ``torch.empty(cols, rows).t()`` gives)."""
    import torch
    M, K = A.shape
    N = B.shape[1]
    for name, t, r in (("A", A, M), ("B", B, K), ("C", C, M)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.stride(0) == 1
                and (t.shape[1] <= 1 or t.stride(1) >= r)):
            raise ValueError(f"{name} must be a column-major float64 CUDA "
                             "tensor")
    if B.shape[0] != K or tuple(C.shape) != (M, N):
        raise ValueError("shapes do not match")
    st = torch.cuda.current_stream().cuda_stream
    rc = load_library().skel_gemm_tf32x3(
        M, N, K, A.data_ptr(), max(A.stride(1), M), B.data_ptr(),
        max(B.stride(1), K), C.data_ptr(), max(C.stride(1), M), st)
    if rc != 0:
        raise SkelError(rc, "skel_gemm_tf32x3 failed")
    return C


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libskel.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library {_build.LIB} is missing; "
                          "run __graft_entry__.build()")
    lib = C.CDLL(_build.LIB)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
    lib.skel_default_params.argtypes = [C.POINTER(_Params)]
    lib.skel_build_tree.argtypes = [C.POINTER(_Geom), C.POINTER(_Params), vp,
                                    C.POINTER(vp)]
    lib.skel_factor.argtypes = [vp]
    lib.skel_update_moved_nodes.argtypes = [vp, i64, vp, C.POINTER(_Geom)]
    lib.skel_update_geometry.argtypes = [vp, C.POINTER(_Geom), vp]
    lib.skel_set_tuning.argtypes = [vp, C.c_char_p, C.c_double]
    lib.skel_get_tuning.argtypes = [vp, C.c_char_p, C.POINTER(C.c_double)]
    lib.skel_solve.argtypes = [vp, i32, dp, dp]
    lib.skel_solve_adjoint.argtypes = [vp, i32, dp, dp]
    lib.skel_eval_velocity.argtypes = [vp, i32, dp, i64, dp, dp, dp]
    lib.skel_eval_velocity_noalloc.argtypes = [vp, i32, dp, i64, dp, dp, dp]
    lib.skel_point_force_rhs.argtypes = [vp, i32, i32, dp, dp, i32, dp]
    lib.skel_matvec.argtypes = [vp, i32, dp, dp]
    lib.skel_grad_bilinear.argtypes = [vp, dp, dp, dp]
    lib.skel_grad_bilinear.restype = C.c_int
    lib.skel_grad_velocity.argtypes = [vp, dp, i64, dp, dp, dp, dp, dp]
    lib.skel_grad_velocity.restype = C.c_int
    lib.skel_velocity_energy.argtypes = [vp, dp, i64, dp, dp,
                                         C.POINTER(C.c_double), dp]
    lib.skel_velocity_energy.restype = C.c_int
    lib.skel_velocity_energy_gradient.argtypes = [vp, dp, i64, dp, dp, dp]
    lib.skel_velocity_energy_gradient.restype = C.c_int
    lib.skel_matvec_df.argtypes = [vp, i32, dp, dp]
    lib.skel_matvec_df.restype = C.c_int
    lib.skel_matvec_adjoint.argtypes = [vp, i32, dp, dp]
    lib.skel_matvec_adjoint.restype = C.c_int
    lib.skel_matvec_adjoint_df.argtypes = [vp, i32, dp, dp]
    lib.skel_matvec_adjoint_df.restype = C.c_int
    lib.skel_stats.argtypes = [vp, C.c_char_p, C.c_size_t]
    lib.skel_last_error.argtypes = [vp]
    lib.skel_last_error.restype = C.c_char_p
    lib.skel_destroy.argtypes = [vp]
    lib.skel_set_timing.argtypes = [vp, i32]
    lib.skel_set_timing.restype = C.c_int
    lib.skel_gemm_tf32x3.argtypes = [i32, i32, i32, dp, i64, dp, i64, dp,
                                     i64, vp]
    lib.skel_gemm_tf32x3.restype = C.c_int
    lib.skel_measure_alu_peaks.argtypes = [C.POINTER(C.c_double)]
    lib.skel_measure_alu_peaks.restype = C.c_int
    lib.skel_release_cached_memory.argtypes = []
    lib.skel_release_cached_memory.restype = C.c_int
    lib.skel_kernel_launches.argtypes = []
    lib.skel_kernel_launches.restype = C.c_int64
    for name in ("skel_build_tree", "skel_factor", "skel_update_moved_nodes",
                 "skel_update_geometry", "skel_set_tuning", "skel_get_tuning",
                 "skel_solve", "skel_solve_adjoint", "skel_eval_velocity",
                 "skel_eval_velocity_noalloc",
                 "skel_point_force_rhs", "skel_matvec", "skel_stats"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


# -- array marshalling ---------------------------------------------------------

def _torch():
    import torch
    return torch


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class _Arr:
    """Keeps a contiguous buffer alive and exposes its pointer."""

    def __init__(self, a, dtype):
        if _is_torch(a):
            torch = _torch()
            tdt = torch.float64 if dtype == np.float64 else (
                torch.int32 if dtype == np.int32 else torch.int64)
            self.obj = a.detach().to(tdt).contiguous()
            self.ptr = self.obj.data_ptr()
            self.cuda = self.obj.is_cuda
        else:
            self.obj = np.ascontiguousarray(np.asarray(a, dtype=dtype))
            self.ptr = self.obj.ctypes.data
            self.cuda = False


def _targets(tx, ty):
    """Target coordinates as two buffers of one length (the library reads
    nt entries of each)."""
    x = _Arr(tx, np.float64)
    y = _Arr(ty, np.float64)
    if x.obj.ndim != 1 or y.obj.ndim != 1 or len(x.obj) != len(y.obj):
        raise ValueError("tx and ty must be 1-D arrays of the same length")
    return x, y, len(x.obj)


def _vec(a, n, what):
    """A length-n FP64 vector buffer (the library reads n entries): a
    vector of length n or a single column (n, 1)."""
    b = _Arr(a, np.float64)
    if b.obj.ndim == 2 and tuple(b.obj.shape) == (n, 1):
        b.obj = b.obj.reshape(n)
    if b.obj.ndim != 1 or len(b.obj) != n:
        raise ValueError(f"{what} must be a vector of length {n}")
    return b


def _rhs_in(a, n):
    """(n,) or (n, nrhs) -> contiguous (nrhs, n) buffer (column-major)."""
    if _is_torch(a):
        t = a.detach().to(_torch().float64)
        one = t.dim() == 1
        t = t.reshape(n, -1).t().contiguous()
        return t, one
    arr = np.asarray(a, dtype=np.float64)
    one = arr.ndim == 1
    return np.ascontiguousarray(arr.reshape(n, -1).T), one


def _like(buf, shape):
    if _is_torch(buf):
        return _torch().empty(shape, dtype=_torch().float64,
                              device=buf.device)
    return np.empty(shape, dtype=np.float64)


def _ptr(a):
    return a.data_ptr() if _is_torch(a) else a.ctypes.data


def _out_rhs(buf, one):
    out = buf.t() if _is_torch(buf) else buf.T
    return out[:, 0] if one else out


# geometry arrays that the shape derivatives differentiate, in the order of
# the gradient layout (then the hole centres)
GEOM_FIELDS = ("x", "y", "dx", "dy", "ddx", "ddy")


class Solver:
    """One geometry, its quadtree and its factorization on the GPU.

    ``geom`` has the fields of a ``workloads.Workload`` (x, y, dx, dy, ddx,
    ddy, dt, comp, centers) as numpy arrays or torch tensors.
    """

    def __init__(self, geom, leaf_size=64, n_proxy=64, proxy_ratio=1.5,
                 id_tol=1e-12, precision=FP64, gmres_tol=1e-12,
                 gmres_maxit=50, stream=None, kernel=STOKES):
        self.lib = load_library()
        prm = _Params()
        self.lib.skel_default_params(C.byref(prm))
        prm.leaf_size, prm.n_proxy = int(leaf_size), int(n_proxy)
        prm.proxy_ratio, prm.id_tol = float(proxy_ratio), float(id_tol)
        prm.precision = int(precision)
        prm.gmres_tol, prm.gmres_maxit = float(gmres_tol), int(gmres_maxit)
        prm.kernel = int(kernel)
        self.kernel = int(kernel)
        self.params = prm
        g, keep = self._geom(geom)
        if stream is None and _is_torch(geom.x) and geom.x.is_cuda:
            stream = _torch().cuda.current_stream().cuda_stream
        self._stream = stream
        h = C.c_void_p()
        self._check(self.lib.skel_build_tree(C.byref(g), C.byref(prm),
                                             C.c_void_p(stream), C.byref(h)),
                    None)
        self.h = h
        self._sizes(g)

    def _sizes(self, g):
        self.N = int(g.N)
        self.p = int(g.p)
        # unknowns: [mu (2 per node); lambda (3 per hole)] for Stokes, mu
        # (1 per node) for the Laplace form
        self.n = (self.N if self.kernel == LAPLACE
                  else 2 * self.N + 3 * self.p)

    # ------------------------------------------------------------------
    def _geom(self, w):
        keep = [_Arr(getattr(w, f), np.float64)
                for f in ("x", "y", "dx", "dy", "ddx", "ddy", "dt")]
        keep.append(_Arr(w.comp, np.int32))
        keep.append(_Arr(w.centers, np.float64))
        g = _Geom()
        g.N = len(keep[0].obj)
        g.p = int(keep[-1].obj.reshape(-1).shape[0] // 2)
        (g.x, g.y, g.dx, g.dy, g.ddx, g.ddy, g.dt, g.comp, g.centers) = \
            [k.ptr for k in keep]
        self._keep = keep
        return g, keep

    def _check(self, rc, h):
        if rc != 0:
            msg = self.lib.skel_last_error(h).decode()
            raise SkelError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.skel_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def factor(self):
        self._check(self.lib.skel_factor(self.h), self.h)

    def update_moved_nodes(self, node_ids, new_geom):
        g, keep = self._geom(new_geom)
        ids = _Arr(node_ids, np.int64)
        self._check(self.lib.skel_update_moved_nodes(
            self.h, len(ids.obj), ids.ptr, C.byref(g)), self.h)

    def update_geometry(self, new_geom, old_id):
        """Update after inserted or deleted holes (skel_update_geometry):
        new_geom may have a different node and hole count; old_id[j] is the
        previous id of new node j, or -1 for a new node (kept ids in
        increasing order)."""
        g, keep = self._geom(new_geom)
        ids = _Arr(old_id, np.int64)
        if len(ids.obj) != int(g.N):
            raise ValueError("old_id needs one entry per new node")
        self._check(self.lib.skel_update_geometry(self.h, C.byref(g), ids.ptr),
                    self.h)
        self._sizes(g)

    TUNING_KEYS = ("cluster_min_n", "cluster_level_boxes", "sweep_rhs_chunk",
                   "cluster_mid_min_n", "cluster_mid_level_boxes",
                   "wide_min_n", "wide_qr_min_n", "tc_products")

    def set_tuning(self, **kw):
        """Launch-shape parameters (skel_set_tuning); the solver must be
        factored again afterwards."""
        for k, v in kw.items():
            self._check(self.lib.skel_set_tuning(self.h, k.encode(),
                                                 float(v)), self.h)

    def set_gmres_fp64_check(self, on=True):
        """Mixed form: decide GMRES convergence on the FP64 operator's
        residual always (on), or on the double-float one when gmres_tol >=
        1e-11 (off, the default).  Keeps the factorization."""
        self._check(self.lib.skel_set_tuning(self.h, b"gmres_fp64_check",
                                             float(bool(on))), self.h)

    def get_tuning(self):
        out = {}
        for k in self.TUNING_KEYS:
            v = C.c_double()
            self._check(self.lib.skel_get_tuning(self.h, k.encode(),
                                                 C.byref(v)), self.h)
            out[k] = int(v.value)
        return out

    def _solve(self, f, fn):
        buf, one = _rhs_in(f, self.n)
        out = _like(buf, tuple(buf.shape))
        self._check(fn(self.h, buf.shape[0], _ptr(buf), _ptr(out)), self.h)
        return _out_rhs(out, one)

    def solve(self, f):
        return self._solve(f, self.lib.skel_solve)

    def solve_adjoint(self, g):
        return self._solve(g, self.lib.skel_solve_adjoint)

    def matvec(self, x):
        return self._solve(x, self.lib.skel_matvec)

    def matvec_adjoint(self, z):
        return self._solve(z, self.lib.skel_matvec_adjoint)

    # -- shape derivatives ---------------------------------------------------

    def _geom_grad(self, g):
        N, p = self.N, self.p
        out = {f: g[i * N:(i + 1) * N] for i, f in enumerate(GEOM_FIELDS)}
        out["centers"] = g[6 * N:].reshape(p, 2)
        return out

    def grad_bilinear(self, z, s):
        """d(z^T A s)/d(geometry) for fixed vectors: dict with the samples'
        fields (x, y, dx, dy, ddx, ddy) and centers."""
        zb = _vec(z, self.n, "z")
        sb = _vec(s, self.n, "s")
        out = _like(zb.obj, (6 * self.N + 2 * self.p,))
        self._check(self.lib.skel_grad_bilinear(self.h, zb.ptr, sb.ptr,
                                                _ptr(out)), self.h)
        return self._geom_grad(out)

    def grad_velocity(self, s, tx, ty, ubar):
        """(E^T ubar, d(ubar . E s)/d(geometry)) for the velocity at fixed
        interior targets; ubar has shape (nt, 2)."""
        sb = _vec(s, self.n, "s")
        tx, ty, nt = _targets(tx, ty)
        ub = _Arr(ubar, np.float64)
        if ub.obj.size != 2 * nt:
            raise ValueError("ubar must have shape (nt, 2)")
        gs = _like(sb.obj, (self.n,))
        g = _like(sb.obj, (6 * self.N + 2 * self.p,))
        self._check(self.lib.skel_grad_velocity(
            self.h, sb.ptr, nt, tx.ptr, ty.ptr, ub.ptr, _ptr(gs), _ptr(g)),
            self.h)
        return gs, self._geom_grad(g)

    def velocity_energy(self, f, tx, ty):
        """J = sum_t |u(x_t)|^2 for the solution s of A s = f
        (skel_velocity_energy).  Returns (J, s)."""
        fb = _vec(f, self.n, "f")
        tx, ty, nt = _targets(tx, ty)
        out = _like(fb.obj, (self.n,))
        J = C.c_double()
        self._check(self.lib.skel_velocity_energy(
            self.h, fb.ptr, nt, tx.ptr, ty.ptr, C.byref(J), _ptr(out)),
            self.h)
        return float(J.value), out

    def velocity_energy_gradient_at(self, s, tx, ty):
        """dJ/d(geometry) at the solution s of the factored geometry
        (skel_velocity_energy_gradient): dict of the samples' fields and
        centers."""
        sb = _vec(s, self.n, "s")
        tx, ty, nt = _targets(tx, ty)
        g = _like(sb.obj, (6 * self.N + 2 * self.p,))
        self._check(self.lib.skel_velocity_energy_gradient(
            self.h, sb.ptr, nt, tx.ptr, ty.ptr, _ptr(g)), self.h)
        return self._geom_grad(g)

    def velocity_energy_gradient(self, f, tx, ty):
        """J = sum_t |u(x_t)|^2 for the solution of A s = f, and dJ/d(geometry)
        by the adjoint method (f must not depend on the differentiated
        samples).  Returns (J, s, gradient dict)."""
        J, s1 = self.velocity_energy(f, tx, ty)
        return J, s1, self.velocity_energy_gradient_at(s1, tx, ty)

    def matvec_df(self, x):
        """A x with the double-layer sums in double-float arithmetic."""
        return self._solve(x, self.lib.skel_matvec_df)

    def matvec_adjoint_df(self, z):
        """A^T z with the double-layer sums in double-float arithmetic."""
        return self._solve(z, self.lib.skel_matvec_adjoint_df)

    def eval_velocity(self, sol, tx, ty):
        """Returns (nt, 2, nrhs) like the oracle's interior_velocity; for
        the Laplace form the potential, (nt, nrhs)."""
        buf, one = _rhs_in(sol, self.n)
        tx, ty, nt = _targets(tx, ty)
        nrhs = buf.shape[0]
        lap = self.kernel == LAPLACE
        out = _like(buf, (nrhs, nt) if lap else (nrhs, nt, 2))
        self._check(self.lib.skel_eval_velocity(self.h, nrhs, _ptr(buf), nt,
                                                tx.ptr, ty.ptr, _ptr(out)),
                    self.h)
        if lap:
            return out.T
        return out.permute(1, 2, 0) if _is_torch(out) else \
            out.transpose(1, 2, 0)

    def eval_potential(self, sol, tx, ty):
        """Laplace form: u = S mu at the targets, (nt, nrhs)."""
        if self.kernel != LAPLACE:
            raise ValueError("eval_potential is for the Laplace form")
        return self.eval_velocity(sol, tx, ty)

    def eval_velocity_noalloc(self, sol, tx, ty, out=None):
        """skel_eval_velocity_noalloc: the library allocates nothing, so sol
        (n,) or (n, nrhs), tx, ty and ``out`` (nrhs, nt, 2) must be CUDA
        tensors.  tx, ty and out must be contiguous float64 tensors on
        sol's device (the kernels write out in place, so a wrong shape or
        dtype is rejected here, before the call).  Returns (nt, 2, nrhs)
        like eval_velocity."""
        buf, one = _rhs_in(sol, self.n)
        nrhs = buf.shape[0]
        torch = _torch() if _is_torch(buf) else None

        def cuda_f64(a):
            return (torch is not None and _is_torch(a) and a.is_cuda and
                    a.dtype == torch.float64 and a.is_contiguous() and
                    a.device == buf.device)

        # torch tensors are checked here (the kernels write out in place);
        # other arrays are passed on as host pointers, which the library
        # refuses (it stages nothing)
        for name, a in (("tx", tx), ("ty", ty)):
            if _is_torch(a) and not (cuda_f64(a) and a.dim() == 1):
                raise ValueError(f"{name} must be a contiguous 1-D float64 "
                                 "CUDA tensor on sol's device")
        if len(tx) != len(ty):
            raise ValueError("tx and ty must have the same length")
        nt = len(tx)
        if out is None:
            out = _like(buf, (nrhs, nt, 2))
        if _is_torch(out) and not (
                cuda_f64(out) and tuple(out.shape) == (nrhs, nt, 2)):
            raise ValueError(f"out must be a contiguous float64 CUDA tensor "
                             f"of shape ({nrhs}, {nt}, 2) on sol's device")
        if not _is_torch(out) and np.asarray(out).shape != (nrhs, nt, 2):
            raise ValueError(f"out must have shape ({nrhs}, {nt}, 2)")
        txa = tx if cuda_f64(tx) else _Arr(tx, np.float64)
        tya = ty if cuda_f64(ty) else _Arr(ty, np.float64)
        ptx = txa.data_ptr() if cuda_f64(tx) else txa.ptr
        pty = tya.data_ptr() if cuda_f64(ty) else tya.ptr
        self._check(self.lib.skel_eval_velocity_noalloc(
            self.h, nrhs, _ptr(buf), nt, ptx, pty, _ptr(out)), self.h)
        return out.permute(1, 2, 0) if _is_torch(out) else \
            out.transpose(1, 2, 0)

    def point_force_rhs(self, src_xy, src_f, holes_zero=False, like=None):
        """Boundary data from point forces; src arrays (nrhs, ns, 2).
        Returns (2N+3p, nrhs) on the device of ``like`` (numpy if None)."""
        sxy = _Arr(src_xy, np.float64)
        sf = _Arr(src_f, np.float64)
        nrhs, ns = sxy.obj.shape[0], sxy.obj.shape[1]
        out = _like(like if like is not None else np.zeros(1),
                    (nrhs, self.n))
        self._check(self.lib.skel_point_force_rhs(
            self.h, nrhs, ns, sxy.ptr, sf.ptr, int(bool(holes_zero)),
            _ptr(out)), self.h)
        return _out_rhs(out, False)

    def set_timing(self, on=True):
        """Per-kernel CUDA-event timing (reported by stats()['kernels'])."""
        self._check(self.lib.skel_set_timing(self.h, int(bool(on))), self.h)

    def stats(self):
        buf = C.create_string_buffer(1 << 16)
        self._check(self.lib.skel_stats(self.h, buf, len(buf)), self.h)
        return json.loads(buf.value.decode())
