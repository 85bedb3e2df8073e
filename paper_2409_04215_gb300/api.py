"""ctypes binding of libmfs (include/mfs.h): argument marshalling only.

Every step of the solver runs in libmfs.so.  Arrays may be torch tensors (CUDA
or CPU) or NumPy arrays; FP64 contiguous copies are made where needed.  CUDA
tensors are passed as device pointers, everything else as host pointers (the
library stages host data itself).  Results come back as torch tensors on the
device of the first array argument (CUDA when the inputs were CUDA tensors).
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libmfs.so")
_lib = None

MFS_OK = 0
_STATUS = {
    0: "MFS_OK",
    1: "MFS_ERR_INVALID_ARG",
    2: "MFS_ERR_CUDA",
    3: "MFS_ERR_OOM",
    4: "MFS_ERR_NOT_CONVERGED",
    5: "MFS_ERR_BREAKDOWN",
    6: "MFS_ERR_ILL_CONDITIONED",
    7: "MFS_ERR_DEVICE_TIMEOUT",
}
EXPORTED = [
    "mfs_default_options",
    "mfs_abi_version",
    "mfs_setup",
    "mfs_update_centers",
    "mfs_matvec",
    "mfs_precond_apply",
    "mfs_pair_sum",
    "mfs_solve_elastance",
    "mfs_solve_mobility",
    "mfs_mobility_vjp",
    "mfs_stokeslet_sum_noalloc",
    "mfs_pair_variant",
    "mfs_pair_variant_info",
    "mfs_fp32_fma_rate",
    "mfs_matvec_transposed",
    "mfs_selftest_bounded_wait",
    "mfs_dirichlet_apply",
    "mfs_dirichlet_matvec",
    "mfs_solve_capacitance",
    "mfs_solve_resistance",
    "mfs_evaluate",
    "mfs_evaluate_stress",
    "mfs_last_error",
    "mfs_setup_error",
    "mfs_destroy",
]


class MFSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _PointSet(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pts", ctypes.c_void_p)]


class _Bodies(ctypes.Structure):
    _fields_ = [
        ("num_bodies", ctypes.c_int32),
        ("centers", ctypes.c_void_p),
        ("quats", ctypes.c_void_p),
        ("shape_id", ctypes.c_void_p),
        ("num_suspensions", ctypes.c_int32),
        ("body_offsets", ctypes.c_void_p),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double),
        ("gmres_tol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("restart", ctypes.c_int32),
        ("eps_trunc", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("max_rhs", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("tensor_cores", ctypes.c_int32),
        ("pair_variant", ctypes.c_int32),
        ("graphs", ctypes.c_int32),
        ("farfield", ctypes.c_int32),
        ("farfield_separation", ctypes.c_double),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("matvecs", ctypes.c_int32),
        ("lanes", ctypes.c_int32),
        ("rel_residual", ctypes.c_double),
        ("ms_setup", ctypes.c_double),
        ("ms_solve", ctypes.c_double),
        ("ms_pairs", ctypes.c_double),
        ("pairs", ctypes.c_double),
        ("launches", ctypes.c_int32),
        ("pair_launches", ctypes.c_int32),
        ("pairs_evaluated", ctypes.c_double),
    ]


@dataclasses.dataclass
class SolveInfo:
    iters: int
    converged: bool
    matvecs: int
    lanes: int
    rel_residual: float
    ms_setup: float
    ms_solve: float
    ms_pairs: float
    pairs: float
    launches: int
    pair_launches: int
    status: int
    pairs_evaluated: float = 0.0


ABI_VERSION = 4  # MFS_ABI_VERSION of the header these structures mirror


def load_library(path: Optional[str] = None):
    """Load libmfs.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"libmfs.so not found at {path}; build it with `python -m paper_2409_04215_gb300.build` "
            "(nvcc, sm_103a). There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.mfs_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.mfs_default_options.restype = None
    lib.mfs_abi_version.restype = i32
    lib.mfs_setup.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(_Bodies), i32, ctypes.POINTER(_PointSet),
                              ctypes.POINTER(_PointSet), ctypes.POINTER(Options), vp]
    lib.mfs_update_centers.argtypes = [vp, vp, vp]
    lib.mfs_matvec.argtypes = [vp, vp, vp, i32, vp]
    lib.mfs_matvec_transposed.argtypes = [vp, vp, vp, i32, vp]
    lib.mfs_precond_apply.argtypes = [vp, vp, vp, i32, i32, vp]
    lib.mfs_pair_sum.argtypes = [vp, vp, vp, i32, i32, vp]
    lib.mfs_solve_elastance.argtypes = [vp, vp, vp, i32, ctypes.POINTER(_Info), vp]
    lib.mfs_solve_mobility.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.POINTER(_Info), vp]
    lib.mfs_mobility_vjp.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
    lib.mfs_dirichlet_apply.argtypes = [vp, vp, vp, i32, vp]
    lib.mfs_dirichlet_matvec.argtypes = [vp, vp, vp, i32, vp]
    lib.mfs_solve_capacitance.argtypes = [vp, vp, vp, i32, ctypes.POINTER(_Info), vp]
    lib.mfs_solve_resistance.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.POINTER(_Info), vp]
    lib.mfs_evaluate.argtypes = [vp, vp, vp, i32, vp, i32, vp]
    lib.mfs_evaluate_stress.argtypes = [vp, vp, vp, vp, i32, vp, vp, i32, vp]
    lib.mfs_pair_variant_info.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.mfs_pair_variant_info.restype = ctypes.c_char_p
    lib.mfs_pair_variant.argtypes = [vp, i32]
    lib.mfs_fp32_fma_rate.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.mfs_selftest_bounded_wait.argtypes = [i32, ctypes.c_int64, vp]
    lib.mfs_pair_variant.restype = ctypes.c_char_p
    lib.mfs_last_error.argtypes = [vp]
    lib.mfs_last_error.restype = ctypes.c_char_p
    lib.mfs_setup_error.restype = ctypes.c_char_p
    lib.mfs_destroy.argtypes = [vp]
    lib.mfs_destroy.restype = None
    for name in EXPORTED:
        if not hasattr(lib, name):
            raise RuntimeError(f"libmfs.so lacks {name}")
    if lib.mfs_abi_version() != ABI_VERSION:
        raise RuntimeError(f"libmfs.so ABI {lib.mfs_abi_version()} != {ABI_VERSION}: rebuild the library")
    _lib = lib
    return lib


def pair_variants():
    """The pair-kernel table: [(index, name, d, nrhs, grad)]."""
    lib = load_library()
    out, i = [], 0
    while True:
        d, r, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        name = lib.mfs_pair_variant_info(i, ctypes.byref(d), ctypes.byref(r), ctypes.byref(g))
        if name is None:
            return out
        out.append((i, name.decode(), d.value, r.value, g.value))
        i += 1


def fp32_fma_rate(packed: bool = True, stream=None, mode: int | None = None) -> float:
    """Measured FP32 FMA throughput of the current CUDA device in TFLOP/s (mfs_fp32_fma_rate):
    f32x2 fma when packed, else scalar fma; `mode` (0-4, see mfs.h) overrides `packed` and selects
    the operand pattern and occupancy.  Synchronises the stream."""
    lib = load_library()
    out = ctypes.c_double()
    torch = _torch()
    st = _stream_ptr(stream, torch.device("cuda", torch.cuda.current_device()))
    rc = lib.mfs_fp32_fma_rate((1 if packed else 0) if mode is None else int(mode), ctypes.byref(out), st)
    if rc != MFS_OK:
        raise MFSError(rc, "mfs_fp32_fma_rate failed")
    return out.value


def selftest_bounded_wait(arrive: bool, limit: int = 1000, stream=None) -> int:
    """Status of mfs_selftest_bounded_wait: MFS_OK (0) when the barrier phase is completed, else the
    bounded wait gives up and the call returns MFS_ERR_DEVICE_TIMEOUT (7)."""
    lib = load_library()
    torch = _torch()
    st = _stream_ptr(stream, torch.device("cuda", torch.cuda.current_device()))
    return int(lib.mfs_selftest_bounded_wait(1 if arrive else 0, int(limit), st))


def default_options(**kw) -> Options:
    lib = load_library()
    o = Options()
    lib.mfs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _torch():
    import torch

    return torch


class _Arg:
    """An FP64 contiguous view of an array argument and the pointer passed to the library."""

    def __init__(self, a):
        torch = _torch()
        if isinstance(a, torch.Tensor):
            t = a.detach()
            if t.dtype != torch.float64:
                t = t.to(torch.float64)
            self.obj = t.contiguous()
            self.ptr = self.obj.data_ptr()
            self.device = self.obj.device
        else:
            self.obj = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            self.ptr = self.obj.ctypes.data
            self.device = None


def _stream_ptr(stream, device):
    torch = _torch()
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if device is not None and device.type == "cuda":
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    return ctypes.c_void_p(0)


class MFS:
    """One discretised multi-body problem (a libmfs context)."""

    def __init__(self, kind: str, centres, shapes: Sequence, quats=None, shape_id=None, body_offsets=None,
                 options: Optional[Options] = None, stream=None, **option_overrides):
        lib = load_library()
        self._lib = lib
        self.kind = kind
        self.d = 1 if kind == "laplace" else 3
        c = np.ascontiguousarray(np.asarray(centres, dtype=np.float64))
        self.P = c.shape[0]
        self._keep = [c]
        pts_proxy = (_PointSet * len(shapes))()
        pts_coll = (_PointSet * len(shapes))()
        self.M, self.N = [], []
        for i, (proxy, colloc) in enumerate(shapes):
            p = np.ascontiguousarray(np.asarray(proxy, dtype=np.float64))
            q = np.ascontiguousarray(np.asarray(colloc, dtype=np.float64))
            self._keep += [p, q]
            pts_proxy[i].n, pts_proxy[i].pts = p.shape[0], p.ctypes.data
            pts_coll[i].n, pts_coll[i].pts = q.shape[0], q.ctypes.data
            self.N.append(p.shape[0])
            self.M.append(q.shape[0])
        b = _Bodies()
        b.num_bodies = self.P
        b.centers = c.ctypes.data
        if quats is not None:
            qq = np.ascontiguousarray(np.asarray(quats, dtype=np.float64))
            self._keep.append(qq)
            b.quats = qq.ctypes.data
        sid = np.zeros(self.P, np.int32) if shape_id is None else np.ascontiguousarray(np.asarray(shape_id, np.int32))
        self._keep.append(sid)
        b.shape_id = sid.ctypes.data
        if body_offsets is not None:
            bo = np.ascontiguousarray(np.asarray(body_offsets, np.int32))
            self._keep.append(bo)
            b.num_suspensions = len(bo) - 1
            b.body_offsets = bo.ctypes.data
        else:
            b.num_suspensions = 1
        self.S = b.num_suspensions
        self.sum_M = int(sum(self.M[s] for s in sid))
        self.sum_N = int(sum(self.N[s] for s in sid))
        opt = options if options is not None else default_options()
        for k, v in option_overrides.items():
            setattr(opt, k, v)
        self.options = opt
        self._ctx = ctypes.c_void_p()
        st = _stream_ptr(stream, None)
        rc = lib.mfs_setup(ctypes.byref(self._ctx), 1 if kind == "stokes" else 0, ctypes.byref(b), len(shapes),
                           pts_proxy, pts_coll, ctypes.byref(opt), st)
        if rc != MFS_OK:
            raise MFSError(rc, lib.mfs_setup_error().decode())

    @classmethod
    def from_workload(cls, wl, **option_overrides):
        """Build from an object with the attributes of mfs_inputs.Workload."""
        shapes = [(sh.proxy, sh.colloc) for sh in wl.shapes]
        overrides = {"mu": float(wl.mu), **option_overrides}
        return cls(wl.kind, wl.centres, shapes, quats=wl.quats, shape_id=wl.shape_id, body_offsets=wl.body_offsets,
                   **overrides)

    # -- lifetime --------------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.mfs_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow_not_converged=False):
        if rc == MFS_OK or (allow_not_converged and rc == 4):
            return rc
        raise MFSError(rc, self._lib.mfs_last_error(self._ctx).decode())

    def _out(self, shape, like: _Arg):
        torch = _torch()
        dev = like.device if like.device is not None else torch.device("cpu")
        return torch.empty(shape, dtype=torch.float64, device=dev)

    # -- entry points (same names as the C ABI) ------------------------------------------
    def pair_variant(self, nrhs: int = 1) -> str:
        return self._lib.mfs_pair_variant(self._ctx, int(nrhs)).decode()

    def update_centers(self, centres, stream=None):
        a = _Arg(centres)
        self._check(self._lib.mfs_update_centers(self._ctx, a.ptr, _stream_ptr(stream, a.device)))

    def matvec(self, gamma, stream=None):
        a = _Arg(gamma)
        nrhs = a.obj.shape[0] if a.obj.ndim == 3 else 1
        y = self._out(tuple(a.obj.shape), a)
        self._check(self._lib.mfs_matvec(self._ctx, a.ptr, y.data_ptr(), nrhs, _stream_ptr(stream, a.device)))
        return y

    def matvec_transposed(self, w, stream=None):
        """y = A^T w (mfs_matvec_transposed), Stokes contexts; same shapes as matvec."""
        a = _Arg(w)
        nrhs = a.obj.shape[0] if a.obj.ndim == 3 else 1
        y = self._out(tuple(a.obj.shape), a)
        self._check(self._lib.mfs_matvec_transposed(self._ctx, a.ptr, y.data_ptr(), nrhs,
                                                    _stream_ptr(stream, a.device)))
        return y

    def precond_apply(self, gamma, project: bool = True, stream=None):
        a = _Arg(gamma)
        nrhs = a.obj.shape[0] if a.obj.ndim == 3 else 1
        shape = (nrhs, self.sum_N, self.d) if a.obj.ndim == 3 else (self.sum_N, self.d)
        lam = self._out(shape, a)
        self._check(self._lib.mfs_precond_apply(self._ctx, a.ptr, lam.data_ptr(), int(project), nrhs,
                                                _stream_ptr(stream, a.device)))
        return lam

    def pair_sum(self, strengths, include_self: bool = False, stream=None):
        a = _Arg(strengths)
        nrhs = a.obj.shape[0] if a.obj.ndim == 3 else 1
        shape = (nrhs, self.sum_M, self.d) if a.obj.ndim == 3 else (self.sum_M, self.d)
        u = self._out(shape, a)
        self._check(self._lib.mfs_pair_sum(self._ctx, a.ptr, u.data_ptr(), nrhs, int(include_self),
                                           _stream_ptr(stream, a.device)))
        return u

    def solve_mobility(self, F, T, stream=None, allow_not_converged=False):
        f, t = _Arg(F), _Arg(T)
        nrhs = f.obj.shape[0] if f.obj.ndim == 3 else 1
        U = self._out(tuple(f.obj.shape), f)
        W = self._out(tuple(f.obj.shape), f)
        info = _Info()
        rc = self._lib.mfs_solve_mobility(self._ctx, f.ptr, t.ptr, U.data_ptr(), W.data_ptr(), nrhs,
                                          ctypes.byref(info), _stream_ptr(stream, f.device))
        self._check(rc, allow_not_converged)
        return U, W, _info(info, rc)

    def solve_elastance(self, Q, stream=None, allow_not_converged=False):
        q = _Arg(Q)
        nrhs = q.obj.shape[0] if q.obj.ndim == 2 else 1
        V = self._out(tuple(q.obj.shape), q)
        info = _Info()
        rc = self._lib.mfs_solve_elastance(self._ctx, q.ptr, V.data_ptr(), nrhs, ctypes.byref(info),
                                           _stream_ptr(stream, q.device))
        self._check(rc, allow_not_converged)
        return V, _info(info, rc)

    # -- Dirichlet problems (Sec. 2): capacitance and resistance ------------------------------
    def dirichlet_apply(self, gamma, stream=None):
        a = _Arg(gamma)
        nrhs = a.obj.shape[0] if a.obj.ndim == 3 else 1
        shape = (nrhs, self.sum_N, self.d) if a.obj.ndim == 3 else (self.sum_N, self.d)
        alpha = self._out(shape, a)
        self._check(self._lib.mfs_dirichlet_apply(self._ctx, a.ptr, alpha.data_ptr(), nrhs,
                                                  _stream_ptr(stream, a.device)))
        return alpha

    def dirichlet_matvec(self, gamma, stream=None):
        a = _Arg(gamma)
        nrhs = a.obj.shape[0] if a.obj.ndim == 3 else 1
        y = self._out(tuple(a.obj.shape), a)
        self._check(self._lib.mfs_dirichlet_matvec(self._ctx, a.ptr, y.data_ptr(), nrhs,
                                                   _stream_ptr(stream, a.device)))
        return y

    def solve_capacitance(self, phi, stream=None, allow_not_converged=False):
        p = _Arg(phi)
        nrhs = p.obj.shape[0] if p.obj.ndim == 2 else 1
        q = self._out(tuple(p.obj.shape), p)
        info = _Info()
        rc = self._lib.mfs_solve_capacitance(self._ctx, p.ptr, q.data_ptr(), nrhs, ctypes.byref(info),
                                             _stream_ptr(stream, p.device))
        self._check(rc, allow_not_converged)
        return q, _info(info, rc)

    def solve_resistance(self, U, Omega, stream=None, allow_not_converged=False):
        u, w = _Arg(U), _Arg(Omega)
        nrhs = u.obj.shape[0] if u.obj.ndim == 3 else 1
        F = self._out(tuple(u.obj.shape), u)
        T = self._out(tuple(u.obj.shape), u)
        info = _Info()
        rc = self._lib.mfs_solve_resistance(self._ctx, u.ptr, w.ptr, F.data_ptr(), T.data_ptr(), nrhs,
                                            ctypes.byref(info), _stream_ptr(stream, u.device))
        self._check(rc, allow_not_converged)
        return F, T, _info(info, rc)

    def evaluate(self, points, owner=None, nrhs: int = 1, stream=None):
        """Field of the last solve at points (npoints, 3): returns (nrhs, npoints, d)."""
        torch = _torch()
        p = _Arg(points)
        npts = int(p.obj.shape[0])
        o = None
        if owner is not None:
            o = owner if isinstance(owner, torch.Tensor) else torch.as_tensor(np.asarray(owner))
            o = o.to(torch.int32).contiguous()
        out = self._out((nrhs, npts, self.d), p)
        self._check(self._lib.mfs_evaluate(self._ctx, p.ptr, None if o is None else o.data_ptr(), npts,
                                           out.data_ptr(), nrhs, _stream_ptr(stream, p.device)))
        return out

    def evaluate_stress(self, points, normals=None, owner=None, nrhs: int = 1, pressure: bool = True,
                        traction: bool = True, stream=None):
        """(pressure (nrhs, npoints) or None, traction (nrhs, npoints, 3) or None) of the last Stokes solve."""
        torch = _torch()
        p = _Arg(points)
        npts = int(p.obj.shape[0])
        n = _Arg(normals) if normals is not None else None
        o = None
        if owner is not None:
            o = owner if isinstance(owner, torch.Tensor) else torch.as_tensor(np.asarray(owner))
            o = o.to(torch.int32).contiguous()
        pr = self._out((nrhs, npts), p) if pressure else None
        tr = self._out((nrhs, npts, 3), p) if traction else None
        self._check(self._lib.mfs_evaluate_stress(self._ctx, p.ptr, None if n is None else n.ptr,
                                                  None if o is None else o.data_ptr(), npts,
                                                  None if pr is None else pr.data_ptr(),
                                                  None if tr is None else tr.data_ptr(), nrhs,
                                                  _stream_ptr(stream, p.device)))
        return pr, tr

    def mobility_vjp(self, dU, dOmega, want_force_grads: bool = False, stream=None):
        a, b = _Arg(dU), _Arg(dOmega)
        nrhs = a.obj.shape[0] if a.obj.ndim == 3 else 1
        dc = self._out((self.P, 3), a)
        dF = self._out(tuple(a.obj.shape), a) if want_force_grads else None
        dT = self._out(tuple(a.obj.shape), a) if want_force_grads else None
        rc = self._lib.mfs_mobility_vjp(self._ctx, a.ptr, b.ptr, nrhs, dc.data_ptr(),
                                        dF.data_ptr() if dF is not None else None,
                                        dT.data_ptr() if dT is not None else None, _stream_ptr(stream, a.device))
        self._check(rc)
        return dc, dF, dT


def _info(i: _Info, rc: int) -> SolveInfo:
    return SolveInfo(i.iters, bool(i.converged), i.matvecs, i.lanes, i.rel_residual, i.ms_setup, i.ms_solve,
                     i.ms_pairs, i.pairs, i.launches, i.pair_launches, rc, i.pairs_evaluated)


def mobility(mfs: "MFS", centres, F, T):
    """(U, Omega) = mobility(centres, F, T) as a differentiable torch operation.

    Forward: mfs_update_centers + mfs_solve_mobility; backward: mfs_mobility_vjp (gradients with
    respect to the body centres, the forces and the torques).  F, T: [nrhs][P][3].
    """
    torch = _torch()

    class _Mobility(torch.autograd.Function):
        @staticmethod
        def forward(ctx_, c, f, t):
            mfs.update_centers(c.detach())
            U, W, _ = mfs.solve_mobility(f.detach(), t.detach())
            return U, W

        @staticmethod
        def backward(ctx_, gU, gW):
            dc, dF, dT = mfs.mobility_vjp(gU.contiguous(), gW.contiguous(), want_force_grads=True)
            return dc.to(gU.device), dF.to(gU.device), dT.to(gU.device)

    return _Mobility.apply(centres, F, T)
