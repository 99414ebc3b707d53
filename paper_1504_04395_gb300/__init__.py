"""GB300 simultaneous short-recurrence Krylov solvers (Rashedi, Birk, Frommer, Ebadi).

Thin ctypes binding of the C interface in include/kr.h.  Every step of a solve
runs in the CUDA library libkrylov_gb300.so; this module only marshals torch
tensors (device memory, streams) into the C calls.  There is no CPU fallback:
importing the package fails loudly if the library has not been built (call
paper_1504_04395_gb300.build.build()).

Functions with the C names (kr_solve, kr_adjoint_solve, kr_op_create_csr,
kr_op_apply, kr_op_apply_reduce, kr_block_reduce, kr_thin_qr, kr_grad_values,
kr_last_error) take torch tensors where the C call takes device pointers.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import LIBPATH

METHODS = {
    "bl_bicg": 0, "bl_bicg_rq": 1, "gl_bicg": 2, "egl_bicg": 3, "bl_bicgstab": 4,
    "bl_bicgstab_rq": 5, "gl_bicgstab": 6, "bl_qmr": 7, "gl_qmr": 8, "egl_qmr": 9, "li_bicg": 10,
    "li_bicgstab": 11, "li_qmr": 12,
}
STATUS = {0: "OK", 1: "BREAKDOWN", 2: "DIVERGED", 3: "NAN", 4: "MAXIT", 5: "TIMEOUT", 6: "BAD_ARG",
          7: "OOM", 8: "CUDA_ERROR", 9: "UNSUPPORTED"}
RED = {"gram": 1, "trace": 2, "sumv": 3, "norm2": 4}
FP64, FP32_REFINE = 0, 1


GRAPHS = {"auto": 0, "on": 1, "off": 2}


class KrOptions(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("maxit", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int32),
        ("shadow_mode", ctypes.c_int32),
        ("shadow", ctypes.c_void_p),
        ("check_every", ctypes.c_int32),
        ("host_buffers", ctypes.c_int32),
        ("history", ctypes.POINTER(ctypes.c_double)),
        ("time_limit_s", ctypes.c_double),
        ("graphs", ctypes.c_int32),
        ("orthonormalize_B", ctypes.c_int32),
        ("deterministic", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class KrInfo(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("matvecs", ctypes.c_int32),
        ("relres_recursive", ctypes.c_double),
        ("relres_true", ctypes.c_double),
        ("status", ctypes.c_int32),
        ("outer_iters", ctypes.c_int32),
        ("fp64_iters", ctypes.c_int32),
        ("breakdown_iter", ctypes.c_int32),
    ]


class KrProfile(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64 * 8),
        ("ms", ctypes.c_double * 8),
        ("flops", ctypes.c_double * 8),
        ("bytes", ctypes.c_double * 8),
    ]


KERNEL_CLASSES = ["spmm", "lincomb", "reduce", "coef", "other", "spmm_c64", "lincomb_c64"]

# exported symbols and their C signatures (must match include/kr.h)
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
SIGNATURES = {
    "kr_options_default": (None, [ctypes.POINTER(KrOptions)]),
    "kr_op_create_csr": (_I32, [_I64, _I64, _P, _P, _P, _I32, ctypes.POINTER(_P)]),
    "kr_op_create_csr_async": (_I32, [_I64, _I64, _P, _P, _P, _I32, _P, ctypes.POINTER(_P)]),
    "kr_op_destroy": (_I32, [_P]),
    "kr_op_create_stencil": (_I32, [_I32, _P, _P, _I32, ctypes.POINTER(_P)]),
    "kr_op_create_lattice4d": (_I32, [_P, _P, ctypes.c_double, _P, _P, _I32, ctypes.POINTER(_P)]),
    "kr_op_update_values": (_I32, [_P, _P, _I32]),
    "kr_op_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I32)]),
    "kr_op_apply": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "kr_op_apply_reduce": (_I32, [_P, _I32, _I32, _P, _P, _P, _I32, _P, _P]),
    "kr_block_reduce": (_I32, [_I64, _I32, _P, _P, _I32, _P, _P]),
    "kr_op_apply_reduce_c64": (_I32, [_P, _I32, _I32, _P, _P, _P, _I32, _P, _P]),
    "kr_block_reduce_c64": (_I32, [_I64, _I32, _P, _P, _I32, _P, _P]),
    "kr_thin_qr": (_I32, [_I64, _I32, _P, _P, _P, _P]),
    "kr_solve": (_I32, [_P, _I32, _I32, _P, _P, ctypes.POINTER(KrOptions), _P, ctypes.POINTER(KrInfo)]),
    "kr_adjoint_solve": (_I32, [_P, _I32, _I32, _P, _P, ctypes.POINTER(KrOptions), _P, ctypes.POINTER(KrInfo)]),
    "kr_grad_values": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "kr_last_error": (ctypes.c_char_p, []),
    "kr_block_reduce_noalloc": (_I32, [_I64, _I32, _P, _P, _I32, _P, _P]),
    "kr_profile_enable": (_I32, [_I32, _I32]),
    "kr_set_column_pairs": (_I32, [_I32]),
    "kr_op_set_preconditioner": (_I32, [_P, _I32]),
    "kr_op_apply_precond": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "kr_set_lattice_rows_per_thread": (_I32, [_I32]),
    "kr_profile_read": (_I32, [ctypes.POINTER(KrProfile), _I32]),
    "kr_probe_fma": (_I32, [_I32, _I64, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "kr_set_tile_kernels": (_I32, [_I32]),
    "kr_set_fused_products": (_I32, [_I32]),
    "kr_take_device_timeouts": (_I32, [_I32, ctypes.POINTER(_I64)]),
}


def load_library(path: str = LIBPATH) -> ctypes.CDLL:
    """Load libkrylov_gb300.so and declare the C signatures; raises if it is missing."""
    if not os.path.exists(path):
        raise RuntimeError(
            "libkrylov_gb300.so is not built (%s); run paper_1504_04395_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class KrylovError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def kr_last_error() -> str:
    v = lib().kr_last_error()
    return v.decode() if v else ""


def _check(status, allow_iteration_status=False):
    if status == 0:
        return status
    if allow_iteration_status and status in (1, 2, 3, 4, 5):
        return status
    raise KrylovError(status, kr_last_error())


# ------------------------------------------------------------------------------------------
# torch marshalling
# ------------------------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _dev_ptr(t, name, dtype=None, shape=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous (row-interleaved n x s layout)" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def method_id(method) -> int:
    if isinstance(method, str):
        return METHODS[method]
    return int(method)


class Operator:
    """Device copy of a CSR matrix A and its explicit adjoint (kr_op)."""

    @classmethod
    def stencil(cls, dims, centre, minus, plus, device=None):
        """Matrix-free (2d+1)-point stencil (kr_op_create_stencil); minus/plus: one value per axis."""
        torch = _torch()
        if device is None:
            device = torch.cuda.current_device()
        d = len(dims)
        coef = [complex(centre)]
        for a in range(d):
            coef += [complex(minus[a]), complex(plus[a])]
        c = np.array([[z.real, z.imag] for z in coef], dtype=np.float64).reshape(-1)
        dm = np.ascontiguousarray(dims, dtype=np.int64)
        self = cls.__new__(cls)
        self.n = int(np.prod(dims))
        self.device = int(device)
        h = ctypes.c_void_p()
        _check(lib().kr_op_create_stencil(d, dm.ctypes.data, c.ctypes.data, self.device, ctypes.byref(h)))
        self._h = h
        self.nnz = self.info()["nnz"]
        return self

    @classmethod
    def lattice4d(cls, dims, diag, hop, gamma, links, device=None):
        """Matrix-free 4D lattice operator (kr_op_create_lattice4d).

        dims: 4 extents; diag: complex diagonal; hop: real hop coefficient; gamma: (4, 4, 4)
        complex array of the gamma matrices; links: (4, sites, 3, 3) complex array U_mu(x).
        """
        torch = _torch()
        if device is None:
            device = torch.cuda.current_device()
        dm = np.ascontiguousarray(dims, dtype=np.int64)
        if dm.shape != (4,):
            raise ValueError("dims must have 4 entries")
        sites = int(np.prod(dm))
        g = np.ascontiguousarray(np.asarray(gamma, dtype=np.complex128))
        if g.shape != (4, 4, 4):
            raise ValueError("gamma must have shape (4, 4, 4)")
        U = np.ascontiguousarray(np.asarray(links, dtype=np.complex128))
        if U.shape != (4, sites, 3, 3):
            raise ValueError("links must have shape (4, sites, 3, 3)")
        d = np.array([complex(diag).real, complex(diag).imag], dtype=np.float64)
        self = cls.__new__(cls)
        self.n = 12 * sites
        self.device = int(device)
        h = ctypes.c_void_p()
        _check(lib().kr_op_create_lattice4d(dm.ctypes.data, d.ctypes.data, float(hop), g.ctypes.data, U.ctypes.data,
                                            self.device, ctypes.byref(h)))
        self._h = h
        self.nnz = self.info()["nnz"]
        return self

    def set_preconditioner(self, kind="ilu0"):
        """Right preconditioner for later kr_solve calls: "ilu0" or None (kr_op_set_preconditioner)."""
        _check(lib().kr_op_set_preconditioner(self.handle, {None: 0, "none": 0, "ilu0": 1}[kind]))
        return self

    def __init__(self, n, rowptr, colidx, vals, device=None):
        torch = _torch()
        if device is None:
            device = torch.cuda.current_device()
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.complex128)
        self.n = int(n)
        self.nnz = int(colidx.shape[0])
        self.device = int(device)
        h = ctypes.c_void_p()
        _check(lib().kr_op_create_csr(self.n, self.nnz, rowptr.ctypes.data, colidx.ctypes.data,
                                      vals.ctypes.data, self.device, ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_tensors(cls, rowptr, colidx, vals, stream=None):
        """Operator from CSR arrays held in torch tensors (kr_op_create_csr_async): int64 rowptr,
        int32 colidx and complex128 vals, all on one CUDA device (copied on `stream`) or all on the
        host."""
        torch = _torch()
        n = int(rowptr.shape[0]) - 1
        nnz = int(colidx.shape[0])
        on_dev = rowptr.is_cuda
        if {t.is_cuda for t in (rowptr, colidx, vals)} != {on_dev}:
            raise ValueError("rowptr, colidx and vals must all be on the device or all on the host")
        for t, name, dt in ((rowptr, "rowptr", torch.int64), (colidx, "colidx", torch.int32),
                            (vals, "vals", torch.complex128)):
            if t.dtype != dt or not t.is_contiguous():
                raise TypeError("%s must be a contiguous %s tensor" % (name, dt))
        if vals.shape[0] != nnz:
            raise ValueError("vals and colidx differ in length")
        self = cls.__new__(cls)
        self.n, self.nnz = n, nnz
        h = ctypes.c_void_p()
        st = _stream(stream) if on_dev else ctypes.c_void_p(0)
        _check(lib().kr_op_create_csr_async(n, nnz, ctypes.c_void_p(rowptr.data_ptr()),
                                            ctypes.c_void_p(colidx.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                            int(on_dev), st, ctypes.byref(h)))
        self._h = h
        self.device = rowptr.device.index if on_dev else torch.cuda.current_device()
        return self

    @property
    def handle(self):
        return self._h

    def info(self):
        n, nnz, ro = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().kr_op_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(ro)))
        return {"n": n.value, "nnz": nnz.value, "real_offdiag": bool(ro.value)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kr_op_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kr_op_update_values(op: Operator, vals):
    """Replace A's stored entries (CSR order of creation); vals: complex128 numpy array or tensor."""
    torch = _torch()
    if isinstance(vals, torch.Tensor):
        v = vals.detach().to(torch.complex128).contiguous()
        if v.is_cuda:
            _check(lib().kr_op_update_values(op.handle, ctypes.c_void_p(v.data_ptr()), 1))
            return
        vals = v.numpy()
    v = np.ascontiguousarray(vals, dtype=np.complex128)
    if v.shape[0] != op.nnz:
        raise ValueError("expected %d values, got %d" % (op.nnz, v.shape[0]))
    _check(lib().kr_op_update_values(op.handle, ctypes.c_void_p(v.ctypes.data), 0))


def kr_op_create_csr(n, rowptr, colidx, vals, device=None) -> Operator:
    return Operator(n, rowptr, colidx, vals, device)


def kr_op_apply(op: Operator, V, Y=None, adjoint=False, stream=None):
    torch = _torch()
    s = V.shape[1]
    if Y is None:
        Y = torch.empty_like(V)
    _check(lib().kr_op_apply(op.handle, int(adjoint), s, _dev_ptr(V, "V", torch.complex128, (op.n, s)),
                             _dev_ptr(Y, "Y", torch.complex128, (op.n, s)), _stream(stream)))
    return Y


def kr_op_apply_reduce(op: Operator, V, U, kind="gram", Y=None, adjoint=False, stream=None, store_y=True):
    torch = _torch()
    s = V.shape[1]
    k = RED[kind] if isinstance(kind, str) else int(kind)
    if Y is None and store_y:
        Y = torch.empty_like(V)
    out = torch.empty((s, s) if k == 1 else (1,), dtype=torch.complex128, device=V.device)
    uptr = ctypes.c_void_p(0) if (U is None) else _dev_ptr(U, "U", torch.complex128)
    yptr = ctypes.c_void_p(0) if Y is None else _dev_ptr(Y, "Y", torch.complex128, (op.n, s))
    _check(lib().kr_op_apply_reduce(op.handle, int(adjoint), s, _dev_ptr(V, "V", torch.complex128, (op.n, s)),
                                    yptr, uptr, k, _dev_ptr(out, "out"), _stream(stream)))
    return Y, out


def kr_block_reduce(U, Y, kind="gram", stream=None):
    torch = _torch()
    n, s = Y.shape
    k = RED[kind] if isinstance(kind, str) else int(kind)
    out = torch.empty((s, s) if k == 1 else (1,), dtype=torch.complex128, device=Y.device)
    uptr = ctypes.c_void_p(0) if (U is None) else _dev_ptr(U, "U", torch.complex128)
    _check(lib().kr_block_reduce(n, s, uptr, _dev_ptr(Y, "Y", torch.complex128), k, _dev_ptr(out, "out"),
                                 _stream(stream)))
    return out


def kr_op_apply_reduce_c64(op: Operator, V, U=None, kind=0, Y=None, adjoint=False, stream=None, store_y=True):
    """Complex64 product Y = op(A) V with an optional fused reduction (kind 0: product only).

    V, Y, U: complex64 device tensors; the reduction result is complex128.
    """
    torch = _torch()
    s = V.shape[1]
    k = RED[kind] if isinstance(kind, str) else int(kind)
    if Y is None and (store_y or k == 0):
        Y = torch.empty_like(V)
    out = torch.empty((s, s) if k == 1 else (1,), dtype=torch.complex128, device=V.device)
    uptr = ctypes.c_void_p(0) if (U is None) else _dev_ptr(U, "U", torch.complex64)
    yptr = ctypes.c_void_p(0) if Y is None else _dev_ptr(Y, "Y", torch.complex64, (op.n, s))
    _check(lib().kr_op_apply_reduce_c64(op.handle, int(adjoint), s, _dev_ptr(V, "V", torch.complex64, (op.n, s)),
                                        yptr, uptr, k, _dev_ptr(out, "out") if k else ctypes.c_void_p(0),
                                        _stream(stream)))
    return Y, (out if k else None)


def kr_block_reduce_c64(U, Y, kind="gram", stream=None):
    """Complex64 block reduction (complex128 result)."""
    torch = _torch()
    n, s = Y.shape
    k = RED[kind] if isinstance(kind, str) else int(kind)
    out = torch.empty((s, s) if k == 1 else (1,), dtype=torch.complex128, device=Y.device)
    uptr = ctypes.c_void_p(0) if (U is None) else _dev_ptr(U, "U", torch.complex64)
    _check(lib().kr_block_reduce_c64(n, s, uptr, _dev_ptr(Y, "Y", torch.complex64), k, _dev_ptr(out, "out"),
                                     _stream(stream)))
    return out


def kr_op_apply_precond(op: Operator, V, Y=None, adjoint=False, stream=None):
    """Y = M^{-1} V (or M^{-H} V) with the operator's preconditioner (complex128 device blocks)."""
    torch = _torch()
    s = V.shape[1]
    if Y is None:
        Y = torch.empty_like(V)
    _check(lib().kr_op_apply_precond(op.handle, int(adjoint), s, _dev_ptr(V, "V", torch.complex128, (op.n, s)),
                                     _dev_ptr(Y, "Y", torch.complex128, (op.n, s)), _stream(stream)))
    return Y


def kr_block_reduce_noalloc(U, Y, out, kind="gram", stream=None):
    """kr_block_reduce into a caller-provided `out` with no device allocation by the library.

    For callers whose device memory is owned by their own allocator or who cannot
    afford an allocation in the call; s <= 16.  `out` must be a complex128 device
    tensor of shape (s, s) for "gram" and (1,) otherwise; U has shape (n, s) for
    "gram" / "trace" and (n,) for "sumv" (ignored for "norm2"); U, Y, out on one device.
    """
    torch = _torch()
    n, s = Y.shape
    k = RED[kind] if isinstance(kind, str) else int(kind)
    if k not in RED.values():
        raise ValueError("unknown reduction kind %r" % (kind,))
    yptr = _dev_ptr(Y, "Y", torch.complex128, (n, s))
    optr = _dev_ptr(out, "out", torch.complex128, (s, s) if k == RED["gram"] else (1,))
    devices = {Y.device, out.device}
    if k == RED["norm2"] or U is None:
        if k != RED["norm2"]:
            raise ValueError("U is required for reduction %r" % (kind,))
        uptr = ctypes.c_void_p(0)
    else:
        uptr = _dev_ptr(U, "U", torch.complex128, (n,) if k == RED["sumv"] else (n, s))
        devices.add(U.device)
    if len(devices) != 1:
        raise ValueError("U, Y and out must be on one device, got %s" % sorted(str(d) for d in devices))
    _check(lib().kr_block_reduce_noalloc(n, s, uptr, yptr, k, optr, _stream(stream)))
    return out


def kr_thin_qr(Z, Q=None, stream=None):
    torch = _torch()
    n, s = Z.shape
    if Q is None:
        Q = torch.empty_like(Z)
    S = torch.empty((s, s), dtype=torch.complex128, device=Z.device)
    _check(lib().kr_thin_qr(n, s, _dev_ptr(Z, "Z", torch.complex128), _dev_ptr(Q, "Q", torch.complex128),
                            _dev_ptr(S, "S"), _stream(stream)))
    return Q, S


@dataclass
class SolveInfo:
    status: str
    iters: int
    matvecs: int
    relres_recursive: float
    relres_true: float
    outer_iters: int
    history: list
    fp64_iters: int = 0
    breakdown_iter: int = 0

    @property
    def converged(self):
        return self.status == "OK"


def _options(tol, maxit, precision, inner_tol, max_outer, shadow, shadow_mode, check_every, host_buffers,
             history, time_limit_s, graphs=0, orthonormalize_B=False):
    o = KrOptions()
    lib().kr_options_default(ctypes.byref(o))
    o.tol = float(tol)
    o.maxit = int(maxit)
    o.precision = int(precision)
    o.inner_tol = float(inner_tol)
    o.max_outer = int(max_outer)
    o.shadow_mode = int(shadow_mode)
    o.shadow = shadow
    o.check_every = int(check_every)
    o.host_buffers = int(host_buffers)
    o.history = history
    o.time_limit_s = float(time_limit_s)
    o.graphs = int(graphs)
    o.orthonormalize_B = int(bool(orthonormalize_B))
    return o


def _solve(fn, op, method, B, X, tol, maxit, precision, inner_tol, max_outer, shadow, shadow_conj, check_every,
           stream, time_limit_s, graphs=0, orthonormalize_B=False):
    torch = _torch()
    n, s = B.shape
    host = not B.is_cuda
    if host:
        if B.dtype != torch.complex128 or not B.is_contiguous():
            raise TypeError("host B must be a contiguous complex128 tensor")
        if X is None:
            X = torch.zeros_like(B)
        bptr = ctypes.c_void_p(B.data_ptr())
        xptr = ctypes.c_void_p(X.data_ptr())
    else:
        bptr = _dev_ptr(B, "B", torch.complex128, (op.n, s))
        if X is None:
            X = torch.zeros_like(B)
        xptr = _dev_ptr(X, "X", torch.complex128, (op.n, s))
    hist = (ctypes.c_double * (maxit + 1))()
    mode, sptr = 0, ctypes.c_void_p(0)
    if shadow is not None:
        mode, sptr = 2, _dev_ptr(shadow, "shadow", torch.complex128)
    elif shadow_conj:
        mode = 1
    o = _options(tol, maxit, precision, inner_tol, max_outer, sptr, mode, check_every, host, hist, time_limit_s,
                 GRAPHS[graphs] if isinstance(graphs, str) else int(graphs), orthonormalize_B)
    info = KrInfo()
    st = fn(op.handle, method_id(method), s, bptr, xptr, ctypes.byref(o), _stream(stream), ctypes.byref(info))
    _check(st, allow_iteration_status=True)
    nh = (info.outer_iters if precision == FP32_REFINE else info.iters) + 1
    si = SolveInfo(status=STATUS[info.status], iters=info.iters, matvecs=info.matvecs,
                   relres_recursive=info.relres_recursive, relres_true=info.relres_true,
                   outer_iters=info.outer_iters, history=[hist[i] for i in range(min(nh, maxit + 1))],
                   fp64_iters=info.fp64_iters, breakdown_iter=info.breakdown_iter)
    return X, si


def kr_solve(op: Operator, method, B, X=None, tol=1e-8, maxit=500, precision=FP64, inner_tol=1e-4, max_outer=30,
             shadow=None, shadow_conj=False, check_every=8, stream=None, time_limit_s=0.0, graphs="auto",
             orthonormalize_B=False):
    """Solve A X = B (B: n x s complex128, CUDA or CPU tensor; X holds X_0, default 0).

    graphs: "auto" (CUDA-graph replay of the iterations for small problems), "on" or "off".
    orthonormalize_B: solve with the orthonormal factor Q of B - A X_0 = Q S (Sec. 5) and map back.
    """
    return _solve(lib().kr_solve, op, method, B, X, tol, maxit, precision, inner_tol, max_outer, shadow,
                  shadow_conj, check_every, stream, time_limit_s, graphs, orthonormalize_B)


def kr_adjoint_solve(op: Operator, method, G, Lam=None, tol=1e-8, maxit=500, precision=FP64, inner_tol=1e-4,
                     max_outer=30, shadow=None, shadow_conj=False, check_every=8, stream=None, time_limit_s=0.0,
                     graphs="auto", orthonormalize_B=False):
    """Solve A^H Lambda = G with the same simultaneous methods."""
    return _solve(lib().kr_adjoint_solve, op, method, G, Lam, tol, maxit, precision, inner_tol, max_outer, shadow,
                  shadow_conj, check_every, stream, time_limit_s, graphs, orthonormalize_B)


def kr_grad_values(op: Operator, Lam, X, stream=None):
    """dL/dA_ij = -sum_c Lambda_ic conj(X_jc) on the stored pattern (CSR order as given)."""
    torch = _torch()
    s = X.shape[1]
    dv = torch.empty(op.nnz, dtype=torch.complex128, device=X.device)
    _check(lib().kr_grad_values(op.handle, s, _dev_ptr(Lam, "Lambda", torch.complex128, (op.n, s)),
                                _dev_ptr(X, "X", torch.complex128, (op.n, s)), _dev_ptr(dv, "dvals"),
                                _stream(stream)))
    return dv


def kr_profile_enable(enable=True, time_kernels=False):
    _check(lib().kr_profile_enable(int(enable), int(time_kernels)))


def kr_set_column_pairs(enable=True):
    """Run complex64 launches with even s on the two-columns-per-thread kernels (default on)."""
    _check(lib().kr_set_column_pairs(int(bool(enable))))


def kr_set_tile_kernels(enable=True):
    """Run complex64 CSR products on the TMA-staged row-tile kernel where it applies (default on)."""
    _check(lib().kr_set_tile_kernels(int(bool(enable))))


def kr_set_fused_products(enable=True):
    """Gl-/eGl-BiCG with alpha from the adjoint product and the update fused with A P (default on)."""
    _check(lib().kr_set_fused_products(int(bool(enable))))


def kr_take_device_timeouts(reset=True):
    """Bounded device waits of the tile kernels that ran out since the last reset (0 normally)."""
    c = ctypes.c_int64()
    _check(lib().kr_take_device_timeouts(int(bool(reset)), ctypes.byref(c)))
    return c.value


def kr_set_lattice_rows_per_thread(rows=0):
    """Matrix-free lattice kernel: 4 rows per thread, 12 (whole sites) or 0 (default per precision)."""
    _check(lib().kr_set_lattice_rows_per_thread(int(rows)))


def kr_probe_fma(precision="fp64", iters=1 << 19, stream=None):
    """Launch the FMA-throughput probe once; returns (flops of the launch, device buffer).  Time it
    with CUDA events on `stream` to obtain the FP64 (or "fp32") FMA rate."""
    torch = _torch()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    fl = ctypes.c_double()
    _check(lib().kr_probe_fma(0 if precision == "fp64" else 2, int(iters), ctypes.c_void_p(out.data_ptr()),
                              ctypes.byref(fl), _stream(stream)))
    return fl.value, out


def kr_profile_read(reset=False):
    """Per kernel class: launches, summed CUDA-event ms, algorithmic flops and bytes."""
    p = KrProfile()
    _check(lib().kr_profile_read(ctypes.byref(p), int(reset)))
    return {name: {"launches": p.launches[i], "ms": p.ms[i], "flops": p.flops[i], "bytes": p.bytes[i]}
            for i, name in enumerate(KERNEL_CLASSES)}


solve = kr_solve
adjoint_solve = kr_adjoint_solve

__all__ = [
    "METHODS", "STATUS", "Operator", "SolveInfo", "KrylovError", "lib", "load_library",
    "kr_op_create_csr", "kr_op_update_values", "kr_op_apply", "kr_op_apply_reduce", "kr_block_reduce", "kr_thin_qr",
    "kr_solve", "kr_adjoint_solve", "kr_grad_values", "kr_last_error", "solve", "adjoint_solve",
    "FP64", "FP32_REFINE", "kr_profile_enable", "kr_profile_read", "kr_set_column_pairs", "kr_op_apply_precond", "kr_set_lattice_rows_per_thread", "kr_op_apply_reduce_c64", "kr_block_reduce_c64", "KERNEL_CLASSES", "kr_block_reduce_noalloc",
    "kr_probe_fma", "kr_set_tile_kernels", "kr_take_device_timeouts", "kr_set_fused_products",
]
