"""Thin Python binding of libnekax.so (ctypes; argument marshalling only).

Every function forwards to the C entry point of the same name in
``include/nekax.h``; all arithmetic happens in the library's CUDA kernels.
Array arguments may be torch tensors (their ``data_ptr()`` is passed), raw
integer addresses, or ``None`` for a NULL pointer.  ``stream`` defaults to the
current torch CUDA stream.  A non-OK status raises :class:`NekError`, except the
solver statuses NOT_CONVERGED and BREAKDOWN, which ``cg_solve`` returns.

There is no fallback: if the library has not been built, importing
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnekax.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_UNSUPPORTED_NX = 2
ERR_CUDA = 3
ERR_NOT_CONVERGED = 4
ERR_BREAKDOWN = 5
ERR_TIMEOUT = 6
ERR_NOMEM = 7
ERR_TOO_LARGE = 8


class NekError(RuntimeError):
    def __init__(self, func, status):
        self.status = status
        detail = ""
        if status == ERR_CUDA:
            detail = ": " + load().nek_last_error().decode()
        super().__init__("%s failed with %s%s" % (func, load().nek_status_string(status).decode(), detail))


AX_FP64 = 0
AX_FF = 1


class NekCgOpts(ctypes.Structure):
    _fields_ = [("check_every", ctypes.c_int), ("time_ax", ctypes.c_int), ("ax_ms_total", ctypes.c_double),
                ("ax_launches", ctypes.c_int), ("kernel_launches", ctypes.c_int), ("ax_impl", ctypes.c_int),
                ("Gff", ctypes.c_void_p)]


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "nek_status_string": ([_I], ctypes.c_char_p),
    "nek_last_error": ([], ctypes.c_char_p),
    "nek_version": ([], _I),
    "nek_gll": ([_I, _P, _P, _P], _I),
    "nek_geom": ([_I64, _I, _P, _P, _P], _I),
    "nek_ax": ([_I64, _I, _P, _P, _P, _P, _P], _I),
    "nek_geom_ff": ([_I64, _I, _P, _P, _P], _I),
    "nek_ax_ff": ([_I64, _I, _P, _P, _P, _P, _P], _I),
    "nek_gs_create": ([_I64, _I, _P, ctypes.POINTER(_P)], _I),
    "nek_gs_destroy": ([_P], _I),
    "nek_gs_info": ([_P, _P, _P, _P], _I),
    "nek_gs_export": ([_P, _P, _P], _I),
    "nek_dssum": ([_P, _P, _P], _I),
    "nek_gs_inv_multiplicity": ([_P, _P, _P], _I),
    "nek_mask": ([_I64, _P, _P, _P], _I),
    "nek_jacobi_minv": ([_P, _I64, _I, _P, _P, _P, _P, _P], _I),
    "nek_dot_c": ([_P, _P, _P, _P, _P], _I),
    "nek_dot_c_noalloc": ([_I64, _P, _P, _P, _P, _P], _I),
    "nek_cg_workspace_bytes": ([_I64, _I, _I], ctypes.c_size_t),
    "nek_cg_solve": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P, _P, _P], _I),
    "nek_cg_solve_ex": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P, _P, ctypes.POINTER(NekCgOpts), _P],
                        _I),
}


def load():
    """Load libnekax.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libnekax.so is not built (run __graft_entry__.build()); there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot pass %r as a pointer" % type(x))


def _stream(stream):
    if stream is None:
        import torch

        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(name, st):
    if st != OK:
        raise NekError(name, st)


def status_string(st: int) -> str:
    return load().nek_status_string(st).decode()


def version() -> int:
    return load().nek_version()


def gll(nx: int):
    """(xi, rho, D) numpy arrays computed by the library's host GLL routine."""
    xi = np.empty(nx)
    rho = np.empty(nx)
    D = np.empty((nx, nx))
    _check("nek_gll", load().nek_gll(nx, xi.ctypes.data, rho.ctypes.data, D.ctypes.data))
    return xi, rho, D


def geom(nelt, nx, corners, G, stream=None):
    _check("nek_geom", load().nek_geom(nelt, nx, _ptr(corners), _ptr(G), _stream(stream)))


def ax(nelt, nx, D, G, u, w, stream=None):
    _check("nek_ax", load().nek_ax(nelt, nx, _ptr(D), _ptr(G), _ptr(u), _ptr(w), _stream(stream)))


def geom_ff(nelt, nx, G, Gff, stream=None):
    _check("nek_geom_ff", load().nek_geom_ff(nelt, nx, _ptr(G), _ptr(Gff), _stream(stream)))


def ax_ff(nelt, nx, D, Gff, u, w, stream=None):
    _check("nek_ax_ff", load().nek_ax_ff(nelt, nx, _ptr(D), _ptr(Gff), _ptr(u), _ptr(w), _stream(stream)))


def mask(n, m, v, stream=None):
    _check("nek_mask", load().nek_mask(n, _ptr(m), _ptr(v), _stream(stream)))


class GsPlan:
    """Owning wrapper of a ``nek_gs*`` plan."""

    def __init__(self, nelt, nx, glo_num):
        glo = np.ascontiguousarray(glo_num, dtype=np.int64).reshape(-1)
        h = _P()
        _check("nek_gs_create", load().nek_gs_create(nelt, nx, glo.ctypes.data, ctypes.byref(h)))
        self._h = h
        self.nelt, self.nx = nelt, nx

    @property
    def handle(self):
        return self._h.value

    def info(self):
        a, b, c = _I64(), _I64(), _I64()
        _check("nek_gs_info", load().nek_gs_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def export(self):
        npts, ng, ns = self.info()
        off = np.empty(ng + 1, dtype=np.int64)
        mem = np.empty(max(ns, 1), dtype=np.int64)
        _check("nek_gs_export", load().nek_gs_export(self._h, off.ctypes.data, mem.ctypes.data))
        return off, mem[:ns]

    def dssum(self, v, stream=None):
        _check("nek_dssum", load().nek_dssum(self._h, _ptr(v), _stream(stream)))

    def inv_multiplicity(self, c, stream=None):
        _check("nek_gs_inv_multiplicity", load().nek_gs_inv_multiplicity(self._h, _ptr(c), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().nek_gs_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def jacobi_minv(gs: GsPlan, nelt, nx, D, G, m, minv, stream=None):
    _check("nek_jacobi_minv", load().nek_jacobi_minv(gs.handle, nelt, nx, _ptr(D), _ptr(G), _ptr(m), _ptr(minv),
                                                     _stream(stream)))


def dot_c(gs: GsPlan, a, b, result, stream=None):
    _check("nek_dot_c", load().nek_dot_c(gs.handle, _ptr(a), _ptr(b), _ptr(result), _stream(stream)))


def dot_c_noalloc(n, c, a, b, result, stream=None):
    """nek_dot_c_noalloc: the weighted dot with library-resident scratch (no allocation)."""
    _check("nek_dot_c_noalloc", load().nek_dot_c_noalloc(n, _ptr(c), _ptr(a), _ptr(b), _ptr(result),
                                                         _stream(stream)))


def cg_workspace_bytes(nelt, nx, need_minv=True) -> int:
    return int(load().nek_cg_workspace_bytes(nelt, nx, 1 if need_minv else 0))


def cg_solve(gs: GsPlan, nelt, nx, D, G, m, minv, f, x, tol=1e-8, max_iter=1000, workspace=None, check_every=1,
             time_ax=False, stream=None, ax_impl=AX_FP64, Gff=None):
    """Jacobi-PCG; returns dict(status, iters, relres, ax_ms_total, ax_launches, kernel_launches)."""
    it = _I(0)
    rr = _D(0.0)
    opts = NekCgOpts(check_every, 1 if time_ax else 0, 0.0, 0, 0, int(ax_impl), _ptr(Gff))
    st = load().nek_cg_solve_ex(gs.handle, nelt, nx, _ptr(D), _ptr(G), _ptr(m), _ptr(minv), _ptr(f), _ptr(x),
                                float(tol), int(max_iter), _ptr(workspace), ctypes.byref(it), ctypes.byref(rr),
                                ctypes.byref(opts), _stream(stream))
    if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        raise NekError("nek_cg_solve", st)
    return dict(status=st, iters=it.value, relres=rr.value, ax_ms_total=opts.ax_ms_total,
                ax_launches=opts.ax_launches, kernel_launches=opts.kernel_launches)
