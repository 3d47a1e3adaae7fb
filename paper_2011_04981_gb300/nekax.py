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
AX_FF_ENERGY = 2  # the element-energy form, for nek_set_ax_epb / nek_get_ax_epb
AX_OZ = 3  # FP64-accurate with the contractions on the tensor cores (Gff: the split of nek_geom_oz)


class NekCgOpts(ctypes.Structure):
    _fields_ = [("check_every", ctypes.c_int), ("time_ax", ctypes.c_int), ("ax_ms_total", ctypes.c_double),
                ("ax_launches", ctypes.c_int), ("kernel_launches", ctypes.c_int), ("ax_impl", ctypes.c_int),
                ("Gff", ctypes.c_void_p)]


class NekBatchStats(ctypes.Structure):
    _fields_ = [("iterations_run", ctypes.c_int), ("converged", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("graph_launches", ctypes.c_int)]


class NekFcgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("relres", ctypes.c_double), ("fell_back_at", ctypes.c_int),
                ("net_applications", ctypes.c_int), ("net_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int)]


class NekMixedInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("relres", ctypes.c_double),
                ("kernel_launches", ctypes.c_int)]


PREC_F32 = 0
PREC_BF16 = 1
PREC_F16 = 2

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
    "nek_ax_ff_energy": ([_I64, _I, _P, _P, _P, _P, _P, _P], _I),
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
    "nek_residual": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "nek_cg_workspace_bytes": ([_I64, _I, _I], ctypes.c_size_t),
    "nek_batch_create": ([_I, _P, _P, _P, ctypes.POINTER(_P)], _I),
    "nek_batch_destroy": ([_P], _I),
    "nek_batch_info": ([_P, _P, _P, _P], _I),
    "nek_batch_gs": ([_P], _P),
    "nek_batch_workspace_bytes": ([_P, _I], ctypes.c_size_t),
    "nek_batch_jacobi_minv": ([_P, _P, _P, _P, _P], _I),
    "nek_batch_cg_solve": ([_P, _P, _P, _P, _P, _P, _P, _D, _I, _I, _P, _P, _P, _P, ctypes.POINTER(NekBatchStats),
                            _P], _I),
    "nek_net_param_count": ([], _I),
    "nek_net_prep": ([_I64, _I, _P, _P, _P, _P, _P], _I),
    "nek_net_target": ([_I64, _I, _P, _P, _P, _P, _P], _I),
    "nek_net_apply": ([_I64, _I, _P, _P, _P, _P, _P, _P], _I),
    "nek_net_apply_bf16": ([_I64, _I, _P, _P, _P, _P, _P, _P], _I),
    "nek_net_apply_bf16_mma": ([_I64, _I, _P, _P, _P, _P, _P, _P], _I),
    "nek_net_tc_selftest": ([_I, _I64, ctypes.POINTER(_I)], _I),
    "nek_ax_oz": ([_I64, _I, _P, _P, _P, _P, _P], _I),
    "nek_geom_oz": ([_I64, _I, _P, _P, _P], _I),
    "nek_ax_oz_selftest": ([_I, _I64, ctypes.POINTER(_I)], _I),
    "nek_net_train_workspace_bytes": ([_I], ctypes.c_size_t),
    "nek_net_forward_batch": ([_I, _P, _P, _P, _P, _P], _I),
    "nek_net_train_grad": ([_I, _P, _P, _P, _P, _P, _P, _P], _I),
    "nek_net_train_grad_energy": ([_I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "nek_adam_step": ([_I, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I, _P],
                      _I),
    "nek_fcg_workspace_bytes": ([_I64, _I, _I], ctypes.c_size_t),
    "nek_fcg_solve": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _P, _P, _D, _I, _I, _D, _P, ctypes.POINTER(NekFcgInfo),
                       _P], _I),
    "nek_fcg_trunc_workspace_bytes": ([_I64, _I, _I, _I], ctypes.c_size_t),
    "nek_fcg_solve_trunc": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _P, _P, _D, _I, _I, _I, _D, _P,
                             ctypes.POINTER(NekFcgInfo), _P], _I),
    "nek_tune_ax": ([_I, _I64, _I, _P, _P, _P, _P, _P, _P, _P], _I),
    "nek_set_ax_epb": ([_I, _I, _I], _I),
    "nek_get_ax_epb": ([_I, _I], _I),
    "nek_lowp_bytes_per_value": ([_I], ctypes.c_size_t),
    "nek_geom_lowp": ([_I64, _I, _I, _P, _P, _P, _P], _I),
    "nek_ax_lowp": ([_I64, _I, _I, _P, _P, _P, _P, _P, _P], _I),
    "nek_ax_lowp_tc": ([_I64, _I, _I, _P, _P, _P, _P, _P, _P], _I),
    "nek_ax_lowp_tc5": ([_I64, _I, _I, _P, _P, _P, _P, _P, _P], _I),
    "nek_cg_mixed_workspace_bytes": ([_I64, _I, _I], ctypes.c_size_t),
    "nek_cg_solve_mixed": ([_P, _I64, _I, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P, _D, _D, _I, _I, _P,
                            ctypes.POINTER(NekMixedInfo), _P], _I),
    "nek_cg_solve": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P, _P, _P], _I),
    "nek_cg_solve_ex": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P, _P, ctypes.POINTER(NekCgOpts), _P],
                        _I),
    "nek_cg_host_staging_bytes": ([_I64, _I], ctypes.c_size_t),
    "nek_cg_solve_host": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P, _P, _P, ctypes.POINTER(NekCgOpts),
                           _P], _I),
    "nek_lvec_create": ([_I64, _P, _P, ctypes.POINTER(_P)], _I),
    "nek_lvec_destroy": ([_P], _I),
    "nek_lvec_size": ([_P], _I64),
    "nek_lvec_scatter": ([_P, _P, _P, _P], _I),
    "nek_lvec_restrict": ([_P, _P, _P, _P], _I),
    "nek_lvec_assemble": ([_P, _P, _P, _P], _I),
    "nek_lvec_ax_ff": ([_P, _I64, _I, _P, _P, _P, _P, _P, _P], _I),
    "nek_lvec_jacobi_minv": ([_P, _I64, _I, _P, _P, _P, _P, _P], _I),
    "nek_lvec_cg_workspace_bytes": ([_P], ctypes.c_size_t),
    "nek_lvec_cg_solve": ([_P, _I64, _I, _P, _P, _P, _P, _P, _D, _I, _P, _P, _P, ctypes.POINTER(NekCgOpts), _P],
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


def geom_oz(nelt, nx, G, Goz, stream=None):
    """G split into float pairs, two adjacent points interleaved (the layout nek_ax_oz reads)."""
    _check("nek_geom_oz", load().nek_geom_oz(nelt, nx, _ptr(G), _ptr(Goz), _stream(stream)))


def ax_oz(nelt, nx, D, Goz, u, w, stream=None):
    """w = AX u to FP64 accuracy with the contractions on the tensor cores (BF16 digits)."""
    _check("nek_ax_oz", load().nek_ax_oz(nelt, nx, _ptr(D), _ptr(Goz), _ptr(u), _ptr(w), _stream(stream)))


def ax_oz_selftest(force_timeout, wait_us):
    """(status, timed_out) of the operator kernel's bounded-wait self-test."""
    t = ctypes.c_int(0)
    st = load().nek_ax_oz_selftest(int(force_timeout), int(wait_us), ctypes.byref(t))
    return st, t.value


def ax_ff_energy(nelt, nx, D, Gff, u, w, edot, stream=None):
    """w = AX u (float-float) and edot[e] = u_e . w_e."""
    _check("nek_ax_ff_energy", load().nek_ax_ff_energy(nelt, nx, _ptr(D), _ptr(Gff), _ptr(u), _ptr(w), _ptr(edot),
                                                       _stream(stream)))


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


def tune_ax(impl, nelt, nx, D, Gx, u, w, stream=None):
    """Time the elements-per-CTA variants and keep the fastest; returns (epb, ms)."""
    e = _I(0)
    ms = ctypes.c_float(0.0)
    _check("nek_tune_ax", load().nek_tune_ax(int(impl), nelt, nx, _ptr(D), _ptr(Gx), _ptr(u), _ptr(w),
                                             ctypes.byref(e), ctypes.byref(ms), _stream(stream)))
    return e.value, ms.value


def set_ax_epb(impl, nx, epb):
    _check("nek_set_ax_epb", load().nek_set_ax_epb(int(impl), nx, epb))


def get_ax_epb(impl, nx):
    return load().nek_get_ax_epb(int(impl), nx)


def geom_lowp(nelt, nx, precision, G, Glp, gscale, stream=None):
    _check("nek_geom_lowp", load().nek_geom_lowp(nelt, nx, precision, _ptr(G), _ptr(Glp), _ptr(gscale),
                                                 _stream(stream)))


def ax_lowp(nelt, nx, precision, D, Glp, gscale, u, w, stream=None):
    _check("nek_ax_lowp", load().nek_ax_lowp(nelt, nx, precision, _ptr(D), _ptr(Glp), _ptr(gscale), _ptr(u),
                                             _ptr(w), _stream(stream)))


def ax_lowp_tc(nelt, nx, precision, D, Glp, gscale, u, w, stream=None):
    _check("nek_ax_lowp_tc", load().nek_ax_lowp_tc(nelt, nx, int(precision), _ptr(D), _ptr(Glp), _ptr(gscale),
                                                   _ptr(u), _ptr(w), _stream(stream)))


def ax_lowp_tc5(nelt, nx, precision, D, Glp, gscale, u, w, stream=None):
    """The reduced-precision operator with its contractions as tcgen05 MMAs (BF16 / FP16, nx 2..11)."""
    _check("nek_ax_lowp_tc5", load().nek_ax_lowp_tc5(nelt, nx, int(precision), _ptr(D), _ptr(Glp), _ptr(gscale),
                                                     _ptr(u), _ptr(w), _stream(stream)))


def cg_solve_mixed(gs, nelt, nx, D, G, Gff, precision, Glp, gscale, m, minv, f, x, tol=1e-8, inner_tol=1e-2,
                   max_outer=50, max_inner=5000, workspace=None, stream=None):
    """FP64 defect correction with reduced-precision inner PCG; returns dict(status, outer, inner, relres)."""
    info = NekMixedInfo()
    st = load().nek_cg_solve_mixed(gs.handle, nelt, nx, _ptr(D), _ptr(G), _ptr(Gff), int(precision), _ptr(Glp),
                                   _ptr(gscale), _ptr(m), _ptr(minv), _ptr(f), _ptr(x), float(tol),
                                   float(inner_tol), int(max_outer), int(max_inner), _ptr(workspace),
                                   ctypes.byref(info), _stream(stream))
    if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        raise NekError("nek_cg_solve_mixed", st)
    return dict(status=st, outer=info.outer_iters, inner=info.inner_iters, relres=info.relres,
                kernel_launches=info.kernel_launches)


class BatchPlan:
    """Owning wrapper of a ``nek_batch*``: problems must be given sorted by nx."""

    def __init__(self, nelts, nxs, glo_concat):
        self.nprob = len(nelts)
        ne = np.ascontiguousarray(nelts, dtype=np.int64)
        nx = np.ascontiguousarray(nxs, dtype=np.int32)
        glo = np.ascontiguousarray(glo_concat, dtype=np.int64).reshape(-1)
        h = _P()
        _check("nek_batch_create", load().nek_batch_create(self.nprob, ne.ctypes.data, nx.ctypes.data,
                                                           glo.ctypes.data, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h.value

    def info(self):
        a, b, c = _I64(), _I(), _I()
        _check("nek_batch_info", load().nek_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def gs_handle(self):
        return load().nek_batch_gs(self._h)

    def workspace_bytes(self, need_minv=True):
        return int(load().nek_batch_workspace_bytes(self._h, 1 if need_minv else 0))

    def jacobi_minv(self, G, m, minv, stream=None):
        _check("nek_batch_jacobi_minv", load().nek_batch_jacobi_minv(self._h, _ptr(G), _ptr(m), _ptr(minv),
                                                                     _stream(stream)))

    def cg_solve(self, G, Gff, m, minv, f, x, tol=1e-8, max_iter=1000, iters_per_graph=10, workspace=None,
                 stream=None):
        it = np.zeros(self.nprob, dtype=np.int32)
        rr = np.zeros(self.nprob)
        stv = np.zeros(self.nprob, dtype=np.int32)
        stats = NekBatchStats()
        st = load().nek_batch_cg_solve(self._h, _ptr(G), _ptr(Gff), _ptr(m), _ptr(minv), _ptr(f), _ptr(x),
                                       float(tol), int(max_iter), int(iters_per_graph), _ptr(workspace),
                                       it.ctypes.data, rr.ctypes.data, stv.ctypes.data, ctypes.byref(stats),
                                       _stream(stream))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            raise NekError("nek_batch_cg_solve", st)
        return dict(status=st, iters=it, relres=rr, statuses=stv, iterations_run=stats.iterations_run,
                    converged=stats.converged, kernel_launches=stats.kernel_launches,
                    graph_launches=stats.graph_launches)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().nek_batch_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def net_param_count():
    return int(load().nek_net_param_count())


def net_prep(nelt, nx, r, minv, xin, scale, stream=None):
    _check("nek_net_prep", load().nek_net_prep(nelt, nx, _ptr(r), _ptr(minv), _ptr(xin), _ptr(scale),
                                               _stream(stream)))


def net_target(nelt, nx, xs, xk, scale, target, stream=None):
    _check("nek_net_target", load().nek_net_target(nelt, nx, _ptr(xs), _ptr(xk), _ptr(scale), _ptr(target),
                                                   _stream(stream)))


def net_apply(nelt, nx, theta, xin, scale, c, z, stream=None):
    _check("nek_net_apply", load().nek_net_apply(nelt, nx, _ptr(theta), _ptr(xin), _ptr(scale), _ptr(c), _ptr(z),
                                                 _stream(stream)))


def net_apply_bf16(nelt, nx, theta, xin, scale, c, z, stream=None):
    _check("nek_net_apply_bf16", load().nek_net_apply_bf16(nelt, nx, _ptr(theta), _ptr(xin), _ptr(scale), _ptr(c),
                                                           _ptr(z), _stream(stream)))


def net_apply_bf16_mma(nelt, nx, theta, xin, scale, c, z, stream=None):
    _check("nek_net_apply_bf16_mma", load().nek_net_apply_bf16_mma(nelt, nx, _ptr(theta), _ptr(xin), _ptr(scale),
                                                                   _ptr(c), _ptr(z), _stream(stream)))


def net_train_workspace_bytes(batch):
    return int(load().nek_net_train_workspace_bytes(batch))


def net_forward_batch(batch, theta, xin, y, workspace, stream=None):
    _check("nek_net_forward_batch", load().nek_net_forward_batch(batch, _ptr(theta), _ptr(xin), _ptr(y),
                                                                 _ptr(workspace), _stream(stream)))


def net_train_grad(batch, theta, xin, target, grad, loss, workspace, stream=None):
    _check("nek_net_train_grad", load().nek_net_train_grad(batch, _ptr(theta), _ptr(xin), _ptr(target), _ptr(grad),
                                                           _ptr(loss), _ptr(workspace), _stream(stream)))


def net_train_grad_energy(batch, theta, xin, target, D, Glp32, gscale, grad, loss, workspace, stream=None):
    _check("nek_net_train_grad_energy", load().nek_net_train_grad_energy(
        batch, _ptr(theta), _ptr(xin), _ptr(target), _ptr(D), _ptr(Glp32), _ptr(gscale), _ptr(grad), _ptr(loss),
        _ptr(workspace), _stream(stream)))


def adam_step(n, theta, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check("nek_adam_step", load().nek_adam_step(n, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), float(lr),
                                                 float(beta1), float(beta2), float(eps), int(step), _stream(stream)))


def fcg_solve(gs, nelt, nx, D, G, Gff, m, minv, theta, f, x, tol=1e-8, max_iter=5000, stag_window=100,
              stag_factor=0.5, workspace=None, stream=None, truncation=1):
    """Truncated flexible CG, FCG(truncation) (nek_fcg_solve_trunc); truncation = 1 is nek_fcg_solve."""
    info = NekFcgInfo()
    st = load().nek_fcg_solve_trunc(gs.handle, nelt, nx, _ptr(D), _ptr(G), _ptr(Gff), _ptr(m), _ptr(minv),
                                    _ptr(theta), _ptr(f), _ptr(x), float(tol), int(max_iter), int(truncation),
                                    int(stag_window), float(stag_factor), _ptr(workspace), ctypes.byref(info),
                                    _stream(stream))
    if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        raise NekError("nek_fcg_solve_trunc", st)
    return dict(status=st, iters=info.iters, relres=info.relres, fell_back_at=info.fell_back_at,
                net_applications=info.net_applications, net_ms=info.net_ms, kernel_launches=info.kernel_launches)


def residual(gs: GsPlan, nelt, nx, D, G, Gff, m, f, x, r, stream=None):
    """r = mask.(f - dssum(AX x)) (nek_residual)."""
    _check("nek_residual", load().nek_residual(gs.handle, nelt, nx, _ptr(D), _ptr(G), _ptr(Gff), _ptr(m), _ptr(f),
                                               _ptr(x), _ptr(r), _stream(stream)))


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


def cg_host_staging_bytes(nelt, nx):
    return int(load().nek_cg_host_staging_bytes(nelt, nx))


def cg_solve_host(gs: GsPlan, nelt, nx, D, G, m, minv, f_host, x_host, tol=1e-8, max_iter=1000, workspace=None,
                  staging=None, check_every=1, time_ax=False, stream=None, ax_impl=AX_FP64, Gff=None):
    """Jacobi-PCG with f and x in host memory (nek_cg_solve_host: the library copies f in and x out)."""
    it = _I(0)
    rr = _D(0.0)
    opts = NekCgOpts(check_every, 1 if time_ax else 0, 0.0, 0, 0, int(ax_impl), _ptr(Gff))
    st = load().nek_cg_solve_host(gs.handle, nelt, nx, _ptr(D), _ptr(G), _ptr(m), _ptr(minv), _ptr(f_host),
                                  _ptr(x_host), float(tol), int(max_iter), _ptr(workspace), _ptr(staging),
                                  ctypes.byref(it), ctypes.byref(rr), ctypes.byref(opts), _stream(stream))
    if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        raise NekError("nek_cg_solve_host", st)
    return dict(status=st, iters=it.value, relres=rr.value, ax_ms_total=opts.ax_ms_total,
                ax_launches=opts.ax_launches, kernel_launches=opts.kernel_launches)


class LvecPlan:
    """Owning wrapper of a ``nek_lvec*`` plan (unique-node vectors, ascending global id)."""

    def __init__(self, glo_num, mask):
        glo = np.ascontiguousarray(glo_num, dtype=np.int64).reshape(-1)
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        if m.shape != glo.shape:
            raise ValueError("glo_num and mask differ in size")
        h = _P()
        _check("nek_lvec_create", load().nek_lvec_create(glo.shape[0], glo.ctypes.data, m.ctypes.data,
                                                         ctypes.byref(h)))
        self._h = h
        self.npts = glo.shape[0]
        self.size = int(load().nek_lvec_size(h))

    @property
    def handle(self):
        return self._h.value

    def scatter(self, uL, uE, stream=None):
        _check("nek_lvec_scatter", load().nek_lvec_scatter(self._h, _ptr(uL), _ptr(uE), _stream(stream)))

    def restrict(self, uE, uL, stream=None):
        _check("nek_lvec_restrict", load().nek_lvec_restrict(self._h, _ptr(uE), _ptr(uL), _stream(stream)))

    def assemble(self, wE, wL, stream=None):
        _check("nek_lvec_assemble", load().nek_lvec_assemble(self._h, _ptr(wE), _ptr(wL), _stream(stream)))

    def ax_ff(self, nelt, nx, D, Gff, uL, wL, wE, stream=None):
        _check("nek_lvec_ax_ff", load().nek_lvec_ax_ff(self._h, nelt, nx, _ptr(D), _ptr(Gff), _ptr(uL), _ptr(wL),
                                                       _ptr(wE), _stream(stream)))

    def jacobi_minv(self, nelt, nx, D, G, minvL, scratchE, stream=None):
        _check("nek_lvec_jacobi_minv", load().nek_lvec_jacobi_minv(self._h, nelt, nx, _ptr(D), _ptr(G), _ptr(minvL),
                                                                   _ptr(scratchE), _stream(stream)))

    def workspace_bytes(self):
        return int(load().nek_lvec_cg_workspace_bytes(self._h))

    def cg_solve(self, nelt, nx, D, Gff, minvL, fL, xL, tol=1e-8, max_iter=1000, workspace=None, check_every=1,
                 time_ax=False, stream=None):
        """Jacobi-PCG on unique-node vectors; returns the dict of :func:`cg_solve`."""
        it = _I(0)
        rr = _D(0.0)
        opts = NekCgOpts(check_every, 1 if time_ax else 0, 0.0, 0, 0, AX_FF, None)
        st = load().nek_lvec_cg_solve(self._h, nelt, nx, _ptr(D), _ptr(Gff), _ptr(minvL), _ptr(fL), _ptr(xL),
                                      float(tol), int(max_iter), _ptr(workspace), ctypes.byref(it), ctypes.byref(rr),
                                      ctypes.byref(opts), _stream(stream))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            raise NekError("nek_lvec_cg_solve", st)
        return dict(status=st, iters=it.value, relres=rr.value, ax_ms_total=opts.ax_ms_total,
                    ax_launches=opts.ax_launches, kernel_launches=opts.kernel_launches)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().nek_lvec_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
