"""Oracle front end: builds and loads the plain-C oracle and adds the dense
brute-force forms (numpy) used on tiny meshes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never touches the
CUDA library.

Functions and the passages they follow (arXiv 2011.04981):

* ``gll``            -- textbook GLL rule and derivative matrix (paper silent; input dxm1 of Listing 1)
* ``geom``           -- 6 symmetric geometric factors x quadrature weight (paper silent; g of Listing 1)
* ``ax``             -- ax / ax_e / local_grad3 / local_grad3_t, Section II-B, Listing 1
* ``element_matrix`` -- dense element operator from the bilinear form (brute force of Listing 1)
* ``gs_build``/``dssum`` -- nearest-neighbour exchange of Section II-B read as direct stiffness summation
* ``jacobi_minv``    -- the basic preconditioner of Section II-B, read as Jacobi
* ``pcg``            -- the CG solve of Section II-B
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

from . import gll as _gll

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nekref.c")
_SO = os.path.join(_HERE, "_nekref.so")
_SO_OMP = os.path.join(_HERE, "_nekref_omp.so")

OK, INVALID, NOT_CONVERGED, BREAKDOWN, NOMEM = 0, 1, 4, 5, 7

_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the C oracle (plain gcc, no FMA contraction).  openmp=True builds
    the same source with -fopenmp into a second library, used only to time the
    oracle on all host cores (same operations in the same order, see nekref.c)."""
    so = _SO_OMP if openmp else _SO
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"] + \
              (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


def openmp_library():
    """Path of the -fopenmp build of the oracle (built on first use), or None
    when this host's compiler cannot build it."""
    try:
        return build(openmp=True)
    except (OSError, subprocess.CalledProcessError):
        return None


def _open(path):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    D = ctypes.c_double
    lib.ref_geom.argtypes = [I64, I, P, P, P, P, P]
    lib.ref_geom.restype = I64
    lib.ref_ax.argtypes = [I64, I, P, P, P, P]
    lib.ref_ax.restype = I
    lib.ref_gs_build.argtypes = [I64, P, P, P]
    lib.ref_gs_build.restype = I64
    lib.ref_dssum.argtypes = [I64, P, P, P]
    lib.ref_dssum.restype = None
    lib.ref_inv_multiplicity.argtypes = [I64, I64, P, P, P]
    lib.ref_inv_multiplicity.restype = None
    lib.ref_mask.argtypes = [I64, P, P]
    lib.ref_mask.restype = None
    lib.ref_diag_local.argtypes = [I64, I, P, P, P]
    lib.ref_diag_local.restype = None
    lib.ref_jacobi_minv.argtypes = [I64, I, P, P, I64, P, P, P, P]
    lib.ref_jacobi_minv.restype = I
    lib.ref_pcg.argtypes = [I64, I, P, P, I64, P, P, P, P, P, P, D, I, P, P, P]
    lib.ref_pcg.restype = I
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _open(_SO)
    return _lib


@contextlib.contextmanager
def using_library(so_path):
    """Route every oracle call through another build of nekref.c (used by the
    tests that plant mistakes in a copy of the oracle to show the pins catch them)."""
    global _lib
    old = _lib
    _lib = _open(so_path)
    try:
        yield
    finally:
        _lib = old


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- GLL
def gll(nx: int):
    """(xi, rho, D) with D[i, l] = l_l'(xi_i)."""
    return _gll.gll(nx)


# ----------------------------------------------------------------------------- geometry
def geom(corners: np.ndarray, nx: int, xi=None, rho=None):
    """G [nelt, nx^3, 6] for trilinear elements given by ``corners [nelt, 8, 3]``."""
    if xi is None:
        xi, rho, _ = gll(nx)
    corners = _f64(corners)
    nelt = corners.shape[0]
    G = np.empty((nelt, nx ** 3, 6))
    mind = ctypes.c_double(0.0)
    bad = _load().ref_geom(nelt, nx, _p(_f64(xi)), _p(_f64(rho)), _p(corners), _p(G), ctypes.byref(mind))
    if bad:
        raise ValueError("non-positive Jacobian at %d nodes (min %g)" % (bad, mind.value))
    return G


# ----------------------------------------------------------------------------- AX
def ax(D: np.ndarray, G: np.ndarray, u: np.ndarray) -> np.ndarray:
    """w = AX(u) element by element (Listing 1)."""
    D = _f64(D)
    nx = D.shape[0]
    u = _f64(u).reshape(-1, nx ** 3)
    G = _f64(G).reshape(u.shape[0], nx ** 3, 6)
    w = np.empty_like(u)
    st = _load().ref_ax(u.shape[0], nx, _p(D), _p(G), _p(u), _p(w))
    if st != OK:
        raise MemoryError("ref_ax")
    return w


def gradient_matrices(D: np.ndarray):
    """Dense Br, Bs, Bt (nx^3 x nx^3): (Ba u)(m) = d u / d r_a at node m, i fastest."""
    nx = D.shape[0]
    I = np.eye(nx)
    Br = np.kron(I, np.kron(I, D))
    Bs = np.kron(I, np.kron(D, I))
    Bt = np.kron(D, np.kron(I, I))
    return Br, Bs, Bt


def element_matrix(D: np.ndarray, Ge: np.ndarray) -> np.ndarray:
    """Dense A_e[p,q] = sum_m sum_ab G_ab(m) (B_a)_{mp} (B_b)_{mq} for one element."""
    B = gradient_matrices(_f64(D))
    comp = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    A = np.zeros((B[0].shape[1],) * 2)
    for a in range(3):
        for b in range(3):
            g = Ge[:, comp[(min(a, b), max(a, b))]]
            A += B[a].T @ (g[:, None] * B[b])
    return A


def assembled_matrix(D, G, glo_num, nglobal):
    """Dense global A = Q^T blockdiag(A_e) Q on global ids (tiny meshes only)."""
    nelt, n3 = glo_num.shape
    A = np.zeros((nglobal, nglobal))
    for e in range(nelt):
        Ae = element_matrix(D, G[e])
        ids = glo_num[e]
        A[np.ix_(ids, ids)] += Ae
    return A


# ----------------------------------------------------------------------------- gather-scatter
def gs_build(glo_num: np.ndarray):
    """CSR (offsets, idx) of all shared-node groups, canonical order."""
    glo = np.ascontiguousarray(glo_num, dtype=np.int64).reshape(-1)
    n = glo.shape[0]
    offsets = np.zeros(n + 1, dtype=np.int64)
    idx = np.zeros(max(n, 1), dtype=np.int64)
    ng = _load().ref_gs_build(n, _p(glo), _p(offsets), _p(idx))
    if ng < 0:
        raise MemoryError("ref_gs_build")
    return offsets[: ng + 1].copy(), idx[: offsets[ng]].copy()


def dssum(offsets, idx, v):
    v = _f64(v).copy()
    shape = v.shape
    v = v.reshape(-1)
    _load().ref_dssum(offsets.shape[0] - 1, _p(offsets), _p(idx), _p(v))
    return v.reshape(shape)


def inv_multiplicity(n, offsets, idx):
    c = np.empty(n)
    _load().ref_inv_multiplicity(n, offsets.shape[0] - 1, _p(offsets), _p(idx), _p(c))
    return c


def mask_apply(mask, v):
    v = _f64(v).copy()
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    _load().ref_mask(m.shape[0], _p(m), _p(v.reshape(-1)))
    return v


# ----------------------------------------------------------------------------- Jacobi / PCG
def diag_local(D, G):
    D = _f64(D)
    nx = D.shape[0]
    G = _f64(G).reshape(-1, nx ** 3, 6)
    d = np.empty((G.shape[0], nx ** 3))
    _load().ref_diag_local(G.shape[0], nx, _p(D), _p(G), _p(d))
    return d


def jacobi_minv(D, G, offsets, idx, mask):
    D = _f64(D)
    nx = D.shape[0]
    G = _f64(G).reshape(-1, nx ** 3, 6)
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(G.shape[0], nx ** 3)
    minv = np.empty((G.shape[0], nx ** 3))
    _load().ref_jacobi_minv(G.shape[0], nx, _p(D), _p(G), offsets.shape[0] - 1, _p(offsets), _p(idx), _p(m),
                            _p(minv))
    return minv


def pcg(D, G, offsets, idx, mask, minv, f, tol=1e-8, max_iter=1000, history=False):
    """Returns (status, x, iters, relres[, history])."""
    D = _f64(D)
    nx = D.shape[0]
    G = _f64(G).reshape(-1, nx ** 3, 6)
    nelt = G.shape[0]
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(nelt, nx ** 3)
    f = _f64(f).reshape(nelt, nx ** 3)
    minv = _f64(minv).reshape(nelt, nx ** 3)
    x = np.empty((nelt, nx ** 3))
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.zeros(max(max_iter, 1))
    st = _load().ref_pcg(nelt, nx, _p(D), _p(G), offsets.shape[0] - 1, _p(offsets), _p(idx), _p(m), _p(minv),
                         _p(f), _p(x), float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rr), _p(hist))
    if history:
        return st, x, it.value, rr.value, hist[: it.value].copy()
    return st, x, it.value, rr.value


class Problem:
    """Everything the oracle derives from one mesh: D, G, gs groups, c, Minv."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.nx = mesh.nx
        self.xi, self.rho, self.D = gll(mesh.nx)
        self.G = geom(mesh.corners, mesh.nx, self.xi, self.rho)
        self.offsets, self.idx = gs_build(mesh.glo_num)
        self.c = inv_multiplicity(mesh.npts, self.offsets, self.idx).reshape(mesh.nelt, -1)
        self.minv = jacobi_minv(self.D, self.G, self.offsets, self.idx, mesh.mask)

    def apply(self, u):
        """Masked, assembled operator on an E-vector: mask(dssum(AX u))."""
        w = ax(self.D, self.G, u)
        w = dssum(self.offsets, self.idx, w)
        return mask_apply(self.mesh.mask, w)

    def residual(self, f, x):
        """||b - A x||_c / ||b||_c with b = mask.f."""
        b = mask_apply(self.mesh.mask, f)
        r = b - self.apply(x)
        return float(np.sqrt(np.sum(self.c * r * r)) / np.sqrt(np.sum(self.c * b * b)))
