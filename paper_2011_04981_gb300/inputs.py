"""Seeded synthetic inputs for the deformed-box Poisson problems.

This module builds only the *problem data*: a box lattice of hexahedral elements
with randomly perturbed vertices, the lexicographic global numbering of the
lattice nodes, the Dirichlet boundary flags and random fields.  It contains none
of the spectral-element arithmetic (no quadrature nodes, no derivative matrix,
no geometric factors, no operator): the oracle and the CUDA path each compute
those themselves from these buffers.

Conventions (shared by every consumer):

* element ``e = a + ex*(b + ey*c)`` for lattice cell (a, b, c);
* local node ``p = i + nx*(j + nx*k)`` (i fastest), so an E-vector is
  ``[nelt][nx][nx][nx]`` with i fastest, the layout of ``u(n,n,n,nelt)`` in the
  paper's Listing 1 (Section II-B);
* element corner ``q = di + 2*dj + 4*dk`` holds vertex ``(a+di, b+dj, c+dk)``;
  corners are ``[nelt][8][3]`` float64;
* global id of local node (i, j, k) of element (a, b, c) is the lattice node
  ``(a*N+i, b*N+j, c*N+k)`` with ``N = nx-1``, numbered x fastest.

Vertex perturbation: every vertex coordinate is moved by ``U[-a, a] * h`` along
each axis on which the vertex is not on the box boundary, so the mesh stays
conforming and the domain stays the box.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2011_04981

# Independent random streams per purpose, so that changing one draw never shifts another.
_STREAM_VERTS = 1
_STREAM_U = 2
_STREAM_F = 3
_STREAM_STRETCH = 4
_STREAM_V = 5
_STREAM_BATCH = 6


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE, int(seed), int(stream)])


@dataclasses.dataclass
class BoxMesh:
    ex: int
    ey: int
    ez: int
    nx: int
    corners: np.ndarray  # [nelt, 8, 3] float64
    glo_num: np.ndarray  # [nelt, nx^3] int64
    mask: np.ndarray  # [nelt, nx^3] uint8, 0 on Dirichlet (box boundary) nodes
    lengths: tuple
    seed: int

    @property
    def nelt(self) -> int:
        return self.ex * self.ey * self.ez

    @property
    def npts(self) -> int:
        return self.nelt * self.nx ** 3

    @property
    def nglobal(self) -> int:
        n = self.nx - 1
        return (self.ex * n + 1) * (self.ey * n + 1) * (self.ez * n + 1)


def vertex_lattice(ex, ey, ez, perturb=0.0, lengths=(1.0, 1.0, 1.0), seed=0):
    """Vertex coordinates ``[ez+1, ey+1, ex+1, 3]`` of a perturbed box lattice."""
    lx, ly, lz = lengths
    hx, hy, hz = lx / ex, ly / ey, lz / ez
    ix = np.arange(ex + 1, dtype=np.float64)
    iy = np.arange(ey + 1, dtype=np.float64)
    iz = np.arange(ez + 1, dtype=np.float64)
    Z, Y, X = np.meshgrid(iz * hz, iy * hy, ix * hx, indexing="ij")
    V = np.stack([X, Y, Z], axis=-1)
    if perturb > 0.0:
        rng = _rng(seed, _STREAM_VERTS)
        d = rng.uniform(-perturb, perturb, size=V.shape)
        interior = [
            (np.arange(ex + 1) > 0) & (np.arange(ex + 1) < ex),
            (np.arange(ey + 1) > 0) & (np.arange(ey + 1) < ey),
            (np.arange(ez + 1) > 0) & (np.arange(ez + 1) < ez),
        ]
        mx = interior[0][None, None, :]
        my = interior[1][None, :, None]
        mz = interior[2][:, None, None]
        V[..., 0] += np.where(mx, d[..., 0] * hx, 0.0)
        V[..., 1] += np.where(my, d[..., 1] * hy, 0.0)
        V[..., 2] += np.where(mz, d[..., 2] * hz, 0.0)
    return V


def element_corners(V: np.ndarray) -> np.ndarray:
    """Gather the 8 corners of every lattice cell: ``[nelt, 8, 3]``."""
    ez, ey, ex = V.shape[0] - 1, V.shape[1] - 1, V.shape[2] - 1
    out = np.empty((ez, ey, ex, 8, 3), dtype=np.float64)
    for q in range(8):
        di, dj, dk = q & 1, (q >> 1) & 1, (q >> 2) & 1
        out[:, :, :, q, :] = V[dk:dk + ez, dj:dj + ey, di:di + ex, :]
    return out.reshape(ex * ey * ez, 8, 3)


def lattice_numbering(ex, ey, ez, nx):
    """Global lattice id and Dirichlet flag of every local node.

    Returns ``glo_num [nelt, nx^3] int64`` and ``mask [nelt, nx^3] uint8``.
    """
    n = nx - 1
    gxn, gyn = ex * n + 1, ey * n + 1
    a = np.arange(ex)
    b = np.arange(ey)
    c = np.arange(ez)
    i = np.arange(nx)
    # shapes: [c, b, a, k, j, i]
    gx = (a[None, None, :, None, None, None] * n + i[None, None, None, None, None, :])
    gy = (b[None, :, None, None, None, None] * n + i[None, None, None, None, :, None])
    gz = (c[:, None, None, None, None, None] * n + i[None, None, None, :, None, None])
    gx, gy, gz = np.broadcast_arrays(gx, gy, gz)
    glo = (gx + gxn * (gy + gyn * gz)).astype(np.int64)
    bnd = (gx == 0) | (gx == ex * n) | (gy == 0) | (gy == ey * n) | (gz == 0) | (gz == ez * n)
    nelt = ex * ey * ez
    return glo.reshape(nelt, nx ** 3), (~bnd).astype(np.uint8).reshape(nelt, nx ** 3)


def box_mesh(ex, ey, ez, nx, perturb=0.1, lengths=(1.0, 1.0, 1.0), seed=0, stretch=None) -> BoxMesh:
    """Deformed box mesh: ``ex*ey*ez`` hexahedra on ``[0,Lx]x[0,Ly]x[0,Lz]``.

    ``perturb`` is the half-width ``a`` of the uniform vertex displacement in units
    of the local spacing h.  ``stretch`` (optional) scales the axes after the
    perturbation; ``stretch="random8"`` draws an anisotropic factor in [1, 8] per
    axis from the seed (the learned-preconditioner family).
    """
    lengths = tuple(float(x) for x in lengths)
    if isinstance(stretch, str):
        if stretch != "random8":
            raise ValueError(stretch)
        rng = _rng(seed, _STREAM_STRETCH)
        stretch = tuple(float(s) for s in np.exp(rng.uniform(0.0, math.log(8.0), size=3)))
    V = vertex_lattice(ex, ey, ez, perturb, lengths, seed)
    if stretch is not None:
        V = V * np.asarray(stretch, dtype=np.float64)[None, None, None, :]
        lengths = tuple(L * s for L, s in zip(lengths, stretch))
    corners = element_corners(V)
    glo, mask = lattice_numbering(ex, ey, ez, nx)
    return BoxMesh(ex, ey, ez, nx, corners, glo, mask, lengths, seed)


def random_local_field(nelt, nx, seed=0, stream=_STREAM_U) -> np.ndarray:
    """Independent ``U[-1,1]`` value at every local node (a discontinuous E-vector)."""
    return _rng(seed, stream).uniform(-1.0, 1.0, size=(nelt, nx ** 3))


def random_global_field(mesh: BoxMesh, seed=0, stream=_STREAM_F) -> np.ndarray:
    """``U[-1,1]`` drawn once per global lattice node and copied to every local
    node that shares it (a consistent E-vector)."""
    g = _rng(seed, stream).uniform(-1.0, 1.0, size=mesh.nglobal)
    return g[mesh.glo_num]


def gdof_count(nelt: int, nx: int) -> int:
    """Local (E-vector) points of a mesh: the unit in which GDOF/s is counted."""
    return int(nelt) * int(nx) ** 3


def batch_problem_specs(nprob=256, seed=0, nelt_range=(8, 4096), nx_choices=(6, 8, 10, 12),
                        aspects=((1, 1, 1), (2, 1, 1), (4, 2, 1))):
    """Box dimensions and nx of a batch of uneven problems.

    Element counts are log-uniform in ``nelt_range``; with aspect ratio (a:b:c),
    ``m = max(1, round(cbrt(nelt/(a*b*c))))`` and the box is ``(a*m, b*m, c*m)``
    elements, so the realised element count is returned, not the drawn one.
    """
    rng = _rng(seed, _STREAM_BATCH)
    lo, hi = math.log(nelt_range[0]), math.log(nelt_range[1])
    specs = []
    for p in range(nprob):
        target = math.exp(rng.uniform(lo, hi))
        a, b, c = aspects[int(rng.integers(len(aspects)))]
        m = max(1, int(round((target / (a * b * c)) ** (1.0 / 3.0))))
        nx = int(nx_choices[int(rng.integers(len(nx_choices)))])
        specs.append(dict(ex=a * m, ey=b * m, ez=c * m, nx=nx, seed=seed * 100003 + p))
    return specs
