"""Oracle for the unique-node ("L-vector") form of the solve (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never touches the
CUDA library.

The paper's CG (Section II-B) works on element-local vectors and makes shared
nodes agree with the nearest-neighbour exchange.  Written on vectors that hold
each global node once (ordered by ascending global id) the same method is:

* Q: unique -> element points, (Q u)[p] = u[l2g[p]];
* the assembled operator A_L = Q^T blockdiag(A_e) Q, A_e the element operator
  of Listing 1 (``ref.ax``), and Q^T the sum over the copies of each node;
* b = mask . f, Jacobi M^-1 = 1 / diag(A_L) on free nodes and 0 on Dirichlet
  nodes;
* preconditioned CG with plain Euclidean inner products, stopped when
  ||r|| / ||b|| <= tol (tol = 0: a fixed number of iterations).
"""
from __future__ import annotations

import numpy as np

from . import ref


def build(glo_num, mask):
    """Returns (l2g [nelt, n3] int64, mask_L [nL] uint8, nL) with unique nodes in ascending global id."""
    glo = np.asarray(glo_num, dtype=np.int64)
    if glo.size and glo.min() < 0:
        raise ValueError("negative global id")
    ids, l2g = np.unique(glo.reshape(-1), return_inverse=True)
    m = np.asarray(mask, dtype=np.uint8).reshape(-1) != 0
    nL = ids.shape[0]
    free = np.zeros(nL, dtype=bool)
    fixed = np.zeros(nL, dtype=bool)
    free[l2g[m]] = True
    fixed[l2g[~m]] = True
    if np.any(free & fixed):
        raise ValueError("copies of a node disagree on the Dirichlet mask")
    return l2g.reshape(glo.shape), free.astype(np.uint8), nL


def gather(l2g, u):
    """Q u: element-local copies of a unique-node vector."""
    return np.asarray(u, dtype=np.float64)[l2g]


def assemble(l2g, nL, w):
    """Q^T w: sum of the element-local values over the copies of each node."""
    return np.bincount(np.asarray(l2g).reshape(-1), weights=np.asarray(w, dtype=np.float64).reshape(-1),
                       minlength=nL)


def apply(D, G, l2g, nL, u):
    """A_L u = Q^T AX Q u (unmasked)."""
    return assemble(l2g, nL, ref.ax(D, G, gather(l2g, u)))


def jacobi_minv(D, G, l2g, nL, mask_L):
    """1 / diag(A_L) on free nodes, 0 on Dirichlet nodes."""
    d = assemble(l2g, nL, ref.diag_local(D, G))
    out = np.zeros(nL)
    free = np.asarray(mask_L) != 0
    out[free] = 1.0 / d[free]
    return out


def pcg(D, G, l2g, nL, mask_L, minv, f, tol=1e-8, max_iter=1000):
    """Jacobi-PCG on unique-node vectors from x = 0; returns (x, iters, relres)."""
    m = (np.asarray(mask_L) != 0).astype(np.float64)
    x = np.zeros(nL)
    r = m * np.asarray(f, dtype=np.float64)
    z = minv * r
    p = z.copy()
    rz = float(r @ z)
    rr = float(r @ r)
    bnorm = np.sqrt(rr)
    if rr == 0.0:
        return x, 0, 0.0
    relres = 1.0
    for it in range(1, max_iter + 1):
        w = m * apply(D, G, l2g, nL, p)
        alpha = rz / float(p @ w)
        x += alpha * p
        r -= alpha * w
        z = minv * r
        rr = float(r @ r)
        rz_new = float(r @ z)
        relres = np.sqrt(rr) / bnorm
        if tol > 0.0 and relres <= tol:
            return x, it, relres
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, max_iter, relres
