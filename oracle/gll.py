"""Oracle: Gauss-Lobatto-Legendre nodes, weights and derivative matrix (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.

The paper takes the derivative matrix ``dxm1`` (and its transpose ``dxtm1``) as
an input of ``ax`` (Section II-B, Listing 1) without defining it; Nekbone's
operator is the standard spectral-element one, so the reading taken here is the
textbook GLL collocation derivative on the ``nx`` Lobatto points of order
``N = nx - 1``:

* nodes: -1, +1 and the roots of L'_N (L_N the Legendre polynomial of degree N);
* weights: rho_i = 2 / (N (N+1) L_N(xi_i)^2);
* D[i, l] = l_l'(xi_i), the derivative at node i of the Lagrange basis function
  of node l, which in closed form is L_N(xi_i) / (L_N(xi_l) (xi_i - xi_l)) off the
  diagonal, -N(N+1)/4 at (0,0), +N(N+1)/4 at (N,N) and 0 elsewhere on the diagonal.

The interior nodes come from numpy's Legendre-series root finder (a companion
matrix eigenproblem), polished by Newton steps on L'_N.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L


def _legendre_coeffs(N: int) -> np.ndarray:
    c = np.zeros(N + 1)
    c[N] = 1.0
    return c


def gll_nodes_weights(nx: int):
    """Return (xi[nx], rho[nx]) in ascending order."""
    if nx < 2:
        raise ValueError("nx must be >= 2")
    N = nx - 1
    cN = _legendre_coeffs(N)
    d1 = L.legder(cN)
    d2 = L.legder(d1)
    interior = np.sort(np.real(L.legroots(d1))) if N >= 2 else np.zeros(0)
    for _ in range(4):  # Newton polish on L'_N
        interior = interior - L.legval(interior, d1) / L.legval(interior, d2)
    xi = np.concatenate([[-1.0], interior, [1.0]])
    LN = L.legval(xi, cN)
    rho = 2.0 / (N * (N + 1) * LN ** 2)
    return xi, rho


def derivative_matrix(xi: np.ndarray) -> np.ndarray:
    """D[i, l] = derivative at xi_i of the Lagrange polynomial of node l."""
    nx = xi.shape[0]
    N = nx - 1
    LN = L.legval(xi, _legendre_coeffs(N))
    D = np.zeros((nx, nx))
    for i in range(nx):
        for l in range(nx):
            if i != l:
                D[i, l] = LN[i] / (LN[l] * (xi[i] - xi[l]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


def gll(nx: int):
    """(xi, rho, D) for nx points per direction."""
    xi, rho = gll_nodes_weights(nx)
    return xi, rho, derivative_matrix(xi)
