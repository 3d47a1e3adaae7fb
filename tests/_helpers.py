"""Test-side geometry helpers (affine elements, exact integrals) independent of the oracle."""
import itertools

import numpy as np


def affine_corners(X0, a, b, c):
    """Corners [8,3] of the parallelepiped X0 + di a + dj b + dk c."""
    out = np.empty((8, 3))
    for q in range(8):
        di, dj, dk = q & 1, (q >> 1) & 1, (q >> 2) & 1
        out[q] = X0 + di * a + dj * b + dk * c
    return out


def affine_nodes(X0, a, b, c, xi):
    """Physical coordinates [nx^3, 3] of the tensor nodes (i fastest)."""
    nx = xi.shape[0]
    K, J, I = np.meshgrid(xi, xi, xi, indexing="ij")
    r, s, t = I.reshape(-1), J.reshape(-1), K.reshape(-1)
    return X0[None] + 0.5 * (1 + r)[:, None] * a[None] + 0.5 * (1 + s)[:, None] * b[None] + 0.5 * (1 + t)[:, None] * c[None]


class Poly3:
    """Random polynomial of total degree <= deg in (x - x0)."""

    def __init__(self, deg, rng, x0):
        self.terms = [m for m in itertools.product(range(deg + 1), repeat=3) if sum(m) <= deg]
        self.coef = rng.uniform(-1, 1, size=len(self.terms))
        self.x0 = np.asarray(x0, dtype=np.float64)

    def __call__(self, X):
        Y = X - self.x0
        return sum(c * Y[:, 0] ** p * Y[:, 1] ** q * Y[:, 2] ** r for c, (p, q, r) in zip(self.coef, self.terms))

    def grad(self, X):
        Y = X - self.x0
        g = np.zeros_like(Y)
        for c, (p, q, r) in zip(self.coef, self.terms):
            if p:
                g[:, 0] += c * p * Y[:, 0] ** (p - 1) * Y[:, 1] ** q * Y[:, 2] ** r
            if q:
                g[:, 1] += c * q * Y[:, 0] ** p * Y[:, 1] ** (q - 1) * Y[:, 2] ** r
            if r:
                g[:, 2] += c * r * Y[:, 0] ** p * Y[:, 1] ** q * Y[:, 2] ** (r - 1)
        return g


def exact_dirichlet_energy_affine(poly, X0, a, b, c, npts):
    """int_e |grad u|^2 dx over the parallelepiped, by Gauss-Legendre (numpy.leggauss)."""
    g, wg = np.polynomial.legendre.leggauss(npts)
    nodes = affine_nodes(X0, a, b, c, g)
    W = np.einsum("k,j,i->kji", wg, wg, wg).reshape(-1)
    detJ = abs(np.linalg.det(np.stack([a, b, c], axis=1))) / 8.0
    gr = poly.grad(nodes)
    return float(np.sum(W * np.sum(gr * gr, axis=1)) * detJ)
