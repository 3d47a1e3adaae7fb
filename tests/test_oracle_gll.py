"""Pins of the oracle's GLL rule and derivative matrix against closed forms.

The paper takes dxm1/dxtm1 as inputs (Section II-B, Listing 1); they are the
textbook Gauss-Lobatto-Legendre collocation objects, so these pins are
mathematical facts independent of how the oracle computes them.
"""
import math

import numpy as np
import pytest

from oracle import gll

NXS = list(range(2, 17))


@pytest.mark.parametrize("nx", NXS)
def test_weights_sum_to_two_and_nodes_symmetric(nx):
    xi, rho = gll.gll_nodes_weights(nx)
    assert xi[0] == -1.0 and xi[-1] == 1.0
    assert np.all(np.diff(xi) > 0)
    assert np.allclose(xi, -xi[::-1], atol=1e-15, rtol=0)
    assert np.allclose(rho, rho[::-1], atol=1e-15, rtol=0)
    assert abs(rho.sum() - 2.0) < 4e-15 * nx


@pytest.mark.parametrize("nx", NXS)
def test_quadrature_exact_to_degree_2N_minus_1(nx):
    N = nx - 1
    xi, rho = gll.gll_nodes_weights(nx)
    for m in range(0, 2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(rho, xi ** m) - exact) < 2e-14 * nx, m
    # and not exact one degree higher (the rule has exactly degree 2N-1)
    m = 2 * N
    assert abs(np.dot(rho, xi ** m) - 2.0 / (m + 1)) > 1e-9


@pytest.mark.parametrize("nx", NXS)
def test_derivative_of_monomials(nx):
    N = nx - 1
    xi, _, D = gll.gll(nx)
    scale = np.abs(D).max()
    for m in range(0, N + 1):
        lhs = D @ (xi ** m)
        rhs = m * xi ** (m - 1) if m > 0 else np.zeros(nx)
        assert np.max(np.abs(lhs - rhs)) < 64 * nx * 2.2e-16 * scale * max(1, m), m
    assert np.max(np.abs(D.sum(axis=1))) < 4 * nx * 2.2e-16 * scale


def test_textbook_small_rules():
    # N=1: trapezoid; D = 1/2 [[-1, 1], [-1, 1]]
    xi, rho, D = gll.gll(2)
    assert np.allclose(rho, [1, 1], rtol=0, atol=1e-15)
    assert np.allclose(D, 0.5 * np.array([[-1, 1], [-1, 1]]), rtol=0, atol=1e-15)
    # N=2: Simpson; D rows from differentiating the quadratic Lagrange basis on {-1,0,1}
    xi, rho, D = gll.gll(3)
    assert np.allclose(xi, [-1, 0, 1], rtol=0, atol=1e-15)
    assert np.allclose(rho, [1 / 3, 4 / 3, 1 / 3], rtol=0, atol=1e-15)
    assert np.allclose(D, [[-1.5, 2.0, -0.5], [-0.5, 0.0, 0.5], [0.5, -2.0, 1.5]], rtol=0, atol=1e-14)
    # N=3: nodes +-1, +-1/sqrt(5); weights 1/6, 5/6
    xi, rho, D = gll.gll(4)
    assert np.allclose(xi, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], rtol=0, atol=1e-15)
    assert np.allclose(rho, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=0, atol=1e-15)
    # N=4: nodes 0, +-sqrt(3/7), +-1; weights 1/10, 49/90, 32/45
    xi, rho, D = gll.gll(5)
    s = math.sqrt(3 / 7)
    assert np.allclose(xi, [-1, -s, 0, s, 1], rtol=0, atol=1e-15)
    assert np.allclose(rho, [0.1, 49 / 90, 32 / 45, 49 / 90, 0.1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("nx", [3, 6, 10, 16])
def test_D_is_lagrange_derivative_by_brute_force(nx):
    """D[i,l] = l_l'(xi_i) computed by differentiating the Lagrange polynomial
    through numpy's polynomial fit (independent route)."""
    xi, _, D = gll.gll(nx)
    for l in range(nx):
        e = np.zeros(nx)
        e[l] = 1.0
        V = np.vander(xi, nx, increasing=True)
        coef = np.linalg.solve(V, e)
        dcoef = np.array([k * coef[k] for k in range(1, nx)])
        deriv = np.vander(xi, nx - 1, increasing=True) @ dcoef
        assert np.max(np.abs(deriv - D[:, l])) < 1e-9 * max(1.0, np.abs(D).max())
