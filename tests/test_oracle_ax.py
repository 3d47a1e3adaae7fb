"""Pins of the oracle's geometric factors and AX operator (Section II-B, Listing 1).

None of these re-types the oracle's formulas: they check mathematical identities
of the operator (kernel, symmetry, energy), closed forms on boxes, and a dense
brute-force form of the bilinear form.
"""
import os

import numpy as np
import pytest

from oracle import ref
from paper_2011_04981_gb300 import inputs, perfmodel
from tests import _helpers as H

EPS = 2.220446049250313e-16


def _golden_counts():
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, val = line.split()[:2]
                vals[name] = float(val)
    return vals


def test_paper_operation_counts():
    g = _golden_counts()
    assert 16 ** 3 == g["points_per_element_nx16"]
    assert perfmodel.ax_flops_per_point(16) == g["flops_per_point_nx16"]
    assert perfmodel.ax_flops_per_element(16) == g["flops_per_element_nx16"]
    assert perfmodel.matmul_flops_per_cycle(16) == g["matmul_flops_per_cycle_nx16"]
    assert round(perfmodel.ax_flops_per_point(16) * 0.3) == g["theoretical_gflops_300mhz"]
    assert abs(perfmodel.ax_flops_per_point(16) * 0.4 - g["theoretical_gflops_400mhz"]) < 1e-9
    assert 800 * 16 ** 3 == g["pipeline_cycles_800_elements"]
    assert 16 ** 3 // 8 == g["fill_cycles_per_element"]


@pytest.mark.parametrize("nx", [2, 3, 5, 8, 10])
def test_geom_axis_aligned_closed_form(nx):
    hx, hy, hz = 0.3, 0.7, 1.9
    X0 = np.array([0.25, -1.0, 3.0])
    C = H.affine_corners(X0, np.array([hx, 0, 0]), np.array([0, hy, 0]), np.array([0, 0, hz]))
    xi, rho, D = ref.gll(nx)
    G = ref.geom(C[None], nx, xi, rho)[0]
    W = np.einsum("k,j,i->kji", rho, rho, rho).reshape(-1) * hx * hy * hz / 8.0
    assert np.allclose(G[:, 0], W * (2 / hx) ** 2, rtol=1e-14, atol=0)
    assert np.allclose(G[:, 3], W * (2 / hy) ** 2, rtol=1e-14, atol=0)
    assert np.allclose(G[:, 5], W * (2 / hz) ** 2, rtol=1e-14, atol=0)
    assert np.all(np.abs(G[:, [1, 2, 4]]) <= 1e-14 * np.abs(G).max())


def _random_affine(rng, h=1.0):
    X0 = rng.uniform(-1, 1, size=3)
    M = h * (np.eye(3) + 0.35 * rng.uniform(-1, 1, size=(3, 3)))
    if np.linalg.det(M) < 0:
        M[:, 0] *= -1
    return X0, M[:, 0].copy(), M[:, 1].copy(), M[:, 2].copy()


@pytest.mark.parametrize("nx", [2, 3, 4, 6, 8, 10, 12])
def test_energy_identity_affine(nx):
    """u^T A_e u = int_e |grad u|^2 for u of total degree <= nx-1 on a sheared parallelepiped."""
    rng = np.random.default_rng(100 + nx)
    xi, rho, D = ref.gll(nx)
    for trial in range(3):
        X0, a, b, c = _random_affine(rng)
        G = ref.geom(H.affine_corners(X0, a, b, c)[None], nx, xi, rho)
        poly = H.Poly3(nx - 1, rng, X0 + 0.5 * (a + b + c))
        u = poly(H.affine_nodes(X0, a, b, c, xi))
        lhs = float(u @ ref.ax(D, G, u[None])[0])
        rhs = H.exact_dirichlet_energy_affine(poly, X0, a, b, c, nx + 2)
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs), (trial, lhs, rhs)


def test_energy_identity_global_sheared_box():
    """Sum over a lattice of parallelepipeds equals the integral over the sheared box."""
    nx = 5
    rng = np.random.default_rng(7)
    mesh = inputs.box_mesh(3, 2, 2, nx, perturb=0.0)
    M = np.eye(3) + 0.3 * rng.uniform(-1, 1, size=(3, 3))
    corners = mesh.corners @ M.T
    xi, rho, D = ref.gll(nx)
    G = ref.geom(corners, nx, xi, rho)
    poly = H.Poly3(nx - 1, rng, np.zeros(3))
    total_lhs = 0.0
    total_rhs = 0.0
    for e in range(mesh.nelt):
        C = corners[e]
        X0, a, b, c = C[0], C[1] - C[0], C[2] - C[0], C[4] - C[0]
        u = poly(H.affine_nodes(X0, a, b, c, xi))
        total_lhs += float(u @ ref.ax(D, G[e:e + 1], u[None])[0])
        total_rhs += H.exact_dirichlet_energy_affine(poly, X0, a, b, c, nx + 2)
    assert abs(total_lhs - total_rhs) <= 1e-12 * abs(total_rhs)


@pytest.mark.parametrize("nx", [2, 4, 8, 10, 16])
def test_constants_in_kernel_on_trilinear_elements(nx):
    mesh = inputs.box_mesh(3, 3, 2, nx, perturb=0.2, seed=3)
    xi, rho, D = ref.gll(nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    w = ref.ax(D, G, 3.5 * np.ones((mesh.nelt, nx ** 3)))
    bound = 8 * nx * EPS * np.abs(G).max() * np.abs(D).max() ** 2 * nx * 3.5 * 6
    assert np.abs(w).max() <= bound


@pytest.mark.parametrize("nx", [3, 6, 10])
def test_symmetry_on_trilinear_elements(nx):
    mesh = inputs.box_mesh(2, 2, 2, nx, perturb=0.2, seed=5)
    xi, rho, D = ref.gll(nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = inputs.random_local_field(mesh.nelt, nx, seed=1)
    v = inputs.random_local_field(mesh.nelt, nx, seed=2)
    Au = ref.ax(D, G, u)
    Av = ref.ax(D, G, v)
    a, b = float(np.sum(v * Au)), float(np.sum(u * Av))
    scale = float(np.sum(np.abs(v) * np.abs(Au)))
    assert abs(a - b) <= 1e-13 * scale


@pytest.mark.parametrize("nx", [2, 3, 4, 5])
def test_dense_brute_force(nx):
    mesh = inputs.box_mesh(2, 2, 1, nx, perturb=0.2, seed=11)
    xi, rho, D = ref.gll(nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = inputs.random_local_field(mesh.nelt, nx, seed=4)
    w = ref.ax(D, G, u)
    for e in range(mesh.nelt):
        Ae = ref.element_matrix(D, G[e])
        we = Ae @ u[e]
        assert np.max(np.abs(w[e] - we)) <= 1e-13 * np.max(np.abs(we))
        # symmetric positive semi-definite with exactly one zero mode (constants)
        assert np.allclose(Ae, Ae.T, rtol=0, atol=1e-13 * np.abs(Ae).max())
        ev = np.linalg.eigvalsh(Ae)
        assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-8 * ev[-1]


@pytest.mark.parametrize("nx", [2, 4, 7, 10])
def test_kronecker_form_on_boxes(nx):
    """Axis-aligned box: A_e = Bz(x)By(x)Ax + Bz(x)Ay(x)Bx + Az(x)By(x)Bx with 1D stiffness/mass."""
    hx, hy, hz = 0.4, 1.1, 0.8
    C = H.affine_corners(np.zeros(3), np.array([hx, 0, 0]), np.array([0, hy, 0]), np.array([0, 0, hz]))
    xi, rho, D = ref.gll(nx)
    G = ref.geom(C[None], nx, xi, rho)
    A1 = lambda h: (2.0 / h) * D.T @ np.diag(rho) @ D
    B1 = lambda h: (h / 2.0) * np.diag(rho)
    A = (np.kron(B1(hz), np.kron(B1(hy), A1(hx))) + np.kron(B1(hz), np.kron(A1(hy), B1(hx)))
         + np.kron(A1(hz), np.kron(B1(hy), B1(hx))))
    u = np.random.default_rng(nx).uniform(-1, 1, size=nx ** 3)
    w = ref.ax(D, G, u[None])[0]
    assert np.max(np.abs(w - A @ u)) <= 1e-13 * np.max(np.abs(A @ u))
