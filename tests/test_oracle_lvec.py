"""Pins of the unique-node oracle against things other than itself: the dense
assembled matrix built element by element, the E-vector C oracle's solve, a
dense direct solve, and the special cases of the method."""
import numpy as np
import pytest

from oracle import lvec, ref
from paper_2011_04981_gb300 import inputs


def _setup(dims, nx, seed=1, perturb=0.15):
    mesh = inputs.box_mesh(*dims, nx, perturb=perturb, seed=seed)
    P = ref.Problem(mesh)
    l2g, mL, nL = lvec.build(mesh.glo_num, mesh.mask)
    return mesh, P, l2g, mL, nL


def test_build_orders_by_global_id_and_checks_the_mask():
    glo = np.array([[5, 9, 2], [9, 2, 7]])
    mask = np.array([[1, 0, 1], [0, 1, 1]], dtype=np.uint8)
    l2g, mL, nL = lvec.build(glo, mask)
    assert nL == 4
    assert l2g.tolist() == [[1, 3, 0], [3, 0, 2]]  # ids 2, 5, 7, 9 -> 0, 1, 2, 3
    assert mL.tolist() == [1, 1, 1, 0]
    with pytest.raises(ValueError):
        lvec.build(glo, np.array([[1, 1, 1], [0, 1, 1]], dtype=np.uint8))  # node 9 free in one copy only
    with pytest.raises(ValueError):
        lvec.build(np.array([[0, -1]]), np.ones((1, 2), dtype=np.uint8))


@pytest.mark.parametrize("dims,nx", [((2, 2, 1), 3), ((2, 1, 2), 4), ((1, 2, 2), 5)])
def test_apply_equals_dense_assembled_matrix(dims, nx):
    """Q^T AX Q u against the dense A = sum_e P_e^T A_e P_e built from the element bilinear form."""
    mesh, P, l2g, mL, nL = _setup(dims, nx)
    assert nL == mesh.nglobal  # the lattice numbering uses every id once: L order = global id order
    A = ref.assembled_matrix(P.D, P.G, mesh.glo_num, mesh.nglobal)
    u = np.random.default_rng(nx).uniform(-1, 1, nL)
    w = lvec.apply(P.D, P.G, l2g, nL, u)
    assert np.max(np.abs(w - A @ u)) <= 1e-12 * np.max(np.abs(A @ u))


def test_jacobi_is_inverse_dense_diagonal():
    mesh, P, l2g, mL, nL = _setup((2, 2, 2), 4)
    A = ref.assembled_matrix(P.D, P.G, mesh.glo_num, mesh.nglobal)
    minv = lvec.jacobi_minv(P.D, P.G, l2g, nL, mL)
    free = mL != 0
    assert np.all(minv[~free] == 0.0)
    assert np.max(np.abs(minv[free] * np.diag(A)[free] - 1.0)) <= 1e-13


def test_solution_equals_dense_direct_solve():
    mesh, P, l2g, mL, nL = _setup((2, 2, 2), 5, seed=4)
    A = ref.assembled_matrix(P.D, P.G, mesh.glo_num, mesh.nglobal)
    f = np.random.default_rng(3).uniform(-1, 1, nL)
    minv = lvec.jacobi_minv(P.D, P.G, l2g, nL, mL)
    x, it, rr = lvec.pcg(P.D, P.G, l2g, nL, mL, minv, f, tol=1e-13, max_iter=5000)
    assert rr <= 1e-13
    free = np.flatnonzero(mL)
    xd = np.zeros(nL)
    xd[free] = np.linalg.solve(A[np.ix_(free, free)], f[free])
    assert np.max(np.abs(x - xd)) <= 1e-10 * np.max(np.abs(xd))
    assert np.all(x[mL == 0] == 0.0)


@pytest.mark.parametrize("dims,nx", [((3, 2, 2), 4), ((2, 3, 1), 6)])
def test_same_iterates_as_the_element_vector_solve(dims, nx):
    """The E-vector C oracle (dssum, 1/multiplicity-weighted dots) and this form are the same method."""
    mesh, P, l2g, mL, nL = _setup(dims, nx, seed=2)
    g = np.random.default_rng(5).uniform(-1, 1, mesh.nglobal)
    fE = g[mesh.glo_num]
    minv = lvec.jacobi_minv(P.D, P.G, l2g, nL, mL)
    for tol, cap in ((1e-10, 3000), (0.0, 17)):
        st, xE, itE, rrE = ref.pcg(P.D, P.G, P.offsets, P.idx, mesh.mask, P.minv, fE, tol, cap)
        xL, itL, rrL = lvec.pcg(P.D, P.G, l2g, nL, mL, minv, g, tol, cap)
        assert itL == itE
        assert abs(rrL - rrE) <= 1e-8 * rrE + 1e-14  # rounding of ||r|| / ||b|| near convergence
        assert np.max(np.abs(xL[l2g] - xE)) <= 1e-10 * np.max(np.abs(xE))
    # Jacobi diagonals agree copy by copy
    assert np.max(np.abs(minv[l2g] - P.minv)) <= 1e-14 * np.max(np.abs(P.minv))


def test_special_cases():
    # all nodes on the boundary: b = 0, x = 0 after 0 iterations
    mesh, P, l2g, mL, nL = _setup((1, 1, 1), 2, perturb=0.0)
    assert mL.sum() == 0
    x, it, rr = lvec.pcg(P.D, P.G, l2g, nL, mL, lvec.jacobi_minv(P.D, P.G, l2g, nL, mL), np.ones(nL), 1e-8, 10)
    assert it == 0 and np.all(x == 0.0)
    # one free node: one iteration gives f / A_pp
    mesh, P, l2g, mL, nL = _setup((1, 1, 1), 3, perturb=0.0)
    assert mL.sum() == 1
    f = np.random.default_rng(0).uniform(1, 2, nL)
    minv = lvec.jacobi_minv(P.D, P.G, l2g, nL, mL)
    x, it, rr = lvec.pcg(P.D, P.G, l2g, nL, mL, minv, f, 1e-12, 10)
    c = int(np.flatnonzero(mL)[0])
    Ae = ref.element_matrix(P.D, P.G[0])
    assert it == 1
    assert abs(x[c] - f[c] / Ae[13, 13]) <= 1e-14 * abs(f[c] / Ae[13, 13])
    # a constant field is in the kernel of the unmasked operator
    mesh, P, l2g, mL, nL = _setup((2, 2, 2), 5)
    w = lvec.apply(P.D, P.G, l2g, nL, np.full(nL, 3.0))
    assert np.max(np.abs(w)) <= 1e-12
