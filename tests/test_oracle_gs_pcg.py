"""Pins of the oracle's gather-scatter, Jacobi diagonal and PCG (Section II-B).

The groups are checked against a pure-Python grouping and the lattice's closed-form
multiplicity counts; dssum against the scatter-matrix form Q Q^T v; the Jacobi
diagonal against the diagonal of the dense assembled matrix; PCG against a dense
direct solve and two special cases with 0 and 1 unknowns.
"""
import collections

import numpy as np
import pytest

from oracle import ref
from paper_2011_04981_gb300 import inputs


@pytest.mark.parametrize("dims,nx", [((1, 1, 1), 2), ((2, 1, 1), 3), ((2, 3, 2), 4), ((3, 3, 3), 5)])
def test_groups_match_pure_python(dims, nx):
    mesh = inputs.box_mesh(*dims, nx, perturb=0.0)
    off, idx = ref.gs_build(mesh.glo_num)
    groups = collections.defaultdict(list)
    for p, g in enumerate(mesh.glo_num.reshape(-1)):
        groups[int(g)].append(p)
    expect = [sorted(v) for k, v in sorted(groups.items()) if len(v) >= 2]
    got = [list(idx[off[g]:off[g + 1]]) for g in range(len(off) - 1)]
    assert got == expect


@pytest.mark.parametrize("dims,nx", [((3, 2, 4), 4), ((4, 4, 4), 6), ((2, 2, 5), 3)])
def test_multiplicity_counts_closed_form(dims, nx):
    ex, ey, ez = dims
    mesh = inputs.box_mesh(ex, ey, ez, nx, perturb=0.0)
    off, idx = ref.gs_build(mesh.glo_num)
    sizes = collections.Counter(np.diff(off).tolist())
    m = nx - 2
    # shared-by-8: interior lattice vertices; by-4: interior of interior edges; by-2: interior of interior faces
    n8 = (ex - 1) * (ey - 1) * (ez - 1)
    n4 = m * (ex * (ey - 1) * (ez - 1) + ey * (ex - 1) * (ez - 1) + ez * (ex - 1) * (ey - 1))
    # vertices on the boundary surface are shared by 4 (on a face) or 2 (on an edge)
    n4 += (ex - 1) * (ey - 1) * 2 + (ex - 1) * (ez - 1) * 2 + (ey - 1) * (ez - 1) * 2
    n2 = m * m * ((ex - 1) * ey * ez + (ey - 1) * ex * ez + (ez - 1) * ex * ey)
    # edge-interior nodes of element edges lying on the boundary faces (not box edges) -> shared by 2
    n2 += m * 2 * (ex * (ey - 1) + ex * (ez - 1) + ey * (ex - 1) + ey * (ez - 1) + ez * (ex - 1) + ez * (ey - 1))
    # lattice vertices on the box edges (not corners) -> shared by 2
    n2 += 4 * ((ex - 1) + (ey - 1) + (ez - 1))
    assert sizes.get(8, 0) == n8
    assert sizes.get(4, 0) == n4
    assert sizes.get(2, 0) == n2
    assert set(sizes) <= {2, 4, 8}
    assert mesh.npts - int(np.sum(np.diff(off))) + len(off) - 1 == mesh.nglobal


def test_dssum_is_scatter_of_gather():
    mesh = inputs.box_mesh(3, 2, 2, 5, perturb=0.0)
    off, idx = ref.gs_build(mesh.glo_num)
    v = inputs.random_local_field(mesh.nelt, 5, seed=9)
    s = ref.dssum(off, idx, v)
    glob = np.zeros(mesh.nglobal)
    np.add.at(glob, mesh.glo_num.reshape(-1), v.reshape(-1))
    assert np.allclose(s.reshape(-1), glob[mesh.glo_num.reshape(-1)], rtol=1e-15, atol=1e-15)
    # weighted by 1/multiplicity, dssum reproduces a consistent field
    f = inputs.random_global_field(mesh, seed=2)
    c = ref.inv_multiplicity(mesh.npts, off, idx).reshape(f.shape)
    assert np.allclose(ref.dssum(off, idx, c * f), f, rtol=1e-15, atol=1e-15)


def test_dssum_order_is_left_to_right():
    """Bit-level: group sum taken in ascending local-index order."""
    mesh = inputs.box_mesh(2, 2, 2, 3, perturb=0.0)
    off, idx = ref.gs_build(mesh.glo_num)
    v = inputs.random_local_field(mesh.nelt, 3, seed=1) * np.exp(np.random.default_rng(0).uniform(-20, 20, (8, 27)))
    s = ref.dssum(off, idx, v).reshape(-1)
    vv = v.reshape(-1)
    for g in range(len(off) - 1):
        mem = idx[off[g]:off[g + 1]]
        acc = vv[mem[0]]
        for q in mem[1:]:
            acc = acc + vv[q]
        assert all(s[q] == acc for q in mem)


def _tiny_problem(dims, nx, perturb=0.2, seed=0):
    mesh = inputs.box_mesh(*dims, nx, perturb=perturb, seed=seed)
    return ref.Problem(mesh)


@pytest.mark.parametrize("dims,nx", [((2, 2, 1), 3), ((2, 1, 2), 4), ((2, 2, 2), 3)])
def test_jacobi_diag_matches_dense_assembled(dims, nx):
    P = _tiny_problem(dims, nx)
    A = ref.assembled_matrix(P.D, P.G, P.mesh.glo_num, P.mesh.nglobal)
    dglob = np.diag(A)[P.mesh.glo_num]
    expect = np.where(P.mesh.mask == 1, 1.0 / dglob, 0.0)
    assert np.allclose(P.minv, expect, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dims,nx", [((2, 2, 2), 3), ((2, 2, 1), 4), ((3, 2, 2), 4)])
def test_pcg_matches_dense_direct_solve(dims, nx):
    P = _tiny_problem(dims, nx, seed=1)
    mesh = P.mesh
    f = inputs.random_global_field(mesh, seed=3)
    st, x, it, rr = ref.pcg(P.D, P.G, P.offsets, P.idx, mesh.mask, P.minv, f, tol=1e-13, max_iter=500)
    assert st == ref.OK and rr <= 1e-13
    A = ref.assembled_matrix(P.D, P.G, mesh.glo_num, mesh.nglobal)
    free = np.zeros(mesh.nglobal, dtype=bool)
    free[mesh.glo_num[mesh.mask == 1]] = True
    fg = np.zeros(mesh.nglobal)
    fg[mesh.glo_num.reshape(-1)] = f.reshape(-1)
    xg = np.zeros(mesh.nglobal)
    Aff = A[np.ix_(free, free)]
    np.linalg.cholesky(Aff)  # SPD after masking
    xg[free] = np.linalg.solve(Aff, fg[free])
    assert np.max(np.abs(x - xg[mesh.glo_num])) <= 1e-10 * np.max(np.abs(xg))
    # PCG in exact arithmetic ends in at most (#unknowns) iterations
    assert it <= int(free.sum()) + 2


def test_pcg_no_unknowns():
    P = _tiny_problem((1, 1, 1), 2, perturb=0.0)
    f = inputs.random_global_field(P.mesh, seed=1)
    st, x, it, rr = ref.pcg(P.D, P.G, P.offsets, P.idx, P.mesh.mask, P.minv, f, tol=1e-8)
    assert st == ref.OK and it == 0 and np.all(x == 0)


def test_pcg_one_unknown():
    P = _tiny_problem((1, 1, 1), 3, perturb=0.0)
    f = inputs.random_global_field(P.mesh, seed=1)
    st, x, it, rr = ref.pcg(P.D, P.G, P.offsets, P.idx, P.mesh.mask, P.minv, f, tol=1e-12)
    assert st == ref.OK and it == 1
    c = 13  # centre node (1,1,1) of a 3^3 element
    A_pp = ref.element_matrix(P.D, P.G[0])[c, c]
    assert abs(x[0, c] - f[0, c] / A_pp) <= 1e-14 * abs(f[0, c] / A_pp)
    assert np.count_nonzero(x) == 1


def test_pcg_fixed_iterations_and_breakdown():
    P = _tiny_problem((2, 2, 2), 4, seed=2)
    f = inputs.random_global_field(P.mesh, seed=4)
    st, x, it, rr = ref.pcg(P.D, P.G, P.offsets, P.idx, P.mesh.mask, P.minv, f, tol=0.0, max_iter=7)
    assert st == ref.OK and it == 7
    st, x, it, rr = ref.pcg(P.D, P.G, P.offsets, P.idx, P.mesh.mask, P.minv, f, tol=1e-30, max_iter=3)
    assert st == ref.NOT_CONVERGED and it == 3
    # an indefinite operator (negated G) gives p.Ap < 0 -> breakdown on the first iteration
    st, x, it, rr = ref.pcg(P.D, -P.G, P.offsets, P.idx, P.mesh.mask, np.abs(P.minv), f, tol=1e-8)
    assert st == ref.BREAKDOWN and it == 1
    fn = f.copy()
    fn[0, 42] = np.nan  # node (2,2,2) of element 0: interior, not masked
    st, x, it, rr = ref.pcg(P.D, P.G, P.offsets, P.idx, P.mesh.mask, P.minv, fn, tol=1e-8)
    assert st == ref.BREAKDOWN


@pytest.mark.parametrize("dims,nx", [((2, 2, 2), 4), ((3, 2, 2), 6), ((2, 3, 2), 10)])
def test_element_energies_give_the_cg_inner_product(dims, nx):
    """The identity the GPU solve uses for <p,w>: for p continuous across elements and zero on the
    mask, <p, mask.dssum(A_L p)>_c equals the sum over elements of p_e . (A_e p_e).  A discontinuous p,
    or one that is not zero on the mask, breaks it (so the check is not vacuous)."""
    mesh = inputs.box_mesh(*dims, nx, perturb=0.15, seed=nx)
    P = ref.Problem(mesh)
    p = ref.mask_apply(mesh.mask, inputs.random_global_field(mesh, seed=3))
    lhs = float(np.sum(P.c * p * P.apply(p)))
    rhs = float(np.sum(p * ref.ax(P.D, P.G, p)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert lhs > 0.0
    for v in (inputs.random_local_field(mesh.nelt, nx, seed=4),  # a different value in every copy of a node
              inputs.random_global_field(mesh, seed=5)):  # continuous but not zero on the mask
        e_sum = float(np.sum(v * ref.ax(P.D, P.G, v)))
        assert abs(float(np.sum(P.c * v * P.apply(v))) - e_sum) > 1e-6 * abs(e_sum)


def test_openmp_build_is_the_same_oracle():
    """The -fopenmp build (used only to time the oracle on all host cores) splits
    independent loops only: AX, dssum and 12 PCG iterations are bit-identical to
    the default build's."""
    so = ref.openmp_library()
    if so is None:
        pytest.skip("no OpenMP-capable C compiler on this host")
    mesh = inputs.box_mesh(5, 4, 3, 7, perturb=0.15, seed=11)
    P = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=12)
    u = inputs.random_local_field(mesh.nelt, 7, seed=13)
    base = (ref.ax(P.D, P.G, u), ref.dssum(P.offsets, P.idx, u),
            ref.pcg(P.D, P.G, P.offsets, P.idx, mesh.mask, P.minv, f, 0.0, 12))
    with ref.using_library(so):
        omp = (ref.ax(P.D, P.G, u), ref.dssum(P.offsets, P.idx, u),
               ref.pcg(P.D, P.G, P.offsets, P.idx, mesh.mask, P.minv, f, 0.0, 12))
    assert np.array_equal(base[0], omp[0]) and np.array_equal(base[1], omp[1])
    assert np.array_equal(base[2][1], omp[2][1]) and base[2][3] == omp[2][3]
