"""GPU parity of the unique-node (L-vector) form against the oracle.

Bars: the plan's maps, scatter, restriction and the assembly of integer-valued
inputs bit-exact; the assembled operator within 1e-12 relative in the max norm
(the same bound as the element operator, which dominates the rounding); the
Jacobi diagonal within 1e-14; the solve to the oracle's iteration count within
2 with a solution whose residual, recomputed by the oracle, meets the
tolerance; and, at the bench's full size, the same iterates as the E-vector
solve on the device (x_E = Q x_L within 1e-10 after 100 fixed iterations).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import lvec as olv  # noqa: E402
from oracle import ref  # noqa: E402
from paper_2011_04981_gb300 import inputs, nekax  # noqa: E402
from paper_2011_04981_gb300.problem import DeviceProblem  # noqa: E402

DEV = "cuda"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    nekax.load()


def _shuffled_mesh(dims, nx, seed):
    """A box mesh whose global ids are permuted and spread out (not 0..n-1), to exercise the ordering."""
    mesh = inputs.box_mesh(*dims, nx, perturb=0.15, seed=seed)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(mesh.nglobal) * 7 + 3
    mesh.glo_num = perm[mesh.glo_num]
    return mesh


@pytest.mark.parametrize("dims,nx", [((3, 2, 1), 3), ((2, 2, 2), 8), ((5, 1, 1), 10), ((1, 1, 1), 2)])
def test_maps_bit_exact(dims, nx):
    mesh = _shuffled_mesh(dims, nx, seed=nx)
    l2g, mL, nL = olv.build(mesh.glo_num, mesh.mask)
    lv = nekax.LvecPlan(mesh.glo_num, mesh.mask)
    assert lv.size == nL
    # scatter of distinct values reveals l2g exactly
    uL = _t(np.arange(nL, dtype=np.float64) * 1.5 - 11.0)
    uE = torch.full((mesh.npts,), float("nan"), dtype=torch.float64, device=DEV)
    lv.scatter(uL, uE)
    assert np.array_equal(uE.cpu().numpy(), (np.arange(nL) * 1.5 - 11.0)[l2g.reshape(-1)])
    back = torch.full((nL,), float("nan"), dtype=torch.float64, device=DEV)
    lv.restrict(uE, back)
    assert torch.equal(back, uL)
    # integer-valued copies: the sum over copies is exact in any order, so bit-exact
    wE = np.random.default_rng(1).integers(-1000, 1000, size=mesh.npts).astype(np.float64)
    wL = torch.full((nL,), float("nan"), dtype=torch.float64, device=DEV)
    lv.assemble(_t(wE), wL)
    assert np.array_equal(wL.cpu().numpy(), olv.assemble(l2g, nL, wE))


@pytest.mark.parametrize("dims,nx", [((3, 2, 2), 4), ((2, 2, 2), 8), ((3, 1, 2), 10), ((2, 1, 1), 12),
                                     ((1, 2, 1), 16), ((2, 2, 1), 7)])
def test_ax_and_jacobi_parity(dims, nx):
    mesh = _shuffled_mesh(dims, nx, seed=nx + 10)
    l2g, mL, nL = olv.build(mesh.glo_num, mesh.mask)
    P = DeviceProblem(mesh, DEV, build_minv=False)
    Gff = P.prepare_ff()
    lv = nekax.LvecPlan(mesh.glo_num, mesh.mask)
    Gh = P.G.cpu().numpy()
    Dh = P.D_host
    u = np.random.default_rng(nx).uniform(-1, 1, nL)
    wL = torch.full((nL,), float("nan"), dtype=torch.float64, device=DEV)
    wE = torch.empty(mesh.npts, dtype=torch.float64, device=DEV)
    lv.ax_ff(mesh.nelt, nx, P.D, Gff, _t(u), wL, wE)
    # scale: the sum over copies of |element result|, which bounds the rounding of the sum
    wloc = ref.ax(Dh, Gh, olv.gather(l2g, u))
    scale = float(np.max(olv.assemble(l2g, nL, np.abs(wloc))))
    assert float(np.max(np.abs(wL.cpu().numpy() - olv.assemble(l2g, nL, wloc)))) <= 1e-12 * scale
    minv = torch.full((nL,), float("nan"), dtype=torch.float64, device=DEV)
    lv.jacobi_minv(mesh.nelt, nx, P.D, P.G, minv, wE)
    ref_minv = olv.jacobi_minv(Dh, Gh, l2g, nL, mL)
    assert _rel(minv.cpu().numpy(), ref_minv) <= 1e-14
    assert np.all(minv.cpu().numpy()[mL == 0] == 0.0)


@pytest.mark.parametrize("dims,nx", [((3, 3, 2), 6), ((4, 3, 3), 8), ((3, 2, 2), 10)])
def test_cg_parity(dims, nx):
    mesh = inputs.box_mesh(*dims, nx, perturb=0.1, seed=3)
    P = DeviceProblem(mesh, DEV)
    l2g, mL, nL = olv.build(mesh.glo_num, mesh.mask)
    Pr = ref.Problem(mesh)
    g = np.random.default_rng(4).uniform(-1, 1, nL)
    xL = torch.full((nL,), float("nan"), dtype=torch.float64, device=DEV)
    res = P.cg_lvec(_t(g), xL, tol=1e-8, max_iter=3000)
    assert res["status"] == nekax.OK, res
    minv = olv.jacobi_minv(Pr.D, Pr.G, l2g, nL, mL)
    xr, itr, rr = olv.pcg(Pr.D, Pr.G, l2g, nL, mL, minv, g, 1e-8, 3000)
    assert abs(res["iters"] - itr) <= 2, (res["iters"], itr)
    x = xL.cpu().numpy()
    # residual recomputed by the oracle in the E-vector form: same system
    assert Pr.residual(g[l2g], x[l2g]) <= 1e-8 * (1 + 1e-3)
    assert _rel(x, xr) <= 1e-6
    assert np.all(x[mL == 0] == 0.0)


def test_cg_fixed_iterations_check_every_and_timing():
    mesh = inputs.box_mesh(4, 3, 3, 8, perturb=0.1, seed=7)
    P = DeviceProblem(mesh, DEV)
    l2g, mL, nL = olv.build(mesh.glo_num, mesh.mask)
    Pr = ref.Problem(mesh)
    g = np.random.default_rng(2).uniform(-1, 1, nL)
    x1 = torch.empty(nL, dtype=torch.float64, device=DEV)
    x2 = torch.empty(nL, dtype=torch.float64, device=DEV)
    r = P.cg_lvec(_t(g), x1, tol=0.0, max_iter=25, time_ax=True)
    assert r["status"] == nekax.OK and r["iters"] == 25 and r["ax_launches"] == 25 and r["ax_ms_total"] > 0
    xr, itr, rr = olv.pcg(Pr.D, Pr.G, l2g, nL, mL, olv.jacobi_minv(Pr.D, Pr.G, l2g, nL, mL), g, 0.0, 25)
    assert _rel(x1.cpu().numpy(), xr) <= 1e-9
    assert abs(r["relres"] - rr) <= 1e-6 * rr
    ra = P.cg_lvec(_t(g), x1, tol=1e-9, max_iter=2000, check_every=1)
    rb = P.cg_lvec(_t(g), x2, tol=1e-9, max_iter=2000, check_every=9)
    assert ra["status"] == rb["status"] == nekax.OK and ra["iters"] == rb["iters"]
    assert torch.equal(x1, x2)


def test_special_cases_and_argument_checks():
    # every node on the boundary: 0 iterations, x = 0
    m0 = inputs.box_mesh(1, 1, 1, 2, perturb=0.0)
    P0 = DeviceProblem(m0, DEV)
    lv0 = P0.lvec()[0]
    x0 = torch.full((lv0.size,), 5.0, dtype=torch.float64, device=DEV)
    r = P0.cg_lvec(torch.ones(lv0.size, dtype=torch.float64, device=DEV), x0, tol=1e-8)
    assert r["status"] == nekax.OK and r["iters"] == 0 and float(x0.abs().max()) == 0.0
    # copies of a node that disagree on the mask are rejected
    m = inputs.box_mesh(2, 1, 1, 3, perturb=0.0)
    bad = m.mask.copy()
    shared = np.flatnonzero(np.bincount(m.glo_num.reshape(-1)) == 2)
    p = int(np.flatnonzero(m.glo_num.reshape(-1) == shared[0])[0])
    bad.reshape(-1)[p] ^= 1
    with pytest.raises(nekax.NekError):
        nekax.LvecPlan(m.glo_num, bad)
    # a plan for another size is rejected by the operator
    P = DeviceProblem(m, DEV)
    lv = P.lvec()[0]
    wL = torch.empty(lv.size, dtype=torch.float64, device=DEV)
    wE = torch.empty(m.npts, dtype=torch.float64, device=DEV)
    with pytest.raises(nekax.NekError):
        lv.ax_ff(m.nelt - 1, 3, P.D, P.prepare_ff(), wL.clone(), wL, wE)


def test_full_size_same_iterates_as_element_vector_solve():
    """32x32x32 elements at nx = 10 (the bench workload), 100 fixed iterations of both forms."""
    mesh = inputs.box_mesh(32, 32, 32, 10, perturb=0.1, seed=1)
    P = DeviceProblem(mesh, DEV)
    lv, minvL, _ = P.lvec()
    gL = np.random.default_rng(9).uniform(-1, 1, lv.size)
    fL = _t(gL)
    fE = torch.empty(mesh.npts, dtype=torch.float64, device=DEV)
    lv.scatter(fL, fE)
    xE = torch.empty_like(fE)
    rE = P.cg(fE, xE, tol=0.0, max_iter=100, ax_impl=nekax.AX_FF)
    xL = torch.empty_like(fL)
    rL = P.cg_lvec(fL, xL, tol=0.0, max_iter=100)
    assert rE["status"] == rL["status"] == nekax.OK
    xLE = torch.empty_like(fE)
    lv.scatter(xL, xLE)
    err = float((xLE - xE).abs().max() / xE.abs().max())
    assert err <= 1e-10, err
    assert abs(rL["relres"] - rE["relres"]) <= 1e-8 * rE["relres"]
    # sampled oracle check of the assembled operator on a few interior nodes
    wL = torch.empty_like(fL)
    wE = torch.empty_like(fE)
    lv.ax_ff(mesh.nelt, 10, P.D, P.prepare_ff(), fL, wL, wE)
    Gh_rows = {}
    rng = np.random.default_rng(0)
    glo = mesh.glo_num
    D = P.D_host
    for e in rng.choice(mesh.nelt, size=4, replace=False):
        for p in rng.choice(1000, size=3, replace=False):
            gid = int(glo[e, p])
            elems = np.flatnonzero(np.any(glo == gid, axis=1))
            tot, scale = 0.0, 0.0
            for ee in elems:
                if ee not in Gh_rows:
                    Gh_rows[ee] = P.G[ee].cpu().numpy()[None]
                ue = gL[glo[ee]][None]  # glo is the lattice numbering: L index = global id
                we = ref.ax(D, Gh_rows[ee], ue)[0]
                tot += float(np.sum(we[glo[ee] == gid]))
                scale += float(np.max(np.abs(we)))  # the max-norm scale of the element result
            got = float(wL[gid])
            assert abs(got - tot) <= 1e-12 * scale, (e, p, got, tot)
