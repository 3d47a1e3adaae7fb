"""GPU parity of the tensor-core FP64-accurate operator (nek_ax_oz) against the oracle.

The operator of Section II-B (Listing 1) with its contractions as BF16-digit
MMAs summed exactly per level: the same 1e-12 bound (relative, max norm) as
the FP64 and float-float kernels, on several CTAs, a ragged last CTA and, with
more elements than the persistent grid, several elements per CTA.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import ref  # noqa: E402
from paper_2011_04981_gb300 import inputs, nekax  # noqa: E402

DEV = "cuda"
TOL_AX = 1e-12
NXS = [2, 4, 6, 8, 10]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    nekax.load()


def _case(nx, nelt, seed, perturb=0.2):
    rng = np.random.default_rng(seed)
    xi, rho, D = ref.gll(nx)
    mesh = inputs.box_mesh(nelt, 1, 1, nx, perturb=perturb, seed=seed % 97)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = rng.uniform(-1, 1, size=(nelt, nx ** 3))
    return D, G, u


def _run(nx, D, G, u):
    nelt = u.shape[0]
    Goz = torch.empty((nelt, nx ** 3, 12), dtype=torch.float32, device=DEV)
    nekax.geom_oz(nelt, nx, _t(G), Goz)
    wd = torch.full((nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    nekax.ax_oz(nelt, nx, _t(D), Goz, _t(u), wd)
    torch.cuda.synchronize()
    return wd.cpu().numpy()


@pytest.mark.parametrize("nx", NXS)
@pytest.mark.parametrize("nelt", [1, 7, 37, 700])
def test_ax_oz_parity_sweep(nx, nelt):
    D, G, u = _case(nx, nelt, nx * 1000 + nelt)
    w = _run(nx, D, G, u)
    assert np.all(np.isfinite(w)), "unwritten output entries"
    wr = ref.ax(D, G, u)
    assert _rel(w, wr) <= TOL_AX
    # and element by element, against each element's own largest |w|
    err = np.max(np.abs(w - wr), axis=1) / np.max(np.abs(wr), axis=1)
    assert np.all(err <= TOL_AX), (int(np.argmax(err)), float(err.max()))


@pytest.mark.parametrize("nx", [4, 10])
def test_ax_oz_result_independent_of_the_cta(nx):
    """Each element's arithmetic is fixed by its data: the first 37 elements give bit-identical results
    whether they are alone (one element per CTA) or part of a 700-element launch (several per CTA)."""
    D, G, u = _case(nx, 700, 5)
    w_all = _run(nx, D, G, u)
    w_few = _run(nx, D, G[:37], u[:37])
    assert np.array_equal(w_all[:37], w_few)


@pytest.mark.parametrize("nx", [8, 10])
def test_ax_oz_wide_dynamic_range(nx):
    """u spanning 1e-9..1 inside an element and 1e-6..1e3 across elements: 1e-12 norm-wise per element."""
    rng = np.random.default_rng(nx)
    nelt = 9
    xi, rho, D = ref.gll(nx)
    mesh = inputs.box_mesh(3, 3, 1, nx, perturb=0.15, seed=nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = rng.uniform(-1, 1, size=(nelt, nx ** 3)) * 10.0 ** rng.uniform(-9, 0, size=(nelt, nx ** 3))
    u *= 10.0 ** np.linspace(-6, 3, nelt)[:, None]
    w = _run(nx, D, G, u)
    wr = ref.ax(D, G, u)
    for e in range(nelt):
        assert _rel(w[e], wr[e]) <= TOL_AX, e


def test_ax_oz_zero_and_constant_inputs():
    """u = 0 gives w = 0 exactly; u constant on an element is in the operator's null space (derivatives
    of a constant vanish), so w is at rounding level of the scale."""
    nx = 10
    D, G, u = _case(nx, 5, 11)
    u[0] = 0.0
    u[1] = 3.25
    w = _run(nx, D, G, u)
    assert np.all(w[0] == 0.0)
    wr = ref.ax(D, G, u)
    assert np.max(np.abs(w[1] - wr[1])) <= 1e-12 * np.abs(D).sum(axis=1).max() ** 2 * np.abs(G[1]).max() * 3.25
    assert _rel(w[2:], wr[2:]) <= TOL_AX


def test_ax_oz_full_size_sampled():
    """The 32x32x32 deformed box at nx = 10 (32768 elements): 98 sampled elements against the oracle."""
    nx = 10
    mesh = inputs.box_mesh(32, 32, 32, nx, perturb=0.1, seed=2)
    from paper_2011_04981_gb300.problem import DeviceProblem

    P = DeviceProblem(mesh, DEV, build_minv=False)
    u = inputs.random_local_field(mesh.nelt, nx, seed=5)
    w = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    P.ax_oz(_t(u), w)
    torch.cuda.synchronize()
    wn = w.cpu().numpy()
    assert np.all(np.isfinite(wn))
    sample = np.concatenate([np.random.default_rng(1).choice(mesh.nelt, size=96, replace=False),
                             [0, mesh.nelt - 1]])
    xi, rho, D = ref.gll(nx)
    G = ref.geom(mesh.corners[sample], nx, xi, rho)
    assert _rel(wn[sample], ref.ax(D, G, u[sample])) <= TOL_AX


def test_geom_oz_is_the_float_float_split_interleaved_by_point_pairs():
    nx = 6
    mesh = inputs.box_mesh(3, 2, 1, nx, perturb=0.2, seed=4)
    G = ref.geom(mesh.corners, nx)
    Gd = _t(G)
    Gff = torch.empty((mesh.nelt, nx ** 3, 12), dtype=torch.float32, device=DEV)
    Goz = torch.empty_like(Gff)
    nekax.geom_ff(mesh.nelt, nx, Gd, Gff)
    nekax.geom_oz(mesh.nelt, nx, Gd, Goz)
    torch.cuda.synchronize()
    f = Gff.cpu().numpy().reshape(mesh.nelt, nx ** 3 // 2, 2, 6, 2)  # [e][pair][point][c][hi/lo]
    z = Goz.cpu().numpy().reshape(mesh.nelt, nx ** 3 // 2, 6, 2, 2)  # [e][pair][c][hi/lo][point]
    assert np.array_equal(z, f.transpose(0, 1, 3, 4, 2))


def test_ax_oz_bounded_wait_runs_out_and_reports():
    """A wait that can never complete (the mbarrier expects one arrival more than the MMAs give) runs out
    after its bound: the kernel flags it, poisons its outputs, frees its tensor memory and returns; a
    normal run afterwards is unaffected."""
    st, to = nekax.ax_oz_selftest(1, 20000)
    assert st == nekax.ERR_TIMEOUT and to == 1
    st, to = nekax.ax_oz_selftest(0, 2000000)
    assert st == nekax.OK and to == 0
    D, G, u = _case(6, 40, 3)
    assert _rel(_run(6, D, G, u), ref.ax(D, G, u)) <= TOL_AX


# ------------------------------------------------------------------ in the Jacobi-PCG solve
@pytest.mark.parametrize("dims,nx", [((3, 3, 3), 6), ((2, 2, 2), 10), ((3, 2, 2), 8), ((3, 3, 3), 2)])
def test_cg_with_oz_operator(dims, nx):
    """The solve with the tensor-core operator (element energies and the fused x / direction update):
    converges to 1e-8 by the oracle's own residual, within 2 iterations of the oracle's count."""
    from paper_2011_04981_gb300.problem import DeviceProblem

    mesh = inputs.box_mesh(*dims, nx, perturb=0.1, seed=3)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=4)
    x = torch.empty((mesh.nelt, nx ** 3), dtype=torch.float64, device=DEV)
    res = P.cg(_t(f), x, tol=1e-8, max_iter=2000, ax_impl=nekax.AX_OZ)
    assert res["status"] == nekax.OK, res
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 1e-8, 2000)
    assert abs(res["iters"] - itr) <= 2, (res["iters"], itr)
    assert Pr.residual(f, x.cpu().numpy()) <= 1e-8 * (1 + 1e-3)
    assert _rel(x.cpu().numpy(), xr) <= 1e-6
    assert np.all(x.cpu().numpy()[mesh.mask == 0] == 0.0)


@pytest.mark.parametrize("nx", [6, 10])
def test_cg_oz_fixed_iterations(nx):
    """After 1, 2 and 23 iterations the iterate matches the oracle's PCG element by element to 1e-9 of
    its scale, and the reported residual to 1e-8 relative."""
    from paper_2011_04981_gb300.problem import DeviceProblem

    mesh = inputs.box_mesh(3, 2, 2, nx, perturb=0.1, seed=7)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=8)
    for its in (1, 2, 23):
        x = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
        res = P.cg(_t(f), x, tol=0.0, max_iter=its, ax_impl=nekax.AX_OZ)
        assert res["status"] == nekax.OK and res["iters"] == its, res
        st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 0.0, its)
        xg = x.cpu().numpy()
        err = np.max(np.abs(xg - xr), axis=1)
        assert np.max(err) <= 1e-9 * np.max(np.abs(xr)), (its, int(np.argmax(err)), float(err.max()))
        assert abs(res["relres"] - rr) <= 1e-8 * rr, (its, res["relres"], rr)


def test_cg_oz_rejects_unsupported_nx_and_missing_split():
    from paper_2011_04981_gb300.problem import DeviceProblem

    mesh = inputs.box_mesh(2, 1, 1, 5, perturb=0.1, seed=3)
    P = DeviceProblem(mesh, DEV)
    f = _t(inputs.random_global_field(mesh, seed=4))
    x = torch.empty_like(f)
    with pytest.raises(nekax.NekError) as ex:
        nekax.cg_solve(P.gs, mesh.nelt, 5, P.D, P.G, P.mask, P.minv, f, x, 1e-8, 10, ax_impl=nekax.AX_OZ,
                       Gff=P.prepare_ff())
    assert ex.value.status == nekax.ERR_UNSUPPORTED_NX
    mesh = inputs.box_mesh(2, 1, 1, 6, perturb=0.1, seed=3)
    P = DeviceProblem(mesh, DEV)
    f = _t(inputs.random_global_field(mesh, seed=4))
    x = torch.empty_like(f)
    with pytest.raises(nekax.NekError) as ex:
        nekax.cg_solve(P.gs, mesh.nelt, 6, P.D, P.G, P.mask, P.minv, f, x, 1e-8, 10, ax_impl=nekax.AX_OZ, Gff=None)
    assert ex.value.status == nekax.ERR_INVALID_ARG
