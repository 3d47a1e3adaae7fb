"""GPU parity: every step of the solve path through the C ABI against the oracle.

Tolerances (FP64 throughout): AX and G within 1e-12 relative in the max norm
(the operator's rounding is O(nx eps) relative to |D|^2|G||u|); gather-scatter
plan and dssum bit-exact (same groups, same left-to-right order); PCG to the
same iteration count within 2 and a solution whose residual, recomputed by the
oracle, meets the tolerance.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import ref  # noqa: E402
from paper_2011_04981_gb300 import inputs, nekax  # noqa: E402
from paper_2011_04981_gb300.problem import DeviceProblem  # noqa: E402

DEV = "cuda"
TOL_AX = 1e-12


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    nekax.load()


# ------------------------------------------------------------------ AX
@pytest.mark.parametrize("nx", list(range(2, 17)))
@pytest.mark.parametrize("nelt", [1, 7, 37])
def test_ax_parity_sweep(nx, nelt):
    """Oracle D and G fed to both sides; several CTAs and a ragged last CTA."""
    rng = np.random.default_rng(nx * 100 + nelt)
    xi, rho, D = ref.gll(nx)
    mesh = inputs.box_mesh(nelt, 1, 1, nx, perturb=0.2, seed=nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = rng.uniform(-1, 1, size=(nelt, nx ** 3))
    wd = torch.full((nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    nekax.ax(nelt, nx, _t(D), _t(G), _t(u), wd)
    torch.cuda.synchronize()
    w = wd.cpu().numpy()
    assert np.all(np.isfinite(w)), "unwritten output entries"
    assert _rel(w, ref.ax(D, G, u)) <= TOL_AX


def test_ax_config1_64_elements_nx8():
    """4x4x4 unit-cube box, nx=8, perturbation 0.05 h, G from the library's own set-up."""
    mesh = inputs.box_mesh(4, 4, 4, 8, perturb=0.05, seed=1)
    P = DeviceProblem(mesh, DEV, build_minv=False)
    Pr = ref.Problem(mesh)
    u = inputs.random_local_field(mesh.nelt, 8, seed=1)
    w = torch.empty((mesh.nelt, 512), dtype=torch.float64, device=DEV)
    P.ax(_t(u), w)
    torch.cuda.synchronize()
    assert _rel(w.cpu().numpy(), ref.ax(Pr.D, Pr.G, u)) <= TOL_AX


def test_ax_full_size_sampled():
    """32768 elements at nx=10 (the benchmark's launch), checked on sampled elements."""
    nx = 10
    mesh = inputs.box_mesh(32, 32, 32, nx, perturb=0.1, seed=2)
    P = DeviceProblem(mesh, DEV, build_minv=False)
    u = inputs.random_local_field(mesh.nelt, nx, seed=5)
    w = torch.empty((mesh.nelt, nx ** 3), dtype=torch.float64, device=DEV)
    P.ax(_t(u), w)
    torch.cuda.synchronize()
    sample = np.random.default_rng(0).choice(mesh.nelt, size=96, replace=False)
    sample = np.concatenate([sample, [0, 1, mesh.nelt - 1]])
    xi, rho, D = ref.gll(nx)
    G = ref.geom(mesh.corners[sample], nx, xi, rho)
    assert _rel(w.cpu().numpy()[sample], ref.ax(D, G, u[sample])) <= TOL_AX


def test_ax_on_side_stream_and_empty():
    nx = 6
    xi, rho, D = ref.gll(nx)
    mesh = inputs.box_mesh(5, 3, 1, nx, perturb=0.1)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = inputs.random_local_field(mesh.nelt, nx)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Dd, Gd, ud = _t(D), _t(G), _t(u)
        wd = torch.empty_like(ud)
        nekax.ax(mesh.nelt, nx, Dd, Gd, ud, wd, stream=s)
    s.synchronize()
    assert _rel(wd.cpu().numpy(), ref.ax(D, G, u)) <= TOL_AX
    nekax.ax(0, nx, Dd, Gd, ud, wd)  # no-op


def test_ax_constant_in_kernel_on_gpu():
    nx = 12
    mesh = inputs.box_mesh(3, 3, 3, nx, perturb=0.2, seed=9)
    P = DeviceProblem(mesh, DEV, build_minv=False)
    u = torch.full((mesh.nelt, nx ** 3), 2.0, dtype=torch.float64, device=DEV)
    w = torch.empty_like(u)
    P.ax(u, w)
    Gmax = float(P.G.abs().max())
    Dmax = float(np.abs(P.D_host).max())
    assert float(w.abs().max()) <= 8 * nx * 2.2e-16 * Gmax * Dmax ** 2 * nx * 2.0 * 6


# ------------------------------------------------------------------ geometry
@pytest.mark.parametrize("nx", [2, 5, 8, 10, 16])
def test_geom_parity(nx):
    mesh = inputs.box_mesh(3, 2, 2, nx, perturb=0.15, seed=nx, lengths=(1.0, 2.0, 0.5))
    G = torch.empty((mesh.nelt, nx ** 3, 6), dtype=torch.float64, device=DEV)
    nekax.geom(mesh.nelt, nx, _t(mesh.corners), G)
    torch.cuda.synchronize()
    Gr = ref.geom(mesh.corners, nx)
    assert _rel(G.cpu().numpy(), Gr) <= 1e-13


# ------------------------------------------------------------------ gather-scatter / mask
@pytest.mark.parametrize("dims,nx", [((1, 1, 1), 2), ((2, 3, 2), 4), ((4, 4, 4), 8), ((5, 2, 3), 5)])
def test_gs_plan_bit_exact(dims, nx):
    mesh = inputs.box_mesh(*dims, nx, perturb=0.0)
    gs = nekax.GsPlan(mesh.nelt, nx, mesh.glo_num)
    off, mem = gs.export()
    ro, rm = ref.gs_build(mesh.glo_num)
    assert np.array_equal(off, ro) and np.array_equal(mem, rm)
    npts, ng, ns = gs.info()
    assert npts == mesh.npts and ng == len(ro) - 1 and ns == len(rm)


def test_gs_plan_non_lattice_ids():
    """Sparse, shuffled global ids (the sort-based plan path)."""
    rng = np.random.default_rng(4)
    glo = rng.integers(0, 40, size=(3, 27)) * 1_000_003
    gs = nekax.GsPlan(3, 3, glo)
    off, mem = gs.export()
    ro, rm = ref.gs_build(glo)
    assert np.array_equal(off, ro) and np.array_equal(mem, rm)


@pytest.mark.parametrize("dims,nx", [((3, 3, 3), 5), ((8, 4, 2), 10)])
def test_dssum_bit_exact(dims, nx):
    mesh = inputs.box_mesh(*dims, nx, perturb=0.0)
    gs = nekax.GsPlan(mesh.nelt, nx, mesh.glo_num)
    v = inputs.random_local_field(mesh.nelt, nx, seed=3) * 10.0 ** np.random.default_rng(1).uniform(-8, 8, (1, nx ** 3))
    vd = _t(v)
    gs.dssum(vd)
    ro, rm = ref.gs_build(mesh.glo_num)
    assert np.array_equal(vd.cpu().numpy(), ref.dssum(ro, rm, v))
    c = torch.empty_like(vd)
    gs.inv_multiplicity(c)
    assert np.array_equal(c.cpu().numpy().reshape(-1), ref.inv_multiplicity(mesh.npts, ro, rm))


def test_mask_and_dot():
    mesh = inputs.box_mesh(4, 3, 2, 6, perturb=0.1)
    gs = nekax.GsPlan(mesh.nelt, 6, mesh.glo_num)
    v = inputs.random_local_field(mesh.nelt, 6, seed=8)
    vd = _t(v)
    nekax.mask(mesh.npts, _t(mesh.mask), vd)
    assert np.array_equal(vd.cpu().numpy(), ref.mask_apply(mesh.mask, v))
    a = inputs.random_global_field(mesh, seed=1)
    b = inputs.random_global_field(mesh, seed=2)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    nekax.dot_c(gs, _t(a), _t(b), out)
    ro, rm = ref.gs_build(mesh.glo_num)
    c = ref.inv_multiplicity(mesh.npts, ro, rm)
    expect = float(np.sum(c * a.reshape(-1) * b.reshape(-1)))
    assert abs(float(out.item()) - expect) <= 1e-13 * np.sum(np.abs(c * a.reshape(-1) * b.reshape(-1)))


# ------------------------------------------------------------------ Jacobi / CG
@pytest.mark.parametrize("dims,nx", [((2, 2, 2), 4), ((4, 3, 2), 7)])
def test_jacobi_minv_parity(dims, nx):
    mesh = inputs.box_mesh(*dims, nx, perturb=0.15, seed=2)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    assert _rel(P.minv.cpu().numpy(), Pr.minv) <= 1e-13


@pytest.mark.parametrize("dims,nx", [((3, 3, 3), 6), ((4, 2, 3), 8), ((2, 2, 2), 10)])
def test_cg_parity(dims, nx):
    mesh = inputs.box_mesh(*dims, nx, perturb=0.1, seed=3)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=4)
    x = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    res = P.cg(_t(f), x, tol=1e-8, max_iter=2000)
    assert res["status"] == nekax.OK, res
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 1e-8, 2000)
    assert st == ref.OK
    assert abs(res["iters"] - itr) <= 2, (res["iters"], itr)
    xg = x.cpu().numpy()
    assert Pr.residual(f, xg) <= 1e-8 * (1 + 1e-3)
    assert _rel(xg, xr) <= 1e-6


def test_cg_check_every_does_not_change_result():
    mesh = inputs.box_mesh(3, 3, 2, 6, perturb=0.1, seed=6)
    P = DeviceProblem(mesh, DEV)
    f = _t(inputs.random_global_field(mesh, seed=1))
    x1 = torch.empty_like(f)
    x2 = torch.empty_like(f)
    r1 = P.cg(f, x1, tol=1e-9, max_iter=1000, check_every=1)
    r2 = P.cg(f, x2, tol=1e-9, max_iter=1000, check_every=7)
    assert r1["status"] == r2["status"] == nekax.OK
    assert r1["iters"] == r2["iters"]
    assert torch.equal(x1, x2)


def test_cg_fixed_iterations_and_timing():
    mesh = inputs.box_mesh(4, 4, 4, 8, perturb=0.1, seed=7)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=2)
    x = torch.empty((mesh.nelt, 512), dtype=torch.float64, device=DEV)
    ws = torch.empty(nekax.cg_workspace_bytes(mesh.nelt, 8, False) // 8 + 32, dtype=torch.float64, device=DEV)
    res = P.cg(_t(f), x, tol=0.0, max_iter=25, workspace=ws, time_ax=True)
    assert res["status"] == nekax.OK and res["iters"] == 25
    assert res["ax_launches"] == 25 and res["ax_ms_total"] > 0
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 0.0, 25)
    assert itr == 25
    assert _rel(x.cpu().numpy(), xr) <= 1e-9
    assert abs(res["relres"] - rr) <= 1e-6 * rr


def test_cg_special_cases_and_failures():
    # no unknowns: x = 0, 0 iterations
    m0 = inputs.box_mesh(1, 1, 1, 2, perturb=0.0)
    P0 = DeviceProblem(m0, DEV)
    f0 = _t(inputs.random_global_field(m0, seed=1))
    x0 = torch.full_like(f0, 7.0)
    r = P0.cg(f0, x0, tol=1e-8)
    assert r["status"] == nekax.OK and r["iters"] == 0 and float(x0.abs().max()) == 0.0
    # one unknown: one iteration, x = b / A_pp
    m1 = inputs.box_mesh(1, 1, 1, 3, perturb=0.0)
    P1 = DeviceProblem(m1, DEV)
    f1 = inputs.random_global_field(m1, seed=1)
    x1 = torch.empty((1, 27), dtype=torch.float64, device=DEV)
    r = P1.cg(_t(f1), x1, tol=1e-12)
    assert r["status"] == nekax.OK and r["iters"] == 1
    Pr = ref.Problem(m1)
    A_pp = ref.element_matrix(Pr.D, Pr.G[0])[13, 13]
    assert abs(float(x1[0, 13]) - f1[0, 13] / A_pp) <= 1e-14 * abs(f1[0, 13] / A_pp)
    # max_iter reached
    m = inputs.box_mesh(3, 3, 3, 6, perturb=0.1, seed=2)
    P = DeviceProblem(m, DEV)
    f = _t(inputs.random_global_field(m, seed=3))
    x = torch.empty_like(f)
    r = P.cg(f, x, tol=1e-14, max_iter=3)
    assert r["status"] == nekax.ERR_NOT_CONVERGED and r["iters"] == 3
    # NaN in f -> breakdown
    fn = f.clone()
    fn[13, 3 + 6 * 3 + 36 * 3] = float("nan")  # node (3,3,3) of the centre element: interior
    r = P.cg(fn, x, tol=1e-8, max_iter=50)
    assert r["status"] == nekax.ERR_BREAKDOWN
    # indefinite operator (negated G) -> p.Ap <= 0 -> breakdown on the first iteration
    r = nekax.cg_solve(P.gs, m.nelt, 6, P.D, -P.G, P.mask, P.minv.abs(), f, x, 1e-8, 50)
    assert r["status"] == nekax.ERR_BREAKDOWN and r["iters"] == 1


# ------------------------------------------------------------------ FP64-accurate float-float AX
@pytest.mark.parametrize("nx", list(range(2, 17)))
@pytest.mark.parametrize("nelt", [1, 7, 37])
def test_ax_ff_parity_sweep(nx, nelt):
    """Same bound as the FP64 kernel: 1e-12 relative in the max norm."""
    rng = np.random.default_rng(nx * 1000 + nelt)
    xi, rho, D = ref.gll(nx)
    mesh = inputs.box_mesh(nelt, 1, 1, nx, perturb=0.2, seed=nx + 1)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = rng.uniform(-1, 1, size=(nelt, nx ** 3))
    Gd = _t(G)
    Gff = torch.empty((nelt, nx ** 3, 12), dtype=torch.float32, device=DEV)
    nekax.geom_ff(nelt, nx, Gd, Gff)
    wd = torch.full((nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    nekax.ax_ff(nelt, nx, _t(D), Gff, _t(u), wd)
    torch.cuda.synchronize()
    w = wd.cpu().numpy()
    assert np.all(np.isfinite(w)), "unwritten output entries"
    assert _rel(w, ref.ax(D, G, u)) <= TOL_AX


@pytest.mark.parametrize("nx", [3, 8, 10, 13])
def test_ax_ff_energy_matches_oracle_and_ignores_epb(nx):
    """edot[e] = u_e . (A_e u_e): against the oracle's operator, and bit-identical whatever the tuned
    elements per CTA (each element's sum runs in an order fixed by nx)."""
    rng = np.random.default_rng(40 + nx)
    nelt = 11
    xi, rho, D = ref.gll(nx)
    mesh = inputs.box_mesh(nelt, 1, 1, nx, perturb=0.2, seed=nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = rng.uniform(-1, 1, size=(nelt, nx ** 3))
    Gff = torch.empty((nelt, nx ** 3, 12), dtype=torch.float32, device=DEV)
    nekax.geom_ff(nelt, nx, _t(G), Gff)
    wr = ref.ax(D, G, u)
    eref = np.einsum("ep,ep->e", u, wr)
    bound = 1e-12 * np.abs(wr).max(axis=1) * np.abs(u).sum(axis=1) + 1e-13 * np.abs(u * wr).sum(axis=1)
    lib = nekax.load()
    outs = []
    try:
        for epb in (1, 2, 4):
            if lib.nek_set_ax_epb(int(nekax.AX_FF), nx, epb) != nekax.OK:
                continue
            w = torch.full((nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
            ed = torch.full((nelt,), float("nan"), dtype=torch.float64, device=DEV)
            nekax.ax_ff_energy(nelt, nx, _t(D), Gff, _t(u), w, ed)
            torch.cuda.synchronize()
            assert _rel(w.cpu().numpy(), wr) <= TOL_AX
            e = ed.cpu().numpy()
            assert np.all(np.abs(e - eref) <= bound), (epb, np.max(np.abs(e - eref) / bound))
            outs.append(e)
    finally:
        lib.nek_set_ax_epb(int(nekax.AX_FF), nx, 0)
    assert len(outs) >= 1
    for e in outs[1:]:
        assert np.array_equal(e, outs[0])


def test_geom_ff_split_is_faithful():
    nx = 7
    mesh = inputs.box_mesh(3, 2, 2, nx, perturb=0.2, seed=4)
    G = ref.geom(mesh.corners, nx)
    Gff = torch.empty((mesh.nelt, nx ** 3, 12), dtype=torch.float32, device=DEV)
    nekax.geom_ff(mesh.nelt, nx, _t(G), Gff)
    g = Gff.cpu().numpy().astype(np.float64)
    back = g[..., 0::2] + g[..., 1::2]
    # hi carries the leading 24 bits (truncated), lo the next 23: |G - hi - lo| <= 2^-46 |G|
    assert np.all(np.abs(back - G) <= 2.0 ** -46 * np.abs(G))
    assert np.all(np.abs(g[..., 0::2]) <= np.abs(G)) and np.all(np.abs(G - g[..., 0::2]) <= 2.0 ** -23 * np.abs(G))


@pytest.mark.parametrize("nx", [8, 10, 16])
def test_ax_ff_wide_dynamic_range(nx):
    """u spanning 1e-9..1 inside an element and 1e-6..1e3 across elements: still 1e-12 norm-wise per element."""
    rng = np.random.default_rng(nx)
    nelt = 9
    xi, rho, D = ref.gll(nx)
    mesh = inputs.box_mesh(3, 3, 1, nx, perturb=0.15, seed=nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = rng.uniform(-1, 1, size=(nelt, nx ** 3)) * 10.0 ** rng.uniform(-9, 0, size=(nelt, nx ** 3))
    u *= 10.0 ** np.linspace(-6, 3, nelt)[:, None]
    Gff = torch.empty((nelt, nx ** 3, 12), dtype=torch.float32, device=DEV)
    nekax.geom_ff(nelt, nx, _t(G), Gff)
    wd = torch.empty((nelt, nx ** 3), dtype=torch.float64, device=DEV)
    nekax.ax_ff(nelt, nx, _t(D), Gff, _t(u), wd)
    torch.cuda.synchronize()
    w = wd.cpu().numpy()
    wr = ref.ax(D, G, u)
    for e in range(nelt):
        assert _rel(w[e], wr[e]) <= TOL_AX, e


def test_ax_ff_full_size_sampled():
    nx = 10
    mesh = inputs.box_mesh(32, 32, 32, nx, perturb=0.1, seed=2)
    P = DeviceProblem(mesh, DEV, build_minv=False)
    u = inputs.random_local_field(mesh.nelt, nx, seed=5)
    w = torch.empty((mesh.nelt, nx ** 3), dtype=torch.float64, device=DEV)
    P.ax_ff(_t(u), w)
    torch.cuda.synchronize()
    sample = np.concatenate([np.random.default_rng(1).choice(mesh.nelt, size=96, replace=False),
                             [0, mesh.nelt - 1]])
    xi, rho, D = ref.gll(nx)
    G = ref.geom(mesh.corners[sample], nx, xi, rho)
    assert _rel(w.cpu().numpy()[sample], ref.ax(D, G, u[sample])) <= TOL_AX


@pytest.mark.parametrize("dims,nx", [((3, 3, 3), 6), ((2, 2, 2), 10), ((3, 2, 2), 7)])
def test_cg_with_ff_operator(dims, nx):
    mesh = inputs.box_mesh(*dims, nx, perturb=0.1, seed=3)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=4)
    x = torch.empty((mesh.nelt, nx ** 3), dtype=torch.float64, device=DEV)
    res = P.cg(_t(f), x, tol=1e-8, max_iter=2000, ax_impl=nekax.AX_FF)
    assert res["status"] == nekax.OK, res
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 1e-8, 2000)
    assert abs(res["iters"] - itr) <= 2, (res["iters"], itr)
    assert Pr.residual(f, x.cpu().numpy()) <= 1e-8 * (1 + 1e-3)
    assert _rel(x.cpu().numpy(), xr) <= 1e-6


@pytest.mark.parametrize("nx", [6, 8, 10, 12, 13])
def test_cg_ff_fixed_iterations(nx):
    """After a fixed number of iterations the float-float solve's iterate and
    residual match the oracle's PCG."""
    mesh = inputs.box_mesh(3, 2, 3, nx, perturb=0.1, seed=nx)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=5)
    x = torch.empty((mesh.nelt, nx ** 3), dtype=torch.float64, device=DEV)
    for its in (1, 2, 23):
        res = P.cg(_t(f), x, tol=0.0, max_iter=its, ax_impl=nekax.AX_FF, time_ax=True)
        assert res["status"] == nekax.OK and res["iters"] == its and res["ax_launches"] == its
        # point flags (2), init (2), then per iteration AX (with element energies and the x / direction
        # update), dssum, alpha, r update, beta; one x update after the loop
        assert res["kernel_launches"] == 2 + 2 + 5 * its + 1
        st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 0.0, its)
        assert _rel(x.cpu().numpy(), xr) <= 1e-9, its
        assert abs(res["relres"] - rr) <= 1e-8 * rr
        assert np.all(x.cpu().numpy()[mesh.mask == 0] == 0.0)


def test_cg_ff_check_every_and_workspace_reuse():
    mesh = inputs.box_mesh(3, 3, 2, 10, perturb=0.1, seed=6)
    P = DeviceProblem(mesh, DEV)
    f = _t(inputs.random_global_field(mesh, seed=1))
    ws = torch.full((nekax.cg_workspace_bytes(mesh.nelt, 10, False) // 8 + 32,), float("nan"),
                    dtype=torch.float64, device=DEV)
    x1 = torch.empty_like(f)
    x2 = torch.empty_like(f)
    r1 = P.cg(f, x1, tol=1e-9, max_iter=1000, check_every=1, ax_impl=nekax.AX_FF, workspace=ws)
    r2 = P.cg(f, x2, tol=1e-9, max_iter=1000, check_every=7, ax_impl=nekax.AX_FF, workspace=ws)
    assert r1["status"] == r2["status"] == nekax.OK
    assert r1["iters"] == r2["iters"]
    assert torch.equal(x1, x2)


def test_cg_ff_fused_update_breakdown_and_no_work():
    """nx = 10 (the operator applies the x / direction update): a NaN in f is a breakdown; b = 0
    returns x = 0 at once; a solve that runs past convergence with check_every > 1 leaves x exactly as
    the solve that stops at once (the pending x update is applied once, the direction is frozen)."""
    mesh = inputs.box_mesh(2, 2, 3, 10, perturb=0.1, seed=8)
    P = DeviceProblem(mesh, DEV)
    f = _t(inputs.random_global_field(mesh, seed=3))
    x = torch.empty_like(f)
    fn = f.clone()
    fn[0, 5 + 10 * 5 + 100 * 5] = float("nan")  # an interior node of element 0
    r = P.cg(fn, x, tol=1e-8, max_iter=50, ax_impl=nekax.AX_FF)
    assert r["status"] == nekax.ERR_BREAKDOWN and r["iters"] <= 1
    r = P.cg(torch.zeros_like(f), x, tol=1e-8, max_iter=50, ax_impl=nekax.AX_FF)
    assert r["status"] == nekax.OK and r["iters"] == 0 and torch.count_nonzero(x) == 0
    x1 = torch.empty_like(f)
    x2 = torch.empty_like(f)
    r1 = P.cg(f, x1, tol=1e-6, max_iter=500, check_every=1, ax_impl=nekax.AX_FF)
    r2 = P.cg(f, x2, tol=1e-6, max_iter=500, check_every=50, ax_impl=nekax.AX_FF)  # overshoots by up to 49
    assert r1["status"] == r2["status"] == nekax.OK and r1["iters"] == r2["iters"]
    assert torch.equal(x1, x2)
    Pr = ref.Problem(mesh)
    assert Pr.residual(f.cpu().numpy(), x1.cpu().numpy()) <= 1e-6 * (1 + 1e-3)


@pytest.mark.parametrize("nx", [7, 8, 10, 12])
def test_cg_ff_solve_bit_identical_across_elements_per_cta(nx):
    """The solve's operator form (element energies, fused x / direction update) at every element count
    per CTA that fits: the iterate after 15 iterations is bit-identical (energies are summed in an order
    fixed by nx, the update is pointwise) and matches the oracle's PCG."""
    mesh = inputs.box_mesh(3, 2, 2, nx, perturb=0.1, seed=20 + nx)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=7)
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 0.0, 15)
    lib = nekax.load()
    outs = []
    try:
        for epb in (1, 2, 4):
            if lib.nek_set_ax_epb(int(nekax.AX_FF_ENERGY), nx, epb) != nekax.OK:
                continue
            x = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
            res = P.cg(_t(f), x, tol=0.0, max_iter=15, ax_impl=nekax.AX_FF)
            assert res["status"] == nekax.OK and res["iters"] == 15
            outs.append(x.cpu().numpy())
    finally:
        lib.nek_set_ax_epb(int(nekax.AX_FF_ENERGY), nx, 0)
    assert len(outs) >= 2
    for xo in outs[1:]:
        assert np.array_equal(xo, outs[0])
    assert _rel(outs[0], xr) <= 1e-9


def test_cg_bench_size_fixed_iterations_match_oracle():
    """The solve the benchmark times, at its size: the 32x32x32 box at nx = 10 with the benchmark's
    seeds, the float-float operator in its solve form (element energies, fused x / direction update,
    one element per CTA, the tuned count), the tensor-core operator in its solve form and the native
    FP64 operator, three fixed iterations each.
    Every element of the iterate is compared with the oracle's PCG; this covers the fused update's
    load and store offsets over all 32.8 M points."""
    nx = 10
    mesh = inputs.box_mesh(32, 32, 32, nx, perturb=0.1, seed=1)
    f = inputs.random_global_field(mesh, seed=2)
    its = 3
    P = DeviceProblem(mesh, DEV)
    lib = nekax.load()
    got = {}
    try:
        assert lib.nek_set_ax_epb(int(nekax.AX_FF_ENERGY), nx, 1) == nekax.OK
        for impl in (nekax.AX_FF, nekax.AX_OZ, nekax.AX_FP64):
            x = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
            res = P.cg(_t(f), x, tol=0.0, max_iter=its, ax_impl=impl)
            assert res["status"] == nekax.OK and res["iters"] == its, res
            got[impl] = (x.cpu().numpy(), res["relres"])
            del x
    finally:
        lib.nek_set_ax_epb(int(nekax.AX_FF_ENERGY), nx, 0)
    del P
    torch.cuda.empty_cache()
    Pr = ref.Problem(mesh)
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 0.0, its)
    assert st == ref.OK and itr == its
    for impl, (xg, relres) in got.items():
        assert np.all(np.isfinite(xg)), impl
        err = np.max(np.abs(xg - xr), axis=1)  # element by element
        worst = int(np.argmax(err))
        assert np.max(err) <= 1e-9 * np.max(np.abs(xr)), (impl, worst, float(err[worst]))
        assert abs(relres - rr) <= 1e-8 * rr, (impl, relres, rr)
        assert np.all(xg[mesh.mask == 0] == 0.0)


def test_cg_host_buffers_same_as_device_solve():
    """nek_cg_solve_host (f and x in host memory, copied by the library) gives the device solve's x bit
    for bit, with pinned and pageable host buffers, staging allocated inside or passed in."""
    nx = 10
    mesh = inputs.box_mesh(3, 2, 3, nx, perturb=0.1, seed=4)
    P = DeviceProblem(mesh, DEV)
    f = inputs.random_global_field(mesh, seed=6)
    xd = torch.empty((mesh.nelt, nx ** 3), dtype=torch.float64, device=DEV)
    rd = P.cg(_t(f), xd, tol=1e-9, max_iter=500, ax_impl=nekax.AX_FF)
    staging = torch.empty(nekax.cg_host_staging_bytes(mesh.nelt, nx) // 8 + 32, dtype=torch.float64, device=DEV)
    for pinned, stg in ((True, None), (False, staging)):
        fh = torch.from_numpy(f.copy())
        xh = torch.full_like(fh, float("nan"))
        if pinned:
            fh, xh = fh.pin_memory(), xh.pin_memory()
        rh = P.cg_host(fh, xh, tol=1e-9, max_iter=500, ax_impl=nekax.AX_FF, staging=stg)
        assert rh["status"] == rd["status"] == nekax.OK and rh["iters"] == rd["iters"]
        assert torch.equal(xh, xd.cpu())
    # NOT_CONVERGED still copies the last iterate back
    xh = torch.full_like(torch.from_numpy(f.copy()), float("nan")).pin_memory()
    xd5 = torch.empty_like(xd)
    r5 = P.cg(_t(f), xd5, tol=1e-12, max_iter=5, ax_impl=nekax.AX_FF)
    rh5 = P.cg_host(torch.from_numpy(f.copy()).pin_memory(), xh, tol=1e-12, max_iter=5, ax_impl=nekax.AX_FF)
    assert r5["status"] == rh5["status"] == nekax.ERR_NOT_CONVERGED and rh5["iters"] == 5
    assert torch.equal(xh, xd5.cpu())
    L = nekax.load()
    A = 0x10000
    args = [P.gs.handle, mesh.nelt, nx, A, A, A, A, A, A, 0.0, 1, None, None, None, None, None, None]
    for pos, bad in ((9, -1.0), (7, None), (8, None), (12, A + 16), (1, mesh.nelt + 1)):
        a = list(args)
        a[pos] = bad
        assert L.nek_cg_solve_host(*a) == nekax.ERR_INVALID_ARG, pos


# ------------------------------------------------------------------ elements-per-CTA variants
@pytest.mark.parametrize("impl", [nekax.AX_FP64, nekax.AX_FF])
@pytest.mark.parametrize("nx", [5, 8, 10])
def test_epb_variants_bit_identical_and_tuner(impl, nx):
    mesh = inputs.box_mesh(5, 3, 3, nx, perturb=0.1, seed=nx)
    P = DeviceProblem(mesh, DEV, build_minv=False)
    Gx = P.prepare_ff() if impl == nekax.AX_FF else P.G
    u = _t(inputs.random_local_field(mesh.nelt, nx, seed=3))
    outs = []
    try:
        for epb in (1, 2, 4):
            if nekax.load().nek_set_ax_epb(int(impl), nx, epb) != nekax.OK:
                continue  # this element count does not fit the kernel at this nx
            w = torch.full_like(u, float("nan"))
            (P.ax_ff if impl == nekax.AX_FF else P.ax)(u, w)
            outs.append(w)
        torch.cuda.synchronize()
        assert len(outs) >= 2
        for w in outs[1:]:
            assert torch.equal(w, outs[0])
        epb, ms = nekax.tune_ax(impl, mesh.nelt, nx, P.D, Gx, u, outs[0])
        assert epb in (1, 2, 4) and ms > 0 and nekax.get_ax_epb(impl, nx) == epb
    finally:
        nekax.set_ax_epb(impl, nx, 0)


# ------------------------------------------------------------------ reduced precision (FP32 / BF16 / FP16)
UNIT_IN = {nekax.PREC_F32: 2.0 ** -24, nekax.PREC_BF16: 2.0 ** -8, nekax.PREC_F16: 2.0 ** -11}


@pytest.mark.parametrize("prec,tc", [(nekax.PREC_F32, False), (nekax.PREC_BF16, False), (nekax.PREC_F16, False),
                                     (nekax.PREC_BF16, True), (nekax.PREC_F16, True)])
@pytest.mark.parametrize("nx", [2, 3, 4, 8, 10, 13, 16])
def test_ax_lowp_componentwise_bound(prec, tc, nx):
    """|w - w_ref| <= C (u_in + (2 nx + 3) u_acc) w_abs with w_abs = AX(|D|, |G|, |u|) from the oracle, C = 4."""
    mesh = inputs.box_mesh(3, 2, 2, nx, perturb=0.15, seed=nx)
    xi, rho, D = ref.gll(nx)
    G = ref.geom(mesh.corners, nx, xi, rho)
    u = inputs.random_local_field(mesh.nelt, nx, seed=7) * 10.0 ** np.linspace(-3, 3, mesh.nelt)[:, None]
    nb = nekax.load().nek_lowp_bytes_per_value(prec)
    dt = {4: torch.float32, 2: torch.float16}[nb]
    Glp = torch.empty((mesh.nelt, nx ** 3, 6), dtype=dt, device=DEV)
    gsc = torch.empty(mesh.nelt, dtype=torch.float32, device=DEV)
    nekax.geom_lowp(mesh.nelt, nx, prec, _t(G), Glp, gsc)
    ud = torch.from_numpy(u.astype(np.float32)).to(DEV)
    wd = torch.full_like(ud, float("nan"))
    (nekax.ax_lowp_tc if tc else nekax.ax_lowp)(mesh.nelt, nx, prec, _t(D), Glp, gsc, ud, wd)
    _check_lowp_bound(prec, nx, D, G, u, wd, "tensor-core %d" % tc)
    if tc and nx <= 11:
        # the tcgen05 form (nx up to 11): the same bound; results equal the mma.sync form's up to the order of
        # the FP32 additions inside a contraction
        w5 = torch.full_like(ud, float("nan"))
        nekax.ax_lowp_tc5(mesh.nelt, nx, prec, _t(D), Glp, gsc, ud, w5)
        _check_lowp_bound(prec, nx, D, G, u, w5, "tcgen05")


def _check_lowp_bound(prec, nx, D, G, u, wd, form):
    torch.cuda.synchronize()
    w = wd.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(w)), form
    u32 = u.astype(np.float32).astype(np.float64)
    w_ref = ref.ax(D, G, u32)
    w_abs = ref.ax(np.abs(D), np.abs(G), np.abs(u32))
    bound = 4.0 * (UNIT_IN[prec] + (2 * nx + 3) * 2.0 ** -24) * w_abs
    ratio = np.max(np.abs(w - w_ref) / bound)
    print("lowp bound ratio: precision %d %s nx %d: %.3f" % (prec, form, nx, ratio))
    assert ratio <= 1.0, (form, ratio)


@pytest.mark.parametrize("prec", [nekax.PREC_F32, nekax.PREC_BF16, nekax.PREC_F16])
@pytest.mark.parametrize("outer_ff", [False, True])
def test_cg_mixed_defect_correction(prec, outer_ff):
    nx = 6
    mesh = inputs.box_mesh(4, 3, 3, nx, perturb=0.1, seed=5)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=6)
    nb = nekax.load().nek_lowp_bytes_per_value(prec)
    Glp = torch.empty((mesh.nelt, nx ** 3, 6), dtype={4: torch.float32, 2: torch.float16}[nb], device=DEV)
    gsc = torch.empty(mesh.nelt, dtype=torch.float32, device=DEV)
    nekax.geom_lowp(mesh.nelt, nx, prec, P.G, Glp, gsc)
    x = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    Gff = P.prepare_ff() if outer_ff else None
    res = nekax.cg_solve_mixed(P.gs, mesh.nelt, nx, P.D, P.G, Gff, prec, Glp, gsc, P.mask, P.minv, _t(f), x,
                               tol=1e-10, inner_tol=1e-2, max_outer=40, max_inner=2000)
    assert res["status"] == nekax.OK, res
    assert res["relres"] <= 1e-10
    assert Pr.residual(f, x.cpu().numpy()) <= 1e-10 * 1.01
    assert res["outer"] >= 2 and res["inner"] > res["outer"]


@pytest.mark.parametrize("dims,nx,prec", [
    ((3, 1, 1), 3, nekax.PREC_F32),    # 81 points: the vector r update's n % 4 tail
    ((3, 1, 1), 3, nekax.PREC_F16),    # the tcgen05 form with the direction update at its smallest nx
    ((2, 2, 1), 11, nekax.PREC_F16),   # ... and at its largest
    ((2, 1, 2), 12, nekax.PREC_BF16),  # the CUDA-core form with the update for BF16 (beyond the tcgen05 form)
    ((1, 3, 1), 13, nekax.PREC_F32),   # two elements per CTA over three elements: a ragged last CTA
])
def test_cg_mixed_direction_update_forms(dims, nx, prec):
    """Defect correction to 1e-10 through each operator form that applies the inner direction update, checked
    with the oracle's residual of the returned x."""
    mesh = inputs.box_mesh(*dims, nx, perturb=0.1, seed=nx)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=nx + 1)
    nb = nekax.load().nek_lowp_bytes_per_value(prec)
    Glp = torch.empty((mesh.nelt, nx ** 3, 6), dtype={4: torch.float32, 2: torch.float16}[nb], device=DEV)
    gsc = torch.empty(mesh.nelt, dtype=torch.float32, device=DEV)
    nekax.geom_lowp(mesh.nelt, nx, prec, P.G, Glp, gsc)
    x = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    res = nekax.cg_solve_mixed(P.gs, mesh.nelt, nx, P.D, P.G, P.prepare_ff(), prec, Glp, gsc, P.mask, P.minv,
                               _t(f), x, tol=1e-10, inner_tol=1e-2, max_outer=60, max_inner=4000)
    assert res["status"] == nekax.OK, res
    assert Pr.residual(f, x.cpu().numpy()) <= 1e-10 * 1.01
    # five launches per inner iteration at most, plus a bounded count per outer step
    assert res["kernel_launches"] <= 5 * res["inner"] + 60 * res["outer"] + 10, res


@pytest.mark.parametrize("prec", [nekax.PREC_F32, nekax.PREC_BF16, nekax.PREC_F16])
def test_cg_mixed_inner_direction_update_fused(prec):
    """The inner operator (the CUDA-core form for FP32, the tcgen05 form for BF16 / FP16) applies the inner
    solve's x / direction update itself, so an inner iteration is five launches (operator, dssum, alpha,
    r update, beta) instead of six with a separate update pass: one outer step of K inner iterations (an
    unreachable inner tolerance) launches 15 + 5K kernels (it would be 14 + 6K)."""
    nx, K = 6, 7
    mesh = inputs.box_mesh(3, 3, 2, nx, perturb=0.1, seed=8)
    P = DeviceProblem(mesh, DEV)
    f = inputs.random_global_field(mesh, seed=9)
    nb = nekax.load().nek_lowp_bytes_per_value(prec)
    Glp = torch.empty((mesh.nelt, nx ** 3, 6), dtype={4: torch.float32, 2: torch.float16}[nb], device=DEV)
    gsc = torch.empty(mesh.nelt, dtype=torch.float32, device=DEV)
    nekax.geom_lowp(mesh.nelt, nx, prec, P.G, Glp, gsc)
    x = torch.full((mesh.nelt, nx ** 3), float("nan"), dtype=torch.float64, device=DEV)
    res = nekax.cg_solve_mixed(P.gs, mesh.nelt, nx, P.D, P.G, P.prepare_ff(), prec, Glp, gsc, P.mask, P.minv,
                               _t(f), x, tol=1e-30, inner_tol=1e-30, max_outer=1, max_inner=K)
    assert res["status"] == nekax.ERR_NOT_CONVERGED and res["outer"] == 1 and res["inner"] == K, res
    assert res["kernel_launches"] == 15 + 5 * K, res
    # the outer step's x: finite, zero on masked nodes, its residual the one the oracle computes, and close
    # to that of K exact Jacobi-PCG iterations (0.119 on this mesh)
    xs = x.cpu().numpy()
    assert np.all(np.isfinite(xs))
    assert np.all(xs.reshape(-1)[mesh.mask.reshape(-1) == 0] == 0.0)
    Pr = ref.Problem(mesh)
    rel = Pr.residual(f, xs)
    assert abs(res["relres"] - rel) <= 1e-9 * rel, (res, rel)
    _, xk, _, _ = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, tol=0.0, max_iter=K)
    assert 0.0 < rel < 2.0 * Pr.residual(f, xk), (rel, Pr.residual(f, xk))


# ------------------------------------------------------------------ batched solves
def _batch_case(seed=0):
    specs = [dict(ex=2, ey=2, ez=2, nx=8), dict(ex=3, ey=2, ez=1, nx=6), dict(ex=2, ey=1, ez=1, nx=10),
             dict(ex=4, ey=2, ez=2, nx=6), dict(ex=1, ey=1, ez=1, nx=3), dict(ex=2, ey=2, ez=1, nx=8)]
    meshes = [inputs.box_mesh(sp["ex"], sp["ey"], sp["ez"], sp["nx"], perturb=0.1, seed=seed + q)
              for q, sp in enumerate(specs)]
    fields = [inputs.random_global_field(m, seed=seed + 50 + q) for q, m in enumerate(meshes)]
    return meshes, fields


@pytest.mark.parametrize("ff", [False, True])
def test_batch_matches_oracle_per_problem(ff):
    from paper_2011_04981_gb300.problem import DeviceBatch

    meshes, fields = _batch_case()
    B = DeviceBatch(meshes, fields, DEV, ff=ff)
    x = torch.full((B.npts,), float("nan"), dtype=torch.float64, device=DEV)
    res = B.solve(x, tol=1e-9, max_iter=3000, iters_per_graph=7)
    assert res["status"] == nekax.OK and res["converged"] == len(meshes), res
    assert res["graph_launches"] > 0
    xs = B.split(x.cpu().numpy())
    iters = [None] * len(meshes)
    for pos, q in enumerate(B.order):
        iters[q] = int(res["iters"][pos])
    for q, m in enumerate(meshes):
        Pr = ref.Problem(m)
        st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, m.mask, Pr.minv, fields[q], 1e-9, 3000)
        assert abs(iters[q] - itr) <= 2, (q, iters[q], itr)
        assert Pr.residual(fields[q], xs[q].reshape(m.nelt, -1)) <= 1e-9 * 1.001


def test_batch_graph_replay_is_bit_identical_to_eager():
    from paper_2011_04981_gb300.problem import DeviceBatch

    meshes, fields = _batch_case(seed=10)
    fields[2] = np.zeros_like(fields[2])  # a problem with b = 0 stops at once
    B = DeviceBatch(meshes, fields, DEV, ff=True)
    x1 = torch.empty((B.npts,), dtype=torch.float64, device=DEV)
    x2 = torch.empty_like(x1)
    r1 = B.solve(x1, tol=1e-9, max_iter=3000, iters_per_graph=0)
    r2 = B.solve(x2, tol=1e-9, max_iter=3000, iters_per_graph=5)
    assert r1["graph_launches"] == 0 and r2["graph_launches"] > 0
    assert np.array_equal(r1["iters"], r2["iters"])
    assert torch.equal(x1, x2)
    # the whole solve as one graph launch (device-side WHILE loop): the same iterates and counts
    x3 = torch.full_like(x1, float("nan"))
    r3 = B.solve(x3, tol=1e-9, max_iter=3000, iters_per_graph=-1)
    assert r3["graph_launches"] == 1 and r3["iterations_run"] == r1["iterations_run"], (r3, r1)
    assert np.array_equal(r1["iters"], r3["iters"])
    assert torch.equal(x1, x3)
    zero_pos = B.order.index(2)
    assert r1["iters"][zero_pos] == 0
    assert float(B.split(x1)[2].abs().max()) == 0.0
    # an iteration budget that ends the device loop before convergence
    r4 = B.solve(x3, tol=1e-9, max_iter=12, iters_per_graph=-1)
    assert r4["status"] == nekax.ERR_NOT_CONVERGED and r4["iterations_run"] == 12


def test_batch_one_launch_native_fp64_operator():
    """The one-launch batched solve with the native FP64 operator (its <p,w> pass instead of element
    energies): the same iterates as eager launches, and per-problem parity with the oracle."""
    from paper_2011_04981_gb300.problem import DeviceBatch

    meshes, fields = _batch_case(seed=20)
    B = DeviceBatch(meshes, fields, DEV, ff=False)
    x1 = torch.empty((B.npts,), dtype=torch.float64, device=DEV)
    x2 = torch.full_like(x1, float("nan"))
    r1 = B.solve(x1, tol=1e-9, max_iter=3000, iters_per_graph=0)
    r2 = B.solve(x2, tol=1e-9, max_iter=3000, iters_per_graph=-1)
    assert r1["status"] == r2["status"] == nekax.OK and r2["graph_launches"] == 1
    assert np.array_equal(r1["iters"], r2["iters"]) and torch.equal(x1, x2)
    xs = B.split(x2.cpu().numpy())
    for q, m in enumerate(meshes):
        Pr = ref.Problem(m)
        assert Pr.residual(fields[q], xs[q].reshape(m.nelt, -1)) <= 1e-9 * 1.001
