"""GPU parity of the learned-preconditioner kernels against the FP64 network oracle.

Weights are drawn and rounded to BF16 first (the kernels stage BF16 weights), so
the only difference left is FP32 accumulation, FP32 erf in GELU and, in the
tensor-core form, the BF16 rounding of the input and the hidden activations.
Every output and every gradient entry is compared with its own error bound from
the oracle (oracle/net.py: forward_bound, loss_and_grad_bound,
energy_loss_and_grad_bound): it must lie inside the rigorous worst-case bound
and inside LAMBDA times the root-sum-square error scale, which is orders of
magnitude tighter; the largest observed ratio to that scale is printed.
Flexible CG is checked by the oracle's residual of its result.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import net as onet  # noqa: E402
from oracle import ref  # noqa: E402
from paper_2011_04981_gb300 import inputs, nekax  # noqa: E402
from paper_2011_04981_gb300.problem import DeviceProblem  # noqa: E402

DEV = "cuda"


def _bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _theta(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    th = rng.normal(scale=scale, size=onet.NPARAM)
    return _bf16(th).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


LAMBDA = 8.0          # safety factor on the rms error scale
U_TC = 2.0 ** -23     # FP32 sums on the tensor cores: at most one ulp per addition
U_BF16 = 2.0 ** -9    # BF16 rounding of the tensor-core form's input and activations


def _check_elementwise(name, got, ref_val, worst, rms):
    """|got - ref| inside the rigorous bound and inside LAMBDA * rms, entry by entry."""
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref_val)
    assert np.all(np.isfinite(got)), name
    bad_w = np.flatnonzero(err > worst)
    assert bad_w.size == 0, (name, "worst-case bound", bad_w[:5], float(np.max(err / worst)))
    ratio = err / np.maximum(rms, 1e-300)
    bad = np.flatnonzero(ratio > LAMBDA)
    assert bad.size == 0, (name, "rms scale", bad[:5], float(np.max(ratio)))
    print("%s: max |err| / rms scale = %.3g (limit %g), max |err| / worst bound = %.3g"
          % (name, float(np.max(ratio)), LAMBDA, float(np.max(err / worst))))
    return float(np.max(ratio))


def test_param_count():
    assert nekax.net_param_count() == onet.NPARAM == 8241


def test_forward_matches_oracle():
    B = 5
    rng = np.random.default_rng(1)
    th = _theta(2)
    x = rng.normal(size=(B, 2, 8, 8, 8))
    ws = torch.empty(nekax.net_train_workspace_bytes(B) // 4 + 64, dtype=torch.float32, device=DEV)
    y = torch.empty((B, 512), dtype=torch.float32, device=DEV)
    nekax.net_forward_batch(B, torch.from_numpy(th.astype(np.float32)).to(DEV),
                            torch.from_numpy(x.astype(np.float32)).to(DEV), y, ws)
    torch.cuda.synchronize()
    x64 = x.astype(np.float32).astype(np.float64)
    yr, _, worst = onet.forward_bound(th, x64, mode="worst")
    _, _, rms = onet.forward_bound(th, x64, mode="rms")
    _check_elementwise("forward", y.cpu().numpy().reshape(B, 512), yr[:, 0].reshape(B, 512),
                       worst[5][:, 0].reshape(B, 512), rms[5][:, 0].reshape(B, 512))


def test_gradient_matches_oracle():
    B = 4
    rng = np.random.default_rng(3)
    th = _theta(4)
    x = rng.normal(size=(B, 2, 8, 8, 8)).astype(np.float32).astype(np.float64)
    t = rng.normal(size=(B, 8, 8, 8)).astype(np.float32).astype(np.float64)
    ws = torch.empty(nekax.net_train_workspace_bytes(B) // 4 + 64, dtype=torch.float32, device=DEV)
    g = torch.empty(onet.NPARAM, dtype=torch.float32, device=DEV)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    nekax.net_train_grad(B, torch.from_numpy(th.astype(np.float32)).to(DEV),
                         torch.from_numpy(x.astype(np.float32)).to(DEV),
                         torch.from_numpy(t.reshape(B, 512).astype(np.float32)).to(DEV), g, loss, ws)
    torch.cuda.synchronize()
    L, gr, worst = onet.loss_and_grad_bound(th, x, t, mode="worst")
    _, _, rms = onet.loss_and_grad_bound(th, x, t, mode="rms")
    assert abs(float(loss.item()) - L) <= 1e-4 * L
    gg = g.cpu().numpy().astype(np.float64)
    o = 0
    for name, shp in onet.SHAPES:
        n = int(np.prod(shp))
        _check_elementwise("grad " + name, gg[o:o + n], gr[o:o + n], worst[o:o + n], rms[o:o + n])
        o += n


def test_prep_and_apply_match_oracle():
    mesh = inputs.box_mesh(3, 2, 2, 8, perturb=0.15, seed=2)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    th = _theta(7)
    r = inputs.random_local_field(mesh.nelt, 8, seed=9) * mesh.mask
    rd = torch.from_numpy(r).to(DEV)
    xin = torch.empty((mesh.nelt, 2, 512), dtype=torch.float32, device=DEV)
    sc = torch.empty(mesh.nelt, dtype=torch.float32, device=DEV)
    nekax.net_prep(mesh.nelt, 8, rd, P.minv, xin, sc)
    c = torch.empty_like(rd)
    P.gs.inv_multiplicity(c)
    z = torch.empty_like(rd)
    nekax.net_apply(mesh.nelt, 8, torch.from_numpy(th.astype(np.float32)).to(DEV), xin, sc, c, z)
    torch.cuda.synchronize()
    x_ref, sr, sj = onet.element_inputs(r, Pr.minv * r)
    xg = xin.cpu().numpy().reshape(mesh.nelt, 2, 512).astype(np.float64)
    # FP64 norms, one FP32 rounding of each normalised value (plus the RMS's own rounding)
    assert np.all(np.abs(xg - x_ref) <= 4 * 2.0 ** -24 * np.abs(x_ref)), float(np.max(np.abs(xg - x_ref)))
    assert np.all(np.abs(sc.cpu().numpy() - sj) <= 2 * 2.0 ** -24 * sj)
    # the network on the kernel's own (FP32) input, then z = y * scale * c
    xh = xg.reshape(mesh.nelt, 2, 8, 8, 8)
    y, _, worst = onet.forward_bound(th, xh, mode="worst")
    _, _, rms = onet.forward_bound(th, xh, mode="rms")
    s = sc.cpu().numpy().astype(np.float64)[:, None] * Pr.c
    yf = y[:, 0].reshape(mesh.nelt, 512)
    extra = 3 * 2.0 ** -24 * np.abs(yf * s)  # the two products of the output scaling
    _check_elementwise("apply", z.cpu().numpy(), yf * s, worst[5][:, 0].reshape(mesh.nelt, 512) * np.abs(s) + extra,
                       np.sqrt((rms[5][:, 0].reshape(mesh.nelt, 512) * s) ** 2 + extra ** 2))


def test_apply_bf16_tensor_cores_match_oracle():
    """The tensor-core inference rounds the input and both hidden activations to
    BF16: against the oracle with the same rounding it agrees to FP32-sum level
    (plus rare rounding ties decided differently), and against the unrounded
    network within the BF16 bound."""
    mesh = inputs.box_mesh(5, 3, 2, 8, perturb=0.15, seed=4)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    th = _theta(12)
    r = inputs.random_local_field(mesh.nelt, 8, seed=3) * mesh.mask
    rd = torch.from_numpy(r).to(DEV)
    xin = torch.empty((mesh.nelt, 2, 512), dtype=torch.float32, device=DEV)
    sc = torch.empty(mesh.nelt, dtype=torch.float32, device=DEV)
    nekax.net_prep(mesh.nelt, 8, rd, P.minv, xin, sc)
    c = torch.empty_like(rd)
    P.gs.inv_multiplicity(c)
    thd = torch.from_numpy(th.astype(np.float32)).to(DEV)
    z = torch.full_like(rd, float("nan"))
    nekax.net_apply_bf16(mesh.nelt, 8, thd, xin, sc, c, z)
    zm = torch.full_like(rd, float("nan"))
    nekax.net_apply_bf16_mma(mesh.nelt, 8, thd, xin, sc, c, zm)
    z32 = torch.empty_like(rd)
    nekax.net_apply(mesh.nelt, 8, thd, xin, sc, c, z32)
    torch.cuda.synchronize()
    xh = xin.cpu().numpy().astype(np.float64).reshape(mesh.nelt, 2, 8, 8, 8)
    s = sc.cpu().numpy().astype(np.float64)[:, None] * Pr.c
    n = mesh.nelt
    yb = onet.forward(th, xh, act_round=onet.bf16_round)[:, 0].reshape(n, 512) * s
    zz = z.cpu().numpy()
    assert np.all(np.isfinite(zz))
    assert _rel(zz, yb) <= 5e-4  # against the same rounding points: FP32-sum level (norm-wise, extra)
    # element by element against the unrounded network, with the BF16 roundings in the bound
    assert _rel(zm.cpu().numpy(), yb) <= 5e-4
    for label, got, u_act, u in (("apply_bf16 (tcgen05)", zz, U_BF16, U_TC),
                                 ("apply_bf16_mma (mma.sync)", zm.cpu().numpy(), U_BF16, U_TC),
                                 ("apply (FP32)", z32.cpu().numpy(), 0.0, 2.0 ** -24)):
        y, _, worst = onet.forward_bound(th, xh, u_act=u_act, u=u, mode="worst")
        _, _, rms = onet.forward_bound(th, xh, u_act=u_act, u=u, mode="rms")
        yf = y[:, 0].reshape(n, 512)
        extra = 3 * 2.0 ** -24 * np.abs(yf * s)
        _check_elementwise(label, got, yf * s, worst[5][:, 0].reshape(n, 512) * np.abs(s) + extra,
                           np.sqrt((rms[5][:, 0].reshape(n, 512) * s) ** 2 + extra ** 2))


def test_apply_bf16_many_elements_every_element_checked():
    """More elements than the tcgen05 kernel's persistent grid (3 CTAs per SM), so every CTA runs several
    elements through the same shared-memory grid and tensor memory; every output of every element against
    the oracle's bound, and the two tensor-core forms against each other."""
    n = 1000
    rng = np.random.default_rng(31)
    th = _theta(32)
    thd = torch.from_numpy(th.astype(np.float32)).to(DEV)
    x = rng.normal(size=(n, 2, 512)).astype(np.float32)
    sc = rng.uniform(0.5, 2.0, size=n).astype(np.float32)
    cc = np.where(rng.uniform(size=(n, 512)) < 0.3, 0.5, 1.0)
    xd, scd, cd = (torch.from_numpy(a).to(DEV) for a in (x, sc, cc))
    z = torch.full((n, 512), float("nan"), dtype=torch.float64, device=DEV)
    zm = torch.full_like(z, float("nan"))
    nekax.net_apply_bf16(n, 8, thd, xd, scd, cd, z)
    nekax.net_apply_bf16_mma(n, 8, thd, xd, scd, cd, zm)
    torch.cuda.synchronize()
    s = sc.astype(np.float64)[:, None] * cc
    xh = x.astype(np.float64).reshape(n, 2, 8, 8, 8)
    y, _, worst = onet.forward_bound(th, xh, u_act=U_BF16, u=U_TC, mode="worst")
    _, _, rms = onet.forward_bound(th, xh, u_act=U_BF16, u=U_TC, mode="rms")
    yf = y[:, 0].reshape(n, 512)
    extra = 3 * 2.0 ** -24 * np.abs(yf * s)
    w = worst[5][:, 0].reshape(n, 512) * np.abs(s) + extra
    r = np.sqrt((rms[5][:, 0].reshape(n, 512) * s) ** 2 + extra ** 2)
    _check_elementwise("apply_bf16 (tcgen05), 1000 elements", z.cpu().numpy(), yf * s, w, r)
    _check_elementwise("apply_bf16_mma, 1000 elements", zm.cpu().numpy(), yf * s, w, r)


def test_tcgen05_kernel_bounded_wait_runs_out_and_reports():
    """The tcgen05 inference kernel's mbarrier waits are bounded: with the barrier expecting one arrival
    more than the MMAs give (a phase that never completes), every wait runs out after the given bound,
    the kernel flags it, poisons its output with NaN, frees its tensor memory and returns; the context
    stays usable, and the same kernel then runs normally."""
    import ctypes

    lib = nekax.load()
    flag = ctypes.c_int(-1)
    assert lib.nek_net_tc_selftest(1, 20000, ctypes.byref(flag)) == nekax.ERR_TIMEOUT
    assert flag.value == 1
    flag.value = -1
    assert lib.nek_net_tc_selftest(0, 2000000, ctypes.byref(flag)) == nekax.OK
    assert flag.value == 0
    assert lib.nek_net_tc_selftest(1, 0, ctypes.byref(flag)) == nekax.ERR_INVALID_ARG
    # and the library's inference still works afterwards (a small parity check)
    test_apply_bf16_tensor_cores_match_oracle()


def test_adam_matches_oracle():
    rng = np.random.default_rng(5)
    n = 1000
    th = rng.normal(size=n).astype(np.float32)
    m = np.zeros(n, dtype=np.float32)
    v = np.zeros(n, dtype=np.float32)
    thd, md, vd = (torch.from_numpy(a.copy()).to(DEV) for a in (th, m, v))
    th64, m64, v64 = th.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 4):
        g = rng.normal(size=n).astype(np.float32)
        nekax.adam_step(n, thd, torch.from_numpy(g).to(DEV), md, vd, 1e-2, step)
        th64, m64, v64 = onet.adam(th64, g.astype(np.float64), m64, v64, step, lr=1e-2)
    torch.cuda.synchronize()
    assert np.max(np.abs(thd.cpu().numpy() - th64)) <= 1e-6


@pytest.mark.parametrize("m", [1, 3, 8])
def test_fcg_truncated_jacobi_mode_matches_pcg(m):
    """FCG(m) with the Jacobi preconditioner: for a fixed SPD preconditioner every window length gives the
    PCG iterates in exact arithmetic, so the iteration count matches the oracle's PCG within 3 and the
    oracle's residual of the result meets the tolerance."""
    mesh = inputs.box_mesh(4, 3, 3, 8, perturb=0.15, seed=4)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=5)
    fd = torch.from_numpy(f).to(DEV)
    x = torch.full_like(fd, float("nan"))
    r = nekax.fcg_solve(P.gs, mesh.nelt, 8, P.D, P.G, P.prepare_ff(), P.mask, P.minv, None, fd, x, tol=1e-8,
                        truncation=m)
    assert r["status"] == nekax.OK and r["net_applications"] == 0
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 1e-8, 5000)
    assert abs(r["iters"] - itr) <= 3, (m, r["iters"], itr)
    assert Pr.residual(f, x.cpu().numpy()) <= 1e-8 * 1.001
    L = nekax.load()
    for bad in (0, 17):
        assert L.nek_fcg_solve_trunc(P.gs.handle, mesh.nelt, 8, P.D.data_ptr(), P.G.data_ptr(), None,
                                     P.mask.data_ptr(), None, None, fd.data_ptr(), x.data_ptr(), 1e-8, 10, bad, 100,
                                     0.5, None, None, None) == nekax.ERR_INVALID_ARG
    assert L.nek_fcg_trunc_workspace_bytes(mesh.nelt, 8, 0, 8) > L.nek_fcg_trunc_workspace_bytes(mesh.nelt, 8, 0, 1)


def test_fcg_truncated_with_network_falls_back_and_converges():
    """FCG(8) with a network that is no preconditioner (random small weights) and a short stagnation
    window: it hands over to Jacobi, empties its direction window, and still reaches the tolerance
    (checked by the oracle's residual)."""
    mesh = inputs.box_mesh(4, 3, 3, 8, perturb=0.15, seed=13)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=14)
    fd = torch.from_numpy(f).to(DEV)
    x = torch.full_like(fd, float("nan"))
    th = torch.from_numpy(_theta(15, scale=0.05).astype(np.float32)).to(DEV)
    r = nekax.fcg_solve(P.gs, mesh.nelt, 8, P.D, P.G, P.prepare_ff(), P.mask, P.minv, th, fd, x, tol=1e-8,
                        max_iter=20000, stag_window=20, stag_factor=0.01, truncation=8)
    assert r["status"] == nekax.OK, r
    assert r["fell_back_at"] > 0 and r["net_applications"] == r["fell_back_at"], r
    assert Pr.residual(f, x.cpu().numpy()) <= 1e-8 * 1.001


def test_residual_and_net_target_match_oracle():
    mesh = inputs.box_mesh(3, 2, 2, 8, perturb=0.15, seed=9)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=1)
    xv = inputs.random_global_field(mesh, seed=2)
    r = torch.full((mesh.nelt, 512), float("nan"), dtype=torch.float64, device=DEV)
    for Gff in (None, P.prepare_ff()):
        nekax.residual(P.gs, mesh.nelt, 8, P.D, P.G, Gff, P.mask, torch.from_numpy(f).to(DEV),
                       torch.from_numpy(xv).to(DEV), r)
        torch.cuda.synchronize()
        r_ref = ref.mask_apply(mesh.mask, f) - Pr.apply(xv)
        assert np.max(np.abs(r.cpu().numpy() - r_ref)) <= 1e-12 * np.max(np.abs(Pr.apply(np.abs(xv))) + np.abs(f))
    # target = (xs - xk) / scale per element, one FP32 rounding
    xs = torch.from_numpy(f).to(DEV)
    xk = torch.from_numpy(xv).to(DEV)
    sc = torch.from_numpy(np.linspace(0.0, 2.0, mesh.nelt).astype(np.float32)).to(DEV)  # element 0: scale 0
    t = torch.full((mesh.nelt, 512), float("nan"), dtype=torch.float32, device=DEV)
    nekax.net_target(mesh.nelt, 8, xs, xk, sc, t)
    torch.cuda.synchronize()
    s = sc.cpu().numpy().astype(np.float64)
    expect = np.where(s[:, None] > 0, (f - xv) / np.where(s > 0, s, 1.0)[:, None], 0.0).astype(np.float32)
    assert np.array_equal(t.cpu().numpy(), expect)


def test_fcg_jacobi_mode_and_random_net():
    mesh = inputs.box_mesh(4, 3, 3, 8, perturb=0.15, seed=4)
    P = DeviceProblem(mesh, DEV)
    Pr = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=5)
    fd = torch.from_numpy(f).to(DEV)
    x = torch.empty_like(fd)
    r0 = nekax.fcg_solve(P.gs, mesh.nelt, 8, P.D, P.G, None, P.mask, P.minv, None, fd, x, tol=1e-8)
    assert r0["status"] == nekax.OK and r0["net_applications"] == 0
    st, xr, itr, rr = ref.pcg(Pr.D, Pr.G, Pr.offsets, Pr.idx, mesh.mask, Pr.minv, f, 1e-8, 5000)
    assert abs(r0["iters"] - itr) <= 3, (r0["iters"], itr)
    assert Pr.residual(f, x.cpu().numpy()) <= 1e-8 * 1.001
    # an untrained network: flexible CG still converges (with Jacobi taking over on stagnation)
    th = torch.from_numpy(_theta(11, scale=0.05).astype(np.float32)).to(DEV)
    x2 = torch.empty_like(fd)
    r1 = nekax.fcg_solve(P.gs, mesh.nelt, 8, P.D, P.G, P.prepare_ff(), P.mask, P.minv, th, fd, x2, tol=1e-8,
                         max_iter=20000, stag_window=30, stag_factor=0.5)
    assert r1["status"] == nekax.OK, r1
    assert r1["net_applications"] >= 1
    assert Pr.residual(f, x2.cpu().numpy()) <= 1e-8 * 1.001


def test_energy_gradient_matches_oracle():
    B = 3
    mesh = inputs.box_mesh(3, 1, 1, 8, perturb=0.2, seed=6)
    P = DeviceProblem(mesh, DEV, build_minv=False)
    Glp = torch.empty((mesh.nelt, 512, 6), dtype=torch.float32, device=DEV)
    gsc = torch.empty(mesh.nelt, dtype=torch.float32, device=DEV)
    nekax.geom_lowp(mesh.nelt, 8, nekax.PREC_F32, P.G, Glp, gsc)
    rng = np.random.default_rng(8)
    th = _theta(12)
    x = rng.normal(size=(B, 2, 8, 8, 8)).astype(np.float32).astype(np.float64)
    t = rng.normal(size=(B, 8, 8, 8)).astype(np.float32).astype(np.float64)
    ws = torch.empty(nekax.net_train_workspace_bytes(B) // 4 + 64, dtype=torch.float32, device=DEV)
    g = torch.empty(onet.NPARAM, dtype=torch.float32, device=DEV)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    nekax.net_train_grad_energy(B, torch.from_numpy(th.astype(np.float32)).to(DEV),
                                torch.from_numpy(x.astype(np.float32)).to(DEV),
                                torch.from_numpy(t.reshape(B, 512).astype(np.float32)).to(DEV), P.D, Glp, gsc, g,
                                loss, ws)
    torch.cuda.synchronize()
    D32 = P.D_host.astype(np.float32).astype(np.float64)
    G = Glp.cpu().numpy().astype(np.float64) * gsc.cpu().numpy().astype(np.float64)[:, None, None]
    A = np.stack([ref.element_matrix(D32, G[e]) for e in range(B)])
    Aabs = np.stack([ref.element_matrix(np.abs(D32), np.abs(G[e])) for e in range(B)])
    L, gr, worst = onet.energy_loss_and_grad_bound(th, x, t, A, Aabs, 8, mode="worst")
    _, _, rms = onet.energy_loss_and_grad_bound(th, x, t, A, Aabs, 8, mode="rms")
    assert abs(float(loss.item()) - L) <= 1e-4 * L
    gg = g.cpu().numpy().astype(np.float64)
    o = 0
    for name, shp in onet.SHAPES:
        n = int(np.prod(shp))
        if name != "b3":  # constants are in the kernel of A: d loss / d b3 is zero up to rounding
            _check_elementwise("energy grad " + name, gg[o:o + n], gr[o:o + n], worst[o:o + n], rms[o:o + n])
        o += n


def test_trained_network_beats_untrained_and_jacobi():
    """The learned-preconditioner experiment at reduced size: pairs from the FP64 solver on 30 meshes of
    the family (8^3 elements), GPU training with the library's kernels, then truncated flexible CG
    (FCG(8)) on a held-out 12^3 mesh of the family.  The trained network must lower the validation
    loss and need fewer iterations than the same solve with the untrained network and than
    Jacobi-PCG; every solve must reach the tolerance without falling back to Jacobi."""
    from paper_2011_04981_gb300 import learned

    data = learned.make_training_data(n_meshes=30, pairs_per_mesh=100, seed=0)
    val = learned.make_training_data(n_meshes=3, pairs_per_mesh=100, seed=1)
    assert len(data) >= 2500
    theta, hist = learned.train(data, epochs=20, batch=256, lr=2e-3, seed=0)
    assert hist[-1] < hist[0]
    theta0 = learned.init_params(0, DEV)
    v_trained = learned.validation_loss(theta, val)
    v_init = learned.validation_loss(theta0, val)
    assert v_trained < v_init, (v_trained, v_init)
    mesh = learned.mesh_family(seed=5, e=12)
    out = learned.compare_on_mesh(theta, mesh, seed=2, theta_untrained=theta0)
    jac, lrn, unt = out["jacobi_pcg"], out["learned_fcg"], out["untrained_fcg"]
    print("held-out 12^3 mesh: Jacobi-PCG %d, FCG(8) trained %d (fell back at %d), untrained %d iterations"
          % (jac["iters"], lrn["iters"], lrn["fell_back_at"], unt["iters"]))
    assert jac["relres"] <= 1e-8 and lrn["relres"] <= 1e-8 and unt["relres"] <= 1e-8
    assert lrn["iters"] < unt["iters"], (lrn, unt)
    assert lrn["iters"] < jac["iters"], (lrn, jac)
    assert lrn["fell_back_at"] == 0
