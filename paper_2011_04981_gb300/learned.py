"""Training and evaluation of the learned element preconditioner.

Everything numerical runs in the library's kernels (solves, operator, network
forward/backward, Adam); this module only orchestrates the calls and moves
buffers.

Training data are (residual, error) pairs produced by the FP64 solver itself:
for each training mesh the solution x* is computed to a relative residual of
1e-13 by Jacobi-PCG, then Jacobi-PCG is rerun from zero and stopped after k
iterations for a few k; with x_k, r_k = mask(b - dssum(AX x_k)) and the error
e_k = x* - x_k, every sampled element contributes the network input
(r_k, Minv r_k normalised by their element RMS) and the target
e_k / rms(Minv r_k) (the preconditioner multiplies the network output back by
rms(Minv r_k) and by 1/multiplicity before summing over elements).  Training
minimises the per-sample relative error in the element energy norm with Adam.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, nekax
from .problem import DeviceProblem

NX = 8


def mesh_family(seed, e=8):
    """A deformed box of the learned-preconditioner family: nx = 8, vertex
    perturbation 0.15 h and a random axis stretch of up to 8:1."""
    return inputs.box_mesh(e, e, e, NX, perturb=0.15, seed=seed, stretch="random8")


def _residual(P, f, x, w):
    """w = mask(f - dssum(AX x)) on the device (nek_residual with the float-float operator)."""
    nekax.residual(P.gs, P.nelt, P.nx, P.D, P.G, P.prepare_ff(), P.mask, f, x, w)


class TrainingSet:
    """Network inputs, targets and each sample's element operator (FP32 G with its scale)."""

    def __init__(self, xin, target, Glp, gscale, D):
        self.xin, self.target, self.Glp, self.gscale, self.D = xin, target, Glp, gscale, D

    def __len__(self):
        return self.xin.shape[0]


def make_training_data(n_meshes=200, pairs_per_mesh=100, snapshots=5, e=8, seed=0, device="cuda"):
    """Returns a TrainingSet on the device: xin [N,2,512], target [N,512], Glp [N,512,6] (FP32), gscale [N]."""
    import torch

    rng = np.random.default_rng(seed)
    X, T, GL, GS = [], [], [], []
    D = None
    for m in range(n_meshes):
        mesh = mesh_family(10_000 + seed * 1000 + m, e)
        P = DeviceProblem(mesh, device)
        P.prepare_ff()
        D = P.D
        Glp = torch.empty((mesh.nelt, 512, 6), dtype=torch.float32, device=device)
        gsc = torch.empty(mesh.nelt, dtype=torch.float32, device=device)
        nekax.geom_lowp(mesh.nelt, NX, nekax.PREC_F32, P.G, Glp, gsc)
        f = torch.from_numpy(inputs.random_global_field(mesh, seed=m)).to(device)
        xs = torch.empty_like(f)
        res = P.cg(f, xs, tol=1e-13, max_iter=20000, ax_impl=nekax.AX_FF, check_every=10)
        n_it = max(2, res["iters"])
        ks = np.unique(np.sort(np.exp(rng.uniform(0.0, math.log(0.8 * n_it), size=snapshots)).astype(int) + 1))
        xk = torch.empty_like(f)
        r = torch.empty_like(f)
        xin = torch.empty((mesh.nelt, 2, 512), dtype=torch.float32, device=device)
        sc = torch.empty(mesh.nelt, dtype=torch.float32, device=device)
        tgt = torch.empty((mesh.nelt, 512), dtype=torch.float32, device=device)
        per = max(1, pairs_per_mesh // len(ks))
        for k in ks:
            P.cg(f, xk, tol=0.0, max_iter=int(k), ax_impl=nekax.AX_FF)
            _residual(P, f, xk, r)
            nekax.net_prep(mesh.nelt, NX, r, P.minv, xin, sc)
            # (xs - xk) / scale; nek_net_apply weights each element's output by 1/multiplicity
            nekax.net_target(mesh.nelt, NX, xs, xk, sc, tgt)
            good = torch.nonzero(sc > 0).flatten()
            sel = good[torch.from_numpy(rng.choice(good.numel(), size=min(per, good.numel()), replace=False)).to(
                device)]
            X.append(xin[sel].clone())
            T.append(tgt[sel].clone())
            GL.append(Glp[sel].clone())
            GS.append(gsc[sel].clone())
        del P
    return TrainingSet(torch.cat(X), torch.cat(T), torch.cat(GL), torch.cat(GS), D)


def init_params(seed=0, device="cuda"):
    """Normal initialisation scaled by 1/sqrt(fan-in) (fan-in = 27 * input channels)."""
    import torch

    rng = np.random.default_rng(seed)
    parts = []
    for cin, cout in ((2, 16), (16, 16), (16, 1)):
        parts.append(rng.normal(scale=1.0 / math.sqrt(27 * cin), size=cout * cin * 27))
        parts.append(np.zeros(cout))
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == nekax.net_param_count()
    return torch.from_numpy(th).to(device)


def _grad(data, idx, batch, theta, g, loss, ws, kind):
    xb = data.xin[idx].contiguous()
    tb = data.target[idx].contiguous()
    if kind == "energy":
        nekax.net_train_grad_energy(batch, theta, xb, tb, data.D, data.Glp[idx].contiguous(),
                                    data.gscale[idx].contiguous(), g, loss, ws)
    else:
        nekax.net_train_grad(batch, theta, xb, tb, g, loss, ws)


def train(data, epochs=20, batch=256, lr=2e-3, seed=0, kind="energy", log=None):
    """Adam on the per-sample relative error (element energy norm, or plain squared
    error with kind="l2"); returns (theta, per-epoch mean loss)."""
    import torch

    dev = data.xin.device
    n = len(data)
    theta = init_params(seed, dev)
    npar = theta.numel()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    g = torch.empty_like(theta)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ws = torch.empty(nekax.net_train_workspace_bytes(batch) // 4 + 64, dtype=torch.float32, device=dev)
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(dev)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            _grad(data, idx, batch, theta, g, loss, ws, kind)
            step += 1
            nekax.adam_step(npar, theta, g, m, v, lr * (0.5 ** (ep / max(1, epochs / 3))), step)
            tot += float(loss.item())
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    return theta, hist


def validation_loss(theta, data, batch=256, kind="energy"):
    import torch

    dev = data.xin.device
    ws = torch.empty(nekax.net_train_workspace_bytes(batch) // 4 + 64, dtype=torch.float32, device=dev)
    g = torch.empty_like(theta)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    tot, cnt = 0.0, 0
    for b0 in range(0, len(data) - batch + 1, batch):
        idx = torch.arange(b0, b0 + batch, device=dev)
        _grad(data, idx, batch, theta, g, loss, ws, kind)
        tot += float(loss.item())
        cnt += 1
    return tot / max(cnt, 1)


TRUNCATION = 8  # FCG(m) window: the directions each new one is made A-orthogonal to


def compare_on_mesh(theta, mesh, seed=0, tol=1e-8, device="cuda", stag_window=200, stag_factor=0.8,
                    truncation=TRUNCATION, theta_untrained=None):
    """Time and iterations to tol: Jacobi-PCG versus truncated flexible CG with the network (and, when
    theta_untrained is given, with that network too)."""
    import torch

    P = DeviceProblem(mesh, device)
    Gff = P.prepare_ff()
    f = torch.from_numpy(inputs.random_global_field(mesh, seed=seed)).to(device)
    x = torch.empty_like(f)
    out = {}
    # warm-up of both paths
    P.cg(f, x, tol=tol, max_iter=5, ax_impl=nekax.AX_FF)
    nekax.fcg_solve(P.gs, mesh.nelt, NX, P.D, P.G, Gff, P.mask, P.minv, theta, f, x, tol=tol, max_iter=5,
                    truncation=truncation)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = P.cg(f, x, tol=tol, max_iter=100000, ax_impl=nekax.AX_FF, check_every=10)
    torch.cuda.synchronize()
    out["jacobi_pcg"] = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "relres": r["relres"]}
    runs = [("learned_fcg", theta)] + ([("untrained_fcg", theta_untrained)] if theta_untrained is not None else [])
    for name, th in runs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = nekax.fcg_solve(P.gs, mesh.nelt, NX, P.D, P.G, Gff, P.mask, P.minv, th, f, x, tol=tol, max_iter=100000,
                            stag_window=stag_window, stag_factor=stag_factor, truncation=truncation)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "relres": r["relres"],
                     "fell_back_at": r["fell_back_at"], "net_ms": r["net_ms"],
                     "net_applications": r["net_applications"], "truncation": truncation,
                     "status": nekax.status_string(r["status"])}
    return out
