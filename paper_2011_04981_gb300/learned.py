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
e_k / multiplicity / rms(Minv r_k).  Training minimises the relative squared
error per sample with Adam.
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
    """w = mask(f - dssum(AX x)) on the device."""
    P.ax_ff(x, w)
    P.gs.dssum(w)
    w.neg_().add_(f)
    nekax.mask(P.npts, P.mask, w)


def make_training_data(n_meshes=200, pairs_per_mesh=100, snapshots=5, e=8, seed=0, device="cuda"):
    """Returns (xin [N,2,512] float32, target [N,512] float32) on the device."""
    import torch

    rng = np.random.default_rng(seed)
    X, T = [], []
    for m in range(n_meshes):
        mesh = mesh_family(10_000 + seed * 1000 + m, e)
        P = DeviceProblem(mesh, device)
        P.prepare_ff()
        f = torch.from_numpy(inputs.random_global_field(mesh, seed=m)).to(device)
        xs = torch.empty_like(f)
        res = P.cg(f, xs, tol=1e-13, max_iter=20000, ax_impl=nekax.AX_FF, check_every=10)
        n_it = max(2, res["iters"])
        ks = np.unique(np.sort(np.exp(rng.uniform(0.0, math.log(0.8 * n_it), size=snapshots)).astype(int) + 1))
        c = torch.empty_like(f)
        P.gs.inv_multiplicity(c)
        xk = torch.empty_like(f)
        r = torch.empty_like(f)
        xin = torch.empty((mesh.nelt, 2, 512), dtype=torch.float32, device=device)
        sc = torch.empty(mesh.nelt, dtype=torch.float32, device=device)
        per = max(1, pairs_per_mesh // len(ks))
        for k in ks:
            P.cg(f, xk, tol=0.0, max_iter=int(k), ax_impl=nekax.AX_FF)
            _residual(P, f, xk, r)
            nekax.net_prep(mesh.nelt, NX, r, P.minv, xin, sc)
            err = (xs - xk) * c
            good = torch.nonzero(sc > 0).flatten()
            sel = good[torch.from_numpy(rng.choice(good.numel(), size=min(per, good.numel()), replace=False)).to(
                device)]
            X.append(xin[sel].clone())
            T.append((err[sel] / sc[sel, None].double()).float())
        del P
    return torch.cat(X), torch.cat(T)


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


def train(xin, target, epochs=20, batch=256, lr=2e-3, seed=0, log=None):
    """Adam on the relative squared error; returns (theta, per-epoch mean loss)."""
    import torch

    dev = xin.device
    n = xin.shape[0]
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
            xb = xin[idx].contiguous()
            tb = target[idx].contiguous()
            nekax.net_train_grad(batch, theta, xb, tb, g, loss, ws)
            step += 1
            nekax.adam_step(npar, theta, g, m, v, lr * (0.5 ** (ep / max(1, epochs / 3))), step)
            tot += float(loss.item())
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    return theta, hist


def validation_loss(theta, xin, target, batch=256):
    import torch

    ws = torch.empty(nekax.net_train_workspace_bytes(batch) // 4 + 64, dtype=torch.float32, device=xin.device)
    g = torch.empty_like(theta)
    loss = torch.zeros(1, dtype=torch.float32, device=xin.device)
    tot, cnt = 0.0, 0
    for b0 in range(0, xin.shape[0] - batch + 1, batch):
        nekax.net_train_grad(batch, theta, xin[b0:b0 + batch].contiguous(), target[b0:b0 + batch].contiguous(), g,
                             loss, ws)
        tot += float(loss.item())
        cnt += 1
    return tot / max(cnt, 1)


def compare_on_mesh(theta, mesh, seed=0, tol=1e-8, device="cuda", stag_window=50, stag_factor=0.1):
    """Time and iterations to tol: Jacobi-PCG versus flexible CG with the network."""
    import torch

    P = DeviceProblem(mesh, device)
    Gff = P.prepare_ff()
    f = torch.from_numpy(inputs.random_global_field(mesh, seed=seed)).to(device)
    x = torch.empty_like(f)
    out = {}
    # warm-up of both paths
    P.cg(f, x, tol=tol, max_iter=5, ax_impl=nekax.AX_FF)
    nekax.fcg_solve(P.gs, mesh.nelt, NX, P.D, P.G, Gff, P.mask, P.minv, theta, f, x, tol=tol, max_iter=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = P.cg(f, x, tol=tol, max_iter=100000, ax_impl=nekax.AX_FF, check_every=10)
    torch.cuda.synchronize()
    out["jacobi_pcg"] = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "relres": r["relres"]}
    t0 = time.perf_counter()
    r = nekax.fcg_solve(P.gs, mesh.nelt, NX, P.D, P.G, Gff, P.mask, P.minv, theta, f, x, tol=tol, max_iter=100000,
                        stag_window=stag_window, stag_factor=stag_factor)
    torch.cuda.synchronize()
    out["learned_fcg"] = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "relres": r["relres"],
                          "fell_back_at": r["fell_back_at"], "net_ms": r["net_ms"],
                          "net_applications": r["net_applications"],
                          "status": nekax.status_string(r["status"])}
    return out
