"""Device-resident problem set-up through the library's own entry points.

Given a mesh from :mod:`inputs`, builds on the GPU everything the solve needs:
D (nek_gll), G (nek_geom), the gather-scatter plan (nek_gs_create), the
Dirichlet mask and the Jacobi inverse diagonal (nek_jacobi_minv).  This module
only moves buffers and calls the C ABI.
"""
from __future__ import annotations

import numpy as np

from . import nekax


class DeviceProblem:
    def __init__(self, mesh, device="cuda", build_minv=True):
        import torch

        self.mesh = mesh
        self.nelt, self.nx = mesh.nelt, mesh.nx
        self.npts = mesh.npts
        self.device = torch.device(device)
        xi, rho, D = nekax.gll(self.nx)
        self.xi, self.rho, self.D_host = xi, rho, D
        self.D = torch.from_numpy(D).to(self.device)
        corners = torch.from_numpy(np.ascontiguousarray(mesh.corners)).to(self.device)
        self.G = torch.empty((self.nelt, self.nx ** 3, 6), dtype=torch.float64, device=self.device)
        nekax.geom(self.nelt, self.nx, corners, self.G)
        del corners
        self.gs = nekax.GsPlan(self.nelt, self.nx, mesh.glo_num)
        self.mask = torch.from_numpy(np.ascontiguousarray(mesh.mask)).to(self.device)
        self.Gff = None
        self.Goz = None
        self.minv = None
        if build_minv:
            self.minv = torch.empty((self.nelt, self.nx ** 3), dtype=torch.float64, device=self.device)
            nekax.jacobi_minv(self.gs, self.nelt, self.nx, self.D, self.G, self.mask, self.minv)

    def prepare_ff(self):
        """Split G into the float-pair layout used by nek_ax_ff (48 B per point)."""
        import torch

        if self.Gff is None:
            self.Gff = torch.empty((self.nelt, self.nx ** 3, 12), dtype=torch.float32, device=self.device)
            nekax.geom_ff(self.nelt, self.nx, self.G, self.Gff)
        return self.Gff

    def _g_split(self, ax_impl):
        """The float-pair split of G that an operator kind reads (None for the native FP64 operator)."""
        if ax_impl == nekax.AX_FF:
            return self.prepare_ff()
        if ax_impl == nekax.AX_OZ:
            return self.prepare_oz()
        return None

    def ax(self, u, w, stream=None):
        nekax.ax(self.nelt, self.nx, self.D, self.G, u, w, stream)

    def ax_ff(self, u, w, stream=None):
        nekax.ax_ff(self.nelt, self.nx, self.D, self.prepare_ff(), u, w, stream)

    def prepare_oz(self):
        """Split G into the pair-interleaved float-pair layout used by nek_ax_oz (48 B per point)."""
        import torch

        if self.Goz is None:
            self.Goz = torch.empty((self.nelt, self.nx ** 3, 12), dtype=torch.float32, device=self.device)
            nekax.geom_oz(self.nelt, self.nx, self.G, self.Goz)
        return self.Goz

    def ax_oz(self, u, w, stream=None):
        nekax.ax_oz(self.nelt, self.nx, self.D, self.prepare_oz(), u, w, stream)

    def cg(self, f, x, tol=1e-8, max_iter=1000, workspace=None, check_every=1, time_ax=False, stream=None,
           ax_impl=nekax.AX_FP64):
        Gff = self._g_split(ax_impl)
        return nekax.cg_solve(self.gs, self.nelt, self.nx, self.D, self.G, self.mask, self.minv, f, x, tol,
                              max_iter, workspace, check_every, time_ax, stream, ax_impl=ax_impl, Gff=Gff)

    def cg_host(self, f_host, x_host, tol=1e-8, max_iter=1000, workspace=None, staging=None, check_every=1,
                time_ax=False, stream=None, ax_impl=nekax.AX_FP64):
        """The same solve with f and x in host memory (the library copies them)."""
        Gff = self._g_split(ax_impl)
        return nekax.cg_solve_host(self.gs, self.nelt, self.nx, self.D, self.G, self.mask, self.minv, f_host,
                                   x_host, tol, max_iter, workspace, staging, check_every, time_ax, stream,
                                   ax_impl=ax_impl, Gff=Gff)

    def lvec(self):
        """Unique-node plan, its Jacobi inverse diagonal and solve workspace (built once)."""
        import torch

        if getattr(self, "_lv", None) is None:
            lv = nekax.LvecPlan(self.mesh.glo_num, self.mesh.mask)
            minvL = torch.empty(lv.size, dtype=torch.float64, device=self.device)
            scratch = torch.empty(self.npts, dtype=torch.float64, device=self.device)
            lv.jacobi_minv(self.nelt, self.nx, self.D, self.G, minvL, scratch)
            del scratch
            ws = torch.empty(lv.workspace_bytes() // 8 + 64, dtype=torch.float64, device=self.device)
            self._lv = (lv, minvL, ws)
        return self._lv

    def cg_lvec(self, fL, xL, tol=1e-8, max_iter=1000, check_every=1, time_ax=False, stream=None):
        """Jacobi-PCG on unique-node vectors (fL, xL of lvec()[0].size entries), AX = nek_ax_ff."""
        lv, minvL, ws = self.lvec()
        return lv.cg_solve(self.nelt, self.nx, self.D, self.prepare_ff(), minvL, fL, xL, tol, max_iter, ws,
                           check_every, time_ax, stream)


class DeviceBatch:
    """Many meshes solved together: concatenated device buffers and a nek_batch plan.  Problems are
    ordered by nx (the plan's requirement) and, within an nx, by size: the larger need more iterations,
    so the finished ones gather at the start of each nx run, which the solve then stops launching."""

    def __init__(self, meshes, fields, device="cuda", ff=True):
        import torch

        order = sorted(range(len(meshes)), key=lambda q: (meshes[q].nx, meshes[q].nelt, q))
        self.order = order
        self.meshes = [meshes[q] for q in order]
        self.device = torch.device(device)
        nelts = [m.nelt for m in self.meshes]
        nxs = [m.nx for m in self.meshes]
        glo = np.concatenate([m.glo_num.reshape(-1) for m in self.meshes])
        self.plan = nekax.BatchPlan(nelts, nxs, glo)
        self.npts = int(sum(m.npts for m in self.meshes))
        self.offsets = np.cumsum([0] + [m.npts for m in self.meshes])
        self.G = torch.empty(self.npts * 6, dtype=torch.float64, device=self.device)
        # geometric factors per problem (one nek_geom call per problem)
        for q, m in enumerate(self.meshes):
            c = torch.from_numpy(np.ascontiguousarray(m.corners)).to(self.device)
            nekax.geom(m.nelt, m.nx, c, self.G[int(self.offsets[q]) * 6:])
        self.mask = torch.from_numpy(np.concatenate([m.mask.reshape(-1) for m in self.meshes])).to(self.device)
        self.f = torch.from_numpy(np.concatenate([fields[q].reshape(-1) for q in order])).to(self.device)
        self.minv = torch.empty(self.npts, dtype=torch.float64, device=self.device)
        self.plan.jacobi_minv(self.G, self.mask, self.minv)
        self.Gff = None
        if ff:
            self.Gff = torch.empty(self.npts * 12, dtype=torch.float32, device=self.device)
            for q, m in enumerate(self.meshes):
                o = int(self.offsets[q])
                nekax.geom_ff(m.nelt, m.nx, self.G[o * 6:], self.Gff[o * 12:])

    def solve(self, x, tol=1e-8, max_iter=5000, iters_per_graph=10, workspace=None):
        return self.plan.cg_solve(self.G, self.Gff, self.mask, self.minv, self.f, x, tol, max_iter, iters_per_graph,
                                  workspace)

    def split(self, v):
        """Per-problem views of a concatenated vector, in the caller's original order."""
        parts = [v[int(self.offsets[q]):int(self.offsets[q + 1])] for q in range(len(self.meshes))]
        out = [None] * len(parts)
        for pos, q in enumerate(self.order):
            out[q] = parts[pos]
        return out
