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

    def ax(self, u, w, stream=None):
        nekax.ax(self.nelt, self.nx, self.D, self.G, u, w, stream)

    def ax_ff(self, u, w, stream=None):
        nekax.ax_ff(self.nelt, self.nx, self.D, self.prepare_ff(), u, w, stream)

    def cg(self, f, x, tol=1e-8, max_iter=1000, workspace=None, check_every=1, time_ax=False, stream=None,
           ax_impl=nekax.AX_FP64):
        Gff = self.prepare_ff() if ax_impl == nekax.AX_FF else None
        return nekax.cg_solve(self.gs, self.nelt, self.nx, self.D, self.G, self.mask, self.minv, f, x, tol,
                              max_iter, workspace, check_every, time_ax, stream, ax_impl=ax_impl, Gff=Gff)
