"""Small conveniences over the C ABI: a mesh handle with its node data, device-buffer helpers and
default solver settings. Device memory comes from torch; every computation is a libchns call."""
from __future__ import annotations

import numpy as np

from . import _lib as capi


class Mesh:
    """Owns a chns_mesh built from a Morton-ordered, 2:1-balanced leaf list."""

    def __init__(self, anchors=None, levels=None, extent=(1.0, 1.0, 1.0), stream=None,
                 handle=None):
        """From a leaf list, or (handle=) taking ownership of a mesh the library created."""
        if handle is None:
            handle = capi.chns_mesh_create(anchors, levels, extent, stream)
        self.handle = handle
        info = capi.chns_mesh_get_info(self.handle)
        self.n_elem = info.n_elem
        self.n_nodes = info.n_nodes
        self.n_hanging = info.n_hanging
        self.n_boundary = info.n_boundary
        self.min_level, self.max_level = info.min_level, info.max_level
        self.extent = np.array(list(info.extent))
        self.node_int = capi.chns_mesh_node_coords(self.handle, self.n_nodes)
        self.boundary = capi.chns_mesh_boundary(self.handle, self.n_nodes).astype(bool)
        self.node_xyz = self.node_int.astype(np.float64) / float(1 << capi.MAXD) * self.extent

    def leaves(self):
        """(anchors, levels) of the mesh in Morton order."""
        return capi.chns_mesh_leaves(self.handle, self.n_elem)

    def close(self):
        if self.handle:
            capi.chns_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_step_params(rtol=1e-8, inner=capi.FP64, pp_check_every=8, inner_rtol=1e-6,
                        newton_rtol=1e-10):
    """Solver settings of a time step: GMRES for CH and velocity prediction, Jacobi-PCG for the
    pressure Poisson and velocity update, all to the relative residual rtol. In the FP32 modes each
    refinement cycle solves its correction to inner_rtol (CG) or 100 x inner_rtol (GMRES)."""
    gm = capi.make_solver(capi.KSP_GMRES, capi.PC_JACOBI, rtol, 4000, 30, inner,
                          100 * inner_rtol)
    cg = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, rtol, 20000, 30, inner, inner_rtol,
                          check_every=pp_check_every)
    cgv = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, rtol, 4000, 30, inner, inner_rtol,
                           check_every=pp_check_every)
    return capi.chns_step_params(gm, gm, cg, cgv, newton_rtol, 1e-14, 10, 2)


class DeviceState:
    """FP64 device fields (phi, mu, u, u_old, p) as torch tensors plus the C view of them."""

    def __init__(self, fields: dict, device="cuda"):
        import torch
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
        self.phi = t(fields["phi"])
        self.mu = t(fields["mu"])
        self.u = [t(fields["u"][i]) for i in range(3)]
        uo = fields.get("u_old", fields["u"])
        self.u_old = [t(uo[i]) for i in range(3)]
        self.p = t(fields["p"])
        self._bind()

    def _bind(self):
        self.c = capi.chns_state(self.phi.data_ptr(), self.mu.data_ptr(),
                                 (capi.C.c_void_p * 3)(*[x.data_ptr() for x in self.u]),
                                 (capi.C.c_void_p * 3)(*[x.data_ptr() for x in self.u_old]),
                                 self.p.data_ptr())

    def host(self):
        return dict(phi=self.phi.cpu().numpy(), mu=self.mu.cpu().numpy(),
                    u=np.stack([x.cpu().numpy() for x in self.u]),
                    u_old=np.stack([x.cpu().numpy() for x in self.u_old]),
                    p=self.p.cpu().numpy())


class VelocityBC:
    """Velocity Dirichlet data on the device: three FP64 arrays of n_nodes (only the entries of
    boundary nodes are read), imposed by chns_step in place of no-slip once attached to the step
    parameters. The arrays must outlive every step that uses them."""

    def __init__(self, g, device="cuda"):
        import torch
        self.g = [torch.as_tensor(np.ascontiguousarray(g[i], dtype=np.float64), device=device)
                  for i in range(3)]

    def attach(self, sp):
        sp.u_bc = (capi.C.c_void_p * 3)(*[x.data_ptr() for x in self.g])
        return sp


def remesh(mesh: Mesh, ds: "DeviceState", threshold=0.95, lmin=None, lmax=None, stream=None):
    """One adaptive remesh (Sec. 5.4): the new mesh from the interface band of ds.phi and every
    field of ds (phi, mu, u, u_old, p) transferred to it. Returns (new Mesh, new DeviceState);
    the old ones are left unchanged."""
    import torch
    lmin = mesh.min_level if lmin is None else lmin
    lmax = mesh.max_level if lmax is None else lmax
    new_mesh = Mesh(handle=capi.chns_mesh_remesh(mesh.handle, ds.phi, threshold, lmin, lmax,
                                                 stream))
    n = new_mesh.n_nodes
    z = lambda: torch.empty(n, dtype=torch.float64, device=ds.phi.device)
    new = DeviceState.__new__(DeviceState)
    new.phi, new.mu, new.p = z(), z(), z()
    new.u = [z() for _ in range(3)]
    new.u_old = [z() for _ in range(3)]
    capi.chns_transfer(mesh.handle, new_mesh.handle,
                       [ds.phi, ds.mu, *ds.u, *ds.u_old, ds.p],
                       [new.phi, new.mu, *new.u, *new.u_old, new.p], stream)
    new._bind()
    return new_mesh, new
