"""Oracle time step: the two-block iteration of the projection scheme.

TEST INFRASTRUCTURE ONLY (see the package header).

Follows the flowchart (Fig. "flowchart_block") and Sec. 4: for blocks l = 0, 1 [reading R11]:
  1. Cahn-Hilliard (phi, mu)^{k+1,(l)} by Newton, advected by u~ = (u^k + u^{k+1,(l-1)})/2 with
     u^{k+1,(-1)} := u^k;
  2. velocity prediction v^{k+1,(l)} with u_hat = (3u^k - u^{k-1})/2 [R1], rho~, eta~ from
     phi~ = (phi^{k+1,(l)} + phi^k)/2 and J_hat from mu~ = (mu^{k+1,(l)} + mu^k)/2;
  3. pressure Poisson p^{k+1,(l)} (mean zero) [R6, R7];
  4. velocity update u^{k+1,(l)}.
Pressure is p/We throughout [R3]. Velocity is zero on the boundary (H^1_0).

Pins: mass conservation of phi across a step, energy behaviour on unforced configurations,
and (for the whole scheme) nothing independent beyond these: parity unpinned for the values of
a full step other than these invariants.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fem, solvers
from .mesh import Mesh


@dataclass
class State:
    phi: np.ndarray
    mu: np.ndarray
    u: np.ndarray        # (3, N) u^k
    u_old: np.ndarray    # (3, N) u^{k-1}
    p: np.ndarray        # p^k / We


def _lin(A, b, kind, x0=None, rtol=1e-12):
    if kind == "direct":
        return solvers.direct(A, b)
    return solvers.gmres(A, b, x0=x0, rtol=rtol)


def chns_step(mesh: Mesh, prm: dict, st: State, lin="direct", newton_rtol=1e-10,
              pp_rtol=1e-12, blocks=2, log=None, forcing=None, t=0.0, velocity_bc=None):
    """One step from the state at time t. Two optional arguments serve the
    manufactured-solution tests only:
    forcing: a callable (x_qp (E, q, 3), time) -> dict(f_v (E, q, 3), f_phi (E, q), f_mu (E, q))
      of body forces, evaluated at the midpoint t + dt/2 where the scheme's time averages are
      centred;
    velocity_bc: a callable (x_nodes (N, 3), time) -> (3, N) velocity values whose boundary
      entries at t + dt are imposed on v^{k+1} and u^{k+1} (Dirichlet data instead of no-slip)."""
    el = fem.Elem(mesh)
    co = fem.Coeffs(prm)
    N = mesh.n_nodes
    bnd = mesh.boundary
    u_hat = 0.5 * (3.0 * st.u - st.u_old)
    phi, mu = st.phi.copy(), st.mu.copy()
    u_blk = st.u.copy()
    p_new = st.p.copy()
    fq = forcing(fem.qp_coords(el), t + 0.5 * co.dt) if forcing is not None else {}
    g = velocity_bc(mesh.node_xyz, t + co.dt) if velocity_bc is not None else np.zeros((3, N))
    for l in range(blocks):
        u_t = 0.5 * (st.u + u_blk)

        def F(x):
            a, b = fem.ch_residual(el, co, x[:N], x[N:], st.phi, st.mu, u_t,
                                   fq.get("f_phi"), fq.get("f_mu"))
            return np.concatenate([a, b])

        def J(x):
            return fem.ch_jacobian(el, co, 0.5 * (x[:N] + st.phi), u_t)

        x, its, fn = solvers.newton(F, J, np.concatenate([phi, mu]), rtol=newton_rtol,
                                    linsolve=lambda A, b: _lin(A, b, lin))
        phi, mu = x[:N], x[N:]
        phi_t, mu_t = 0.5 * (phi + st.phi), 0.5 * (mu + st.mu)
        vs = fem.VMSState(el, co, phi_t, u_hat, mu_t, fq.get("f_v"))
        Am = fem.momentum(vs)
        bv = fem.vp_rhs(vs, st.u, st.p)
        v = np.zeros((3, N))
        for i in range(3):
            A2, b2 = solvers.dirichlet(Am, bv[i], bnd, g[i])
            v[i] = _lin(A2, b2, lin)
        Ap = fem.poisson(el, co, phi_t)
        bp = fem.pp_rhs(vs, v, st.u, st.p)
        p_new, pits, _ = solvers.pcg(Ap, bp, x0=st.p, rtol=pp_rtol, mean_zero=True)
        Mr = fem.mass_rho(el, co, phi_t)
        bu = fem.vu_rhs(vs, v, st.u, st.p, p_new)
        u_new = np.zeros((3, N))
        for i in range(3):
            A2, b2 = solvers.dirichlet(Mr, bu[i], bnd, g[i])
            u_new[i] = _lin(A2, b2, lin)
        u_blk = u_new
        if log is not None:
            log.append(dict(block=l, newton_its=its, newton_res=fn, pp_its=pits))
    return State(phi=phi, mu=mu, u=u_blk, u_old=st.u.copy(), p=p_new)
