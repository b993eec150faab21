"""Oracle finite-element operators and right-hand sides (FP64, assembled sparse matrices).

TEST INFRASTRUCTURE ONLY (see the package header).

Discretisation: continuous Q1 (trilinear) elements on axis-aligned box leaves (r = 1, Sec. 4.1),
2x2x2 Gauss quadrature, reference cell [-1,1]^3 with Jacobian diag(h/2). Coefficients are
evaluated at quadrature points from the Q1 interpolant of nodal fields. Element matrices are
formed by plain einsum over elements and assembled as A = P^T (sum_e A_e) P (mesh.Mesh).

Model (Sec. 3): rho(phi) = alpha phi + beta, eta(phi) = gamma phi + xi with
alpha = (rho_+ - rho_-)/(2 rho_+), beta = (rho_+ + rho_-)/(2 rho_+) (same for eta);
psi(phi) = (phi^2 - 1)^2 / 4, psi' = phi^3 - phi; mobility m = 1; g_hat = (0, -1, 0).
Density and viscosity use the pulled-back phi* = clamp(phi, -1, 1) (Eq. "phi_for_density").

Operators (readings of ambiguous passages are listed by number in the design notes):
* pressure Poisson (Def. weak_VMS_disc_pp_vel):   (grad q, (1/rho~) grad p)          [reading R6]
* velocity update (Def. weak_VMS_disc_vel_update): (w, rho~ u)
* velocity prediction (Def. weak_VMS_disc): the linear operator in v^{c,k+1} with the RBVMS
  closure rho~ v^f = -tau_m R_m, tau_m with C_I = 6 and G = diag(4/h^2) [readings R1, R3, R4, R5, R8]
  (R4: the printed radicand of tau_m is floored at 4/dt^2, i.e. tau_m <= dt/2)
* Cahn-Hilliard (Def. weak_VMS_disc_CH): residual and Newton Jacobian in (phi^{k+1}, mu^{k+1})
  [reading R2: the diffusion term enters with a plus sign, as in the strong form]

Pins: closed-form Q1 stiffness/mass on a cube, symmetry and constant null space of the Poisson
operator, reduction of the momentum operator to (rho/dt) M + (eta/(2Re)) K + VMS mass-like
term at zero velocity, CH mass conservation, Jacobian = finite difference of the residual
(tests/test_oracle_fem.py). tau_m and the VMS right-hand-side terms have no independent pin
beyond the consistency checks: parity unpinned for their values.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import CORNER_BITS, Mesh

GAUSS = 1.0 / np.sqrt(3.0)
QP = (2 * CORNER_BITS - 1).astype(np.float64) * GAUSS     # (8 qp, 3), x fastest
SGN = (2 * CORNER_BITS - 1).astype(np.float64)            # (8 nodes, 3) corner signs
GHAT = np.array([0.0, -1.0, 0.0])


def _basis():
    """N[q,a], dN[q,a,d] (reference), d2N[q,a,d,e] (reference) at the Gauss points."""
    f = 0.5 * (1.0 + SGN[None, :, :] * QP[:, None, :])    # (q, a, d) 1D factors
    df = 0.5 * SGN[None, :, :] * np.ones((8, 1, 1))       # derivative of 1D factors
    N = f.prod(axis=2)
    dN = np.zeros((8, 8, 3))
    d2N = np.zeros((8, 8, 3, 3))
    for d in range(3):
        t = df[:, :, d].copy()
        for e in range(3):
            if e != d:
                t = t * f[:, :, e]
        dN[:, :, d] = t
        for e in range(3):
            if e == d:
                continue        # second derivative of a linear 1D factor is zero
            u = df[:, :, d] * df[:, :, e]
            for g in range(3):
                if g != d and g != e:
                    u = u * f[:, :, g]
            d2N[:, :, d, e] = u
    return N, dN, d2N


N_Q, DN_REF, D2N_REF = _basis()


class Coeffs:
    """Density/viscosity maps and non-dimensional groups from a parameter dict."""

    def __init__(self, prm: dict):
        self.prm = prm
        rp, rm = 1.0, 1.0 / prm["rho_ratio"]
        ep, em = 1.0, 1.0 / prm["eta_ratio"]
        self.alpha = (rp - rm) / (2 * rp)
        self.beta = (rp + rm) / (2 * rp)
        self.gamma = (ep - em) / (2 * ep)
        self.xi = (ep + em) / (2 * ep)
        for k in ("Re", "We", "Cn", "Pe", "Fr", "dt", "C_I"):
            setattr(self, k, float(prm[k]))

    def rho(self, phi):
        return self.alpha * np.clip(phi, -1.0, 1.0) + self.beta

    def eta(self, phi):
        return self.gamma * np.clip(phi, -1.0, 1.0) + self.xi


class Elem:
    """Per-element geometry: physical gradients at the Gauss points and det J."""

    def __init__(self, mesh: Mesh):
        self.mesh = mesh
        h = mesh.h                                            # (E, 3)
        self.detJ = h.prod(axis=1) / 8.0                      # weights are 1
        s = 2.0 / h                                           # (E, 3)
        self.G = DN_REF[None, :, :, :] * s[:, None, None, :]  # (E, q, a, d)
        self.H = D2N_REF[None] * s[:, None, None, :, None] * s[:, None, None, None, :]
        self.gGd = (4.0 / h ** 2)                             # diagonal of G_ij in tau_m

    def val(self, nodal):
        """Values at qps (E, q) of a nodal field (N,)."""
        return np.einsum("qa,ea->eq", N_Q, self.mesh.element_values(nodal))

    def grad(self, nodal):
        """Gradients at qps (E, q, 3)."""
        return np.einsum("eqad,ea->eqd", self.G, self.mesh.element_values(nodal))

    def hess(self, nodal):
        """Hessian of the element interpolant at qps (E, q, 3, 3)."""
        return np.einsum("kqaij,ka->kqij", self.H, self.mesh.element_values(nodal))


def qp_coords(el: Elem) -> np.ndarray:
    """Physical coordinates of the Gauss points (E, q, 3): element anchor + h (1 + xi) / 2."""
    m = el.mesh
    x0 = m.anchors.astype(np.float64) / float(1 << 20) * m.extent[None, :]
    return x0[:, None, :] + m.h[:, None, :] * 0.5 * (1.0 + QP[None, :, :])


# ============================================================================ scalar operators
def stiffness(el: Elem, cq: np.ndarray) -> sp.csr_matrix:
    """(grad q, c grad p) with c given at the qps (E, q)."""
    Ae = np.einsum("e,eq,eqad,eqbd->eab", el.detJ, cq, el.G, el.G)
    return el.mesh.assemble_matrix(Ae)


def mass(el: Elem, cq: np.ndarray) -> sp.csr_matrix:
    """(q, c p) with c at the qps."""
    Ae = np.einsum("e,eq,qa,qb->eab", el.detJ, cq, N_Q, N_Q)
    return el.mesh.assemble_matrix(Ae)


def poisson(el: Elem, co: Coeffs, phi_t: np.ndarray) -> sp.csr_matrix:
    """Pressure-Poisson operator (grad q, (1/rho(phi~*)) grad p), Def. weak_VMS_disc_pp_vel."""
    return stiffness(el, 1.0 / co.rho(el.val(phi_t)))


def mass_rho(el: Elem, co: Coeffs, phi_t: np.ndarray) -> sp.csr_matrix:
    """Velocity-update operator (w, rho~ u) (one component), Def. weak_VMS_disc_vel_update."""
    return mass(el, co.rho(el.val(phi_t)))


def phi_mass(el: Elem, phi: np.ndarray) -> float:
    """Integral of phi over the domain by the same quadrature (1^T M phi)."""
    return float(np.einsum("e,eq->", el.detJ, el.val(phi)))


# ============================================================================ Cahn-Hilliard
def ch_residual(el: Elem, co: Coeffs, phi, mu, phi_k, mu_k, u_t, f_phi=None, f_mu=None):
    """Residual of the discrete CH equations (Def. weak_VMS_disc_CH) at (phi, mu) = new-time
    unknowns; u_t (3, N) is the advecting velocity u~. Returns (F_phi, F_mu).

    f_phi, f_mu (E, q): optional body forces at the Gauss points, used only by the
    manufactured-solution tests (Sec. 6.1 puts the residual of a chosen solution on the right-hand
    sides): -(q, f_phi) is added to F_phi and +(q, f_mu) to F_mu, the weak forms of
    dphi/dt + div(u phi) - lap(mu)/(Pe Cn) = f_phi and -mu + psi'(phi) - Cn^2 lap(phi) + f_mu = 0."""
    pt = 0.5 * (phi + phi_k)
    mt = 0.5 * (mu + mu_k)
    pq, gpt = el.val(pt), el.grad(pt)
    gmt = el.grad(mt)
    mtq = el.val(mt)
    dphi = el.val(phi - phi_k) / co.dt
    uq = np.stack([el.val(u_t[i]) for i in range(3)], axis=-1)       # (E, q, 3)
    flux = uq * pq[..., None]                                        # u~ phi~
    fphi = (np.einsum("e,qa,eq->ea", el.detJ, N_Q, dphi)
            - np.einsum("e,eqad,eqd->ea", el.detJ, el.G, flux)
            + (1.0 / (co.Pe * co.Cn)) * np.einsum("e,eqad,eqd->ea", el.detJ, el.G, gmt))
    fmu = (np.einsum("e,qa,eq->ea", el.detJ, N_Q, -mtq + (pq ** 3 - pq))
           + co.Cn ** 2 * np.einsum("e,eqad,eqd->ea", el.detJ, el.G, gpt))
    if f_phi is not None:
        fphi = fphi - np.einsum("e,qa,eq->ea", el.detJ, N_Q, f_phi)
    if f_mu is not None:
        fmu = fmu + np.einsum("e,qa,eq->ea", el.detJ, N_Q, f_mu)
    return el.mesh.assemble_vector(fphi), el.mesh.assemble_vector(fmu)


def ch_jacobian(el: Elem, co: Coeffs, phi_t, u_t) -> sp.csr_matrix:
    """Newton Jacobian of the CH residual w.r.t. (phi^{k+1}, mu^{k+1}), block order [phi; mu].
    phi_t = phi~ at the current iterate (for psi''(phi~) = 3 phi~^2 - 1)."""
    pq = el.val(phi_t)
    uq = np.stack([el.val(u_t[i]) for i in range(3)], axis=-1)
    M = np.einsum("e,qa,qb->eab", el.detJ, N_Q, N_Q)
    Mpsi = np.einsum("e,eq,qa,qb->eab", el.detJ, 3.0 * pq ** 2 - 1.0, N_Q, N_Q)
    K = np.einsum("e,eqad,eqbd->eab", el.detJ, el.G, el.G)
    C = np.einsum("e,eqad,eqd,qb->eab", el.detJ, el.G, uq, N_Q)      # (grad q . u~, dphi)
    A_pp = el.mesh.assemble_matrix(M / co.dt - 0.5 * C)
    A_pm = el.mesh.assemble_matrix((0.5 / (co.Pe * co.Cn)) * K)
    A_mp = el.mesh.assemble_matrix(0.5 * Mpsi + 0.5 * co.Cn ** 2 * K)
    A_mm = el.mesh.assemble_matrix(-0.5 * M)
    return sp.bmat([[A_pp, A_pm], [A_mp, A_mm]]).tocsr()


# ============================================================================ momentum (VP)
class VMSState:
    """Quadrature-point coefficients of the RBVMS momentum operator for one block:
    rho~, eta~, grad eta~, u_hat, J_hat, tau_m (Def. weak_VMS_disc, tau_m definition)."""

    def __init__(self, el: Elem, co: Coeffs, phi_t, u_hat, mu_t, f_v=None):
        """f_v (E, q, 3): optional body force of the manufactured-solution tests, part of the
        strong residual R_m (R_m - f_v) and of the right-hand side (w, f_v)."""
        self.el, self.co = el, co
        self.f_v = f_v
        pq = el.val(phi_t)
        self.rho = co.rho(pq)
        self.eta = co.eta(pq)
        inside = (np.abs(pq) < 1.0)[..., None]
        self.geta = co.gamma * el.grad(phi_t) * inside                 # [R8]
        self.uh = np.stack([el.val(u_hat[i]) for i in range(3)], axis=-1)
        self.J = -(co.alpha / co.Cn) * el.grad(mu_t)                   # [R5]
        G = el.gGd[:, None, :]                                          # (E, 1, 3)
        # printed tau_m, with its radicand floored at 4/dt^2 (tau_m <= dt/2) [reading R4: the
        # mixed term u.G.J/(rho Pe) can take the printed radicand below 4/dt^2 and negative where
        # J/(rho Pe) >> u; elsewhere the printed value is used as it stands]
        ugu = np.sum(self.uh * G * self.uh, axis=-1)
        ugj = (1.0 / (self.rho * co.Pe)) * np.sum(self.uh * G * self.J, axis=-1)
        t = (4.0 / co.dt ** 2 + ugu + ugj
             + co.C_I * (self.eta / (self.rho * co.Re)) ** 2 * np.sum(G ** 2, axis=-1))
        self.tau = np.maximum(t, 4.0 / co.dt ** 2) ** -0.5
        # forcing d_j(d_i phi d_j phi) from the element Hessian (reading R8)
        gp = el.grad(phi_t)
        Hp = el.hess(phi_t)
        lap = np.trace(Hp, axis1=2, axis2=3)
        self.gphi = gp
        self.force = np.einsum("eqij,eqj->eqi", Hp, gp) + gp * lap[..., None]

    def rlin_basis(self):
        """R^lin applied to each basis function: (E, q, b)."""
        el, co = self.el, self.co
        adv = np.einsum("eqd,eqbd->eqb", self.uh, el.G)
        jdv = np.einsum("eqd,eqbd->eqb", self.J, el.G)
        edv = np.einsum("eqd,eqbd->eqb", self.geta, el.G)
        return (self.rho[..., None] * N_Q[None] / co.dt + 0.5 * self.rho[..., None] * adv
                + (0.5 / co.Pe) * jdv - (0.5 / co.Re) * edv)

    def test_vms(self):
        """Weights of the VMS test terms: tau (1/2 u_hat.grad N_a + 1/(2 Pe rho~) J.grad N_a)."""
        el, co = self.el, self.co
        adv = np.einsum("eqd,eqad->eqa", self.uh, el.G)
        jdv = np.einsum("eqd,eqad->eqa", self.J, el.G)
        return self.tau[..., None] * (0.5 * adv + (0.5 / (co.Pe * self.rho[..., None])) * jdv)

    def residual_m(self, v, u_k, p_k):
        """Full R_m,i at qps (E, q, 3) for a velocity v^{c,k+1} (3, N) (Def. of R_m)."""
        el, co = self.el, self.co
        vt = 0.5 * (v + u_k)
        out = np.zeros(self.rho.shape + (3,))
        gp = el.grad(p_k)
        for i in range(3):
            gvt = el.grad(vt[i])
            out[..., i] = (self.rho * (el.val(v[i]) - el.val(u_k[i])) / co.dt
                           + self.rho * np.sum(self.uh * gvt, axis=-1)
                           + (1.0 / co.Pe) * np.sum(self.J * gvt, axis=-1)
                           + (co.Cn / co.We) * self.force[..., i]
                           + gp[..., i]
                           - (1.0 / co.Re) * np.sum(self.geta * gvt, axis=-1)
                           - self.rho * GHAT[i] / co.Fr)
            if self.f_v is not None:
                out[..., i] -= self.f_v[..., i]
        return out


def momentum(vs: VMSState) -> sp.csr_matrix:
    """Scalar velocity-prediction operator (same for each component; no cross terms)."""
    el, co = vs.el, vs.co
    adv = np.einsum("eqd,eqbd->eqb", vs.uh, el.G)
    jdv = np.einsum("eqd,eqbd->eqb", vs.J, el.G)
    Ae = (np.einsum("e,eq,qa,qb->eab", el.detJ, vs.rho / co.dt, N_Q, N_Q)
          + 0.5 * np.einsum("e,eq,qa,eqb->eab", el.detJ, vs.rho, N_Q, adv)
          + (0.5 / co.Pe) * np.einsum("e,qa,eqb->eab", el.detJ, N_Q, jdv)
          + (0.5 / co.Re) * np.einsum("e,eq,eqad,eqbd->eab", el.detJ, vs.eta, el.G, el.G)
          + np.einsum("e,eqa,eqb->eab", el.detJ, vs.test_vms(), vs.rlin_basis()))
    return el.mesh.assemble_matrix(Ae)


def vp_rhs(vs: VMSState, u_k, p_k):
    """Right-hand side of the velocity prediction for each component (3, N)."""
    el, co = vs.el, vs.co
    gp = el.grad(p_k)
    tv = vs.test_vms()
    out = []
    for i in range(3):
        uq, gu = el.val(u_k[i]), el.grad(u_k[i])
        r0 = (-vs.rho * uq / co.dt + 0.5 * vs.rho * np.sum(vs.uh * gu, -1)
              + (0.5 / co.Pe) * np.sum(vs.J * gu, -1) + (co.Cn / co.We) * vs.force[..., i]
              + gp[..., i] - (0.5 / co.Re) * np.sum(vs.geta * gu, -1)
              - vs.rho * GHAT[i] / co.Fr)
        f_n = (vs.rho * uq / co.dt - 0.5 * vs.rho * np.sum(vs.uh * gu, -1)
               - (0.5 / co.Pe) * np.sum(vs.J * gu, -1) - gp[..., i]
               + vs.rho * GHAT[i] / co.Fr)                               # times N_a
        if vs.f_v is not None:
            r0 = r0 - vs.f_v[..., i]
            f_n = f_n + vs.f_v[..., i]
        f_g = (-(0.5 / co.Re) * vs.eta[..., None] * gu
               + (co.Cn / co.We) * vs.gphi[..., i:i + 1] * vs.gphi)        # dotted with grad N_a
        be = (np.einsum("e,qa,eq->ea", el.detJ, N_Q, f_n)
              + np.einsum("e,eqad,eqd->ea", el.detJ, el.G, f_g)
              - np.einsum("e,eqa,eq->ea", el.detJ, tv, r0))
        out.append(el.mesh.assemble_vector(be))
    return np.stack(out)


# ============================================================================ projection (PP, VU)
def pp_rhs(vs: VMSState, v, u_k, p_k):
    """Pressure-Poisson right-hand side (Def. weak_VMS_disc_pp_vel), scalar test q [R6]:
    -(2/dt)(q, div v) - (2/dt)(grad q, tau R_m / rho~) + (grad q, grad p^k / rho~)."""
    el, co = vs.el, vs.co
    div = sum(el.grad(v[i])[..., i] for i in range(3))
    Rm = vs.residual_m(v, u_k, p_k)
    gp = el.grad(p_k)
    vec = (-(2.0 / co.dt) * vs.tau[..., None] * Rm + gp) / vs.rho[..., None]
    be = (np.einsum("e,qa,eq->ea", el.detJ, N_Q, -(2.0 / co.dt) * div)
          + np.einsum("e,eqad,eqd->ea", el.detJ, el.G, vec))
    return el.mesh.assemble_vector(be)


def vu_rhs(vs: VMSState, v, u_k, p_k, p_new):
    """Velocity-update right-hand side (Def. weak_VMS_disc_vel_update), per component (3, N):
    (w, rho~ v) - (w, tau R_m) - (dt/2)(w, d_i (p^{k+1} - p^k))."""
    el, co = vs.el, vs.co
    Rm = vs.residual_m(v, u_k, p_k)
    gdp = el.grad(p_new - p_k)
    out = []
    for i in range(3):
        f = vs.rho * el.val(v[i]) - vs.tau * Rm[..., i] - 0.5 * co.dt * gdp[..., i]
        out.append(el.mesh.assemble_vector(np.einsum("e,qa,eq->ea", el.detJ, N_Q, f)))
    return np.stack(out)


# ============================================================================ diagnostics
def energy(el: Elem, co: Coeffs, phi, u) -> float:
    """Total energy (Eq. energy_functional) with the gravity term outside the 1/(Cn We) factor
    [reading R15]; y is the second physical coordinate at each qp."""
    pq = el.val(phi)
    gp = el.grad(phi)
    uq = np.stack([el.val(u[i]) for i in range(3)], axis=-1)
    rho = co.rho(pq)
    # physical y at the qps: element y0 + h_y (1 + xi_y)/2
    y0 = el.mesh.anchors[:, 1] / float(1 << 20) * el.mesh.extent[1]
    yq = y0[:, None] + el.mesh.h[:, 1:2] * 0.5 * (1.0 + QP[None, :, 1])
    psi = 0.25 * (pq ** 2 - 1.0) ** 2
    dens = (0.5 * rho * np.sum(uq ** 2, -1)
            + (1.0 / (co.Cn * co.We)) * (psi + 0.5 * co.Cn ** 2 * np.sum(gp ** 2, -1))
            + (1.0 / co.Fr) * rho * yq)
    return float(np.einsum("e,eq->", el.detJ, dens))
