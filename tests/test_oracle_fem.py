"""Oracle finite-element pins: closed forms, invariants and consistency of the discrete forms."""
import os

import numpy as np
import pytest

from chns_workloads import configs, octree
from oracle import fem
from oracle.mesh import Mesh

GOLD = os.path.join(os.path.dirname(__file__), "golden", "q1_cube_element.txt")


def _golden():
    rows = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        rows[k] = np.array([float(x) for x in v])
    return rows


def _ndiff(a, b):
    return bin(a ^ b).count("1")


PRM = dict(Re=35.0, We=2.0, Cn=0.05, Pe=50.0, Fr=1.0, rho_ratio=20.0, eta_ratio=5.0, dt=1e-3,
           C_I=6.0)


def _hang_mesh(seed=0, extent=(1.0, 1.0, 1.0)):
    a, l = configs.random_balanced(seed, 1, 4, 0.3)
    return Mesh(a, l, extent)


def test_element_matrices_closed_form():
    g = _golden()
    a, l = octree.uniform(0)
    m = Mesh(a, l)
    el = fem.Elem(m)
    K = np.einsum("eqad,eqbd->eab", el.G, el.G)[0] * el.detJ[0]
    M = np.einsum("qa,qb->ab", fem.N_Q, fem.N_Q) * el.detJ[0]
    h = 1.0
    for i in range(8):
        for j in range(8):
            k = _ndiff(i, j)
            assert abs(K[i, j] - h / 12 * g["S"][k]) < 1e-14
            assert abs(M[i, j] - h ** 3 / 216 * g["M"][k]) < 1e-15


def test_uniform_stencil_27pt():
    g = _golden()
    a, l = octree.uniform(3)
    m = Mesh(a, l)
    el = fem.Elem(m)
    A = fem.stiffness(el, np.ones((m.n_elem, 8)))
    h = 1.0 / 8
    # interior node (4,4,4) on the level-3 grid
    target = np.array([4, 4, 4]) << (20 - 3)
    i = int(np.nonzero(np.all(m.node_int == target, axis=1))[0][0])
    row = A.getrow(i).toarray().ravel()
    for j in np.nonzero(row)[0]:
        k = int(np.sum(m.node_int[j] != m.node_int[i]))
        assert abs(row[j] - h / 3 * g["L"][k]) < 1e-14
    assert np.count_nonzero(np.abs(row) > 1e-15) == 1 + 12 + 8


@pytest.mark.parametrize("seed", [0, 1])
def test_poisson_symmetric_nullspace_psd_patch(seed):
    m = _hang_mesh(seed, extent=(1.0, 4.0, 1.0))
    el = fem.Elem(m)
    co = fem.Coeffs(PRM)
    rng = np.random.default_rng(seed)
    phi = np.tanh(rng.standard_normal(m.n_nodes) * 2)
    A = fem.poisson(el, co, phi)
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()
    assert np.abs(A @ np.ones(m.n_nodes)).max() < 1e-13 * abs(A).max()
    x = rng.standard_normal(m.n_nodes)
    assert x @ (A @ x) > 0
    # patch test with constant coefficient: linear fields give zero interior residual
    K = fem.stiffness(el, np.ones((m.n_elem, 8)))
    lin = 0.3 + m.node_xyz @ np.array([1.0, -2.0, 0.5])
    assert np.abs((K @ lin)[~m.boundary]).max() < 1e-12
    # constant density reduces to rho^{-1} K
    A1 = fem.poisson(el, co, np.full(m.n_nodes, 0.25))
    assert abs(A1 - K / co.rho(0.25)).max() < 1e-13


def test_mass_integrates_volume():
    m = _hang_mesh(2, extent=(1.0, 4.0, 1.0))
    el = fem.Elem(m)
    M = fem.mass(el, np.ones((m.n_elem, 8)))
    one = np.ones(m.n_nodes)
    assert abs(one @ (M @ one) - 4.0) < 1e-13
    assert abs(fem.phi_mass(el, one) - 4.0) < 1e-13


def _ch_setup(seed=0):
    m = _hang_mesh(seed)
    el = fem.Elem(m)
    co = fem.Coeffs(PRM)
    rng = np.random.default_rng(seed)
    N = m.n_nodes
    phi, mu = np.tanh(rng.standard_normal(N)), rng.standard_normal(N)
    phik, muk = np.tanh(rng.standard_normal(N)), rng.standard_normal(N)
    u = rng.standard_normal((3, N))
    u[:, m.boundary] = 0.0
    return m, el, co, phi, mu, phik, muk, u


def test_ch_jacobian_is_derivative_of_residual():
    m, el, co, phi, mu, phik, muk, u = _ch_setup(0)
    N = m.n_nodes
    J = fem.ch_jacobian(el, co, 0.5 * (phi + phik), u)
    d = np.random.default_rng(9).standard_normal(2 * N)
    eps = 1e-6

    def F(x):
        return np.concatenate(fem.ch_residual(el, co, x[:N], x[N:], phik, muk, u))
    x = np.concatenate([phi, mu])
    fd = (F(x + eps * d) - F(x - eps * d)) / (2 * eps)
    assert np.abs(fd - J @ d).max() < 1e-7 * np.abs(J @ d).max()


def test_ch_mass_conservation_identity():
    # testing with q = 1 (sum of all rows): all gradient terms vanish (Prop. mass_conservation)
    m, el, co, phi, mu, phik, muk, u = _ch_setup(1)
    fphi, _ = fem.ch_residual(el, co, phi, mu, phik, muk, u)
    expect = (fem.phi_mass(el, phi) - fem.phi_mass(el, phik)) / co.dt
    assert abs(fphi.sum() - expect) < 1e-10 * abs(expect)


def test_ch_equilibrium_is_steady():
    # phi = +1 and mu = 0 everywhere solve the discrete CH equations for a fluid at rest
    m, el, co, *_ = _ch_setup(2)
    N = m.n_nodes
    one, zero = np.ones(N), np.zeros(N)
    u = np.zeros((3, N))
    fp, fm = fem.ch_residual(el, co, one, zero, one, zero, u)
    assert np.abs(fp).max() < 1e-12 and np.abs(fm).max() < 1e-12


def test_momentum_reduces_at_rest():
    m = _hang_mesh(3)
    el = fem.Elem(m)
    co = fem.Coeffs(PRM)
    N = m.n_nodes
    z3 = np.zeros((3, N))
    vs = fem.VMSState(el, co, np.full(N, 0.3), z3, np.full(N, 0.7))
    A = fem.momentum(vs)
    M = fem.mass(el, np.ones((m.n_elem, 8)))
    K = fem.stiffness(el, np.ones((m.n_elem, 8)))
    ref = co.rho(0.3) / co.dt * M + co.eta(0.3) / (2 * co.Re) * K
    assert abs(A - ref).max() < 1e-12 * abs(ref).max()


def test_vp_split_matches_printed_residual():
    """A v - b (operator/right-hand-side split) equals the velocity-prediction residual written
    out term by term as printed (Def. weak_VMS_disc), with the RBVMS terms tested by
    tau (u_hat.grad w / 2 + J_hat.grad w / (2 Pe rho~)) against the full R_m(v)."""
    m = _hang_mesh(4)
    el = fem.Elem(m)
    co = fem.Coeffs(PRM)
    rng = np.random.default_rng(4)
    N = m.n_nodes
    phit = np.tanh(1.5 * rng.standard_normal(N))
    uh, uk = rng.standard_normal((3, N)), rng.standard_normal((3, N))
    mut, pk = rng.standard_normal(N), rng.standard_normal(N)
    v = rng.standard_normal((3, N))
    vs = fem.VMSState(el, co, phit, uh, mut)
    A = fem.momentum(vs)
    b = fem.vp_rhs(vs, uk, pk)
    Rm = vs.residual_m(v, uk, pk)
    tv = vs.test_vms()
    rho, eta, J = vs.rho, vs.eta, vs.J
    gp = el.grad(pk)
    gph = el.grad(phit)
    for i in range(3):
        gv, gu = el.grad(v[i]), el.grad(uk[i])
        vq, uq = el.val(v[i]), el.val(uk[i])
        t_n = (rho * (vq - uq) / co.dt + 0.5 * rho * np.sum(uh_q(el, uh) * (gv + gu), -1)
               + 0.5 / co.Pe * np.sum(J * (gv + gu), -1) + gp[..., i]
               - rho * fem.GHAT[i] / co.Fr)
        t_g = (0.5 / co.Re) * eta[..., None] * (gv + gu) - (co.Cn / co.We) * gph[..., i:i + 1] * gph
        re = (np.einsum("e,qa,eq->ea", el.detJ, fem.N_Q, t_n)
              + np.einsum("e,eqad,eqd->ea", el.detJ, el.G, t_g)
              + np.einsum("e,eqa,eq->ea", el.detJ, tv, Rm[..., i]))
        r = m.assemble_vector(re)
        assert np.abs(A @ v[i] - b[i] - r).max() < 1e-10 * np.abs(r).max()


def uh_q(el, uh):
    return np.stack([el.val(uh[i]) for i in range(3)], axis=-1)


def test_tau_m_limits():
    # with u_hat = 0 and constant phi, tau_m = (4/dt^2 + C_I (eta/(rho Re))^2 G:G)^(-1/2)
    a, l = octree.uniform(2)
    m = Mesh(a, l)
    el = fem.Elem(m)
    co = fem.Coeffs(PRM)
    N = m.n_nodes
    vs = fem.VMSState(el, co, np.full(N, -0.2), np.zeros((3, N)), np.zeros(N))
    h = 0.25
    GG = 3 * (4 / h ** 2) ** 2
    ref = (4 / co.dt ** 2 + co.C_I * (co.eta(-0.2) / (co.rho(-0.2) * co.Re)) ** 2 * GG) ** -0.5
    assert np.allclose(vs.tau, ref, rtol=1e-14)


@pytest.mark.parametrize("axis", [0, 1])
def test_tau_m_advective_limit_is_half_the_transit_time(axis):
    """With dt and Re so large that their terms vanish, a uniform velocity U along one axis of a
    box element gives tau_m = h_d / (2 U): half the time the flow takes to cross the element
    along that axis (G = diag(4 / h_d^2) on the reference cell [-1, 1]^3). On the (1, 4, 1) box
    the y sides are 4x longer, so tau_m along y is 4x that along x."""
    a, l = octree.uniform(2)
    m = Mesh(a, l, (1.0, 4.0, 1.0))
    el = fem.Elem(m)
    co = fem.Coeffs(dict(PRM, dt=1e30, Re=1e30))
    N = m.n_nodes
    U = 0.7
    u = np.zeros((3, N))
    u[axis] = U
    vs = fem.VMSState(el, co, np.full(N, 0.3), u, np.zeros(N))
    h = [0.25, 1.0, 0.25][axis]
    assert np.allclose(vs.tau, h / (2 * U), rtol=1e-12)


def test_tau_m_with_the_diffusive_flux_velocity():
    """Adding a chemical-potential gradient along the flow: J = -(alpha / Cn) grad mu enters the
    advective radicand as u.G.J / (rho Pe), i.e. the transit time is taken with u and the
    diffusive flux velocity J / (rho Pe) together: tau_m = h / (2 sqrt(U (U + J_x / (rho Pe)))).
    A sign or factor slip in that term moves tau_m by more than the tolerance."""
    a, l = octree.uniform(2)
    m = Mesh(a, l)
    el = fem.Elem(m)
    co = fem.Coeffs(dict(PRM, dt=1e30, Re=1e30))
    N = m.n_nodes
    U, slope, phi0 = 0.7, 0.15, 0.3
    u = np.zeros((3, N))
    u[0] = U
    mu = slope * m.node_xyz[:, 0]
    vs = fem.VMSState(el, co, np.full(N, phi0), u, mu)
    Jx = -(co.alpha / co.Cn) * slope
    rho = co.rho(phi0)
    ref = 0.25 / (2 * np.sqrt(U * (U + Jx / (rho * co.Pe))))
    assert abs(Jx / (rho * co.Pe)) > 0.05 * U  # the term matters at this tolerance
    assert np.allclose(vs.tau, ref, rtol=1e-12)
