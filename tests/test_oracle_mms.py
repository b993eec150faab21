"""Manufactured-solution convergence of the oracle's discretisation (Q1, 2x2x2 Gauss, hanging
nodes interpolated from their parents, Sec. 4.1 and Sec. 5.4): for smooth exact solutions the
L2 error of the discrete solution falls as h^2 under uniform refinement (the paper's spatial
order for Q1, Sec. 6.1). A dropped term, a wrong sign or a wrong coefficient in an operator makes
the discrete problem consistent with a different equation, and the error then stalls.

Operators: the variable-density pressure Poisson operator (grad q, (1/rho(phi)) grad p) with
natural boundary conditions, on uniform and on adaptive 2:1 meshes; the linearised
Cahn-Hilliard pair (the Newton Jacobian of Def. weak_VMS_disc_CH without advection); the
velocity-prediction operator at rest ((rho/dt) M + (1/(2 Re)) (grad w, eta grad v), no-slip
walls). Loads are the quadrature of the exact forcing against the basis functions."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from chns_workloads import configs, octree
from chns_workloads.octree import MAXD
from oracle import fem, solvers
from oracle.fem import N_Q
from oracle.mesh import Mesh

PI = np.pi
PRM = dict(Re=20.0, We=1.0, Cn=0.1, Pe=50.0, Fr=1.0, rho_ratio=10.0, eta_ratio=5.0, dt=1e-2,
           C_I=6.0)


def _refine_all(a, l):
    """Every leaf split into its 8 children (2:1 balance is kept)."""
    kids = []
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], dtype=np.int64)
        kids.append(a.astype(np.int64) + off[None, :] * (1 << (MAXD - 1 - l.astype(np.int64)))[:, None])
    a2 = np.concatenate(kids).astype(np.uint32)
    l2 = np.concatenate([l + 1] * 8).astype(np.uint8)
    return octree.morton_sort(a2, l2)


def _qp_coords(el):
    return [el.val(el.mesh.node_xyz[:, d]) for d in range(3)]


def _load(el, fq):
    return el.mesh.assemble_vector(np.einsum("e,qa,eq->ea", el.detJ, N_Q, fq))


def _l2(el, nodal, exact_q):
    d = el.val(nodal) - exact_q
    return np.sqrt(np.einsum("e,eq->", el.detJ, d * d))


def _phi(x, y, z):
    return 0.5 * np.sin(2 * PI * x) * np.cos(2 * PI * y) * np.cos(2 * PI * z)


def _phi_grad(x, y, z):
    return (0.5 * 2 * PI * np.cos(2 * PI * x) * np.cos(2 * PI * y) * np.cos(2 * PI * z),
            -0.5 * 2 * PI * np.sin(2 * PI * x) * np.sin(2 * PI * y) * np.cos(2 * PI * z),
            -0.5 * 2 * PI * np.sin(2 * PI * x) * np.cos(2 * PI * y) * np.sin(2 * PI * z))


def _poisson_error(mesh):
    """p = cos(pi x) cos(pi y) cos(pi z) (zero normal derivative, zero mean), rho = rho(phi)."""
    el, co = fem.Elem(mesh), fem.Coeffs(PRM)
    x = mesh.node_xyz
    phi = _phi(x[:, 0], x[:, 1], x[:, 2])
    A = fem.poisson(el, co, phi)
    X, Y, Z = _qp_coords(el)
    p = np.cos(PI * X) * np.cos(PI * Y) * np.cos(PI * Z)
    gp = (-PI * np.sin(PI * X) * np.cos(PI * Y) * np.cos(PI * Z),
          -PI * np.cos(PI * X) * np.sin(PI * Y) * np.cos(PI * Z),
          -PI * np.cos(PI * X) * np.cos(PI * Y) * np.sin(PI * Z))
    rho = co.alpha * _phi(X, Y, Z) + co.beta        # |phi| <= 1/2: no clamping
    grho = [co.alpha * g for g in _phi_grad(X, Y, Z)]
    # f = -div((1/rho) grad p) = -(1/rho) lap p + (1/rho^2) grad rho . grad p
    f = 3 * PI ** 2 * p / rho + sum(grho[d] * gp[d] for d in range(3)) / rho ** 2
    ph, _, _ = solvers.pcg(A, _load(el, f), rtol=1e-12, mean_zero=True)
    vol = np.einsum("e,eq->", el.detJ, np.ones_like(p))
    ph = ph - np.einsum("e,eq->", el.detJ, el.val(ph)) / vol  # mean zero like the exact p
    return _l2(el, ph, p)


def _rates(errors):
    e = np.asarray(errors)
    return np.log2(e[:-1] / e[1:])


def test_poisson_variable_density_second_order_uniform():
    errs = [_poisson_error(Mesh(*octree.uniform(L))) for L in (2, 3, 4)]
    r = _rates(errs)
    assert errs[-1] < 0.1 * errs[0], errs  # two halvings of h: ~16x
    assert r[-1] > 1.8, (errs, r)


def test_poisson_second_order_on_adaptive_hanging_node_mesh():
    a, l = configs.random_balanced(1, 1, 3, 0.3)
    meshes = [Mesh(a, l)]
    for _ in range(2):
        a, l = _refine_all(a, l)
        meshes.append(Mesh(a, l))
    assert all(m.n_hanging > 0 for m in meshes)
    errs = [_poisson_error(m) for m in meshes]
    r = _rates(errs)
    assert r[-1] > 1.7, (errs, r)


def _ch_error(level):
    """Linearised CH pair without advection at constant phi~ = c0 (psi'' constant):
       dphi/dt - k lap dmu = f1,  -dmu/2 + psi'' dphi/2 - (Cn^2/2) lap dphi = f2
    (k = 1/(2 Pe Cn), the diffusion signs of reading R2), natural boundary conditions."""
    mesh = Mesh(*octree.uniform(level))
    el, co = fem.Elem(mesh), fem.Coeffs(PRM)
    n = mesh.n_nodes
    c0 = 0.3
    J = fem.ch_jacobian(el, co, np.full(n, c0), np.zeros((3, n)))
    X, Y, Z = _qp_coords(el)
    dphi = np.cos(PI * X) * np.cos(PI * Y) * np.cos(PI * Z)
    dmu = np.cos(2 * PI * X) * np.cos(PI * Y) * np.cos(2 * PI * Z)
    k = 0.5 / (co.Pe * co.Cn)
    psi2 = 3 * c0 ** 2 - 1
    f1 = dphi / co.dt + k * 9 * PI ** 2 * dmu
    f2 = -0.5 * dmu + 0.5 * psi2 * dphi + 0.5 * co.Cn ** 2 * 3 * PI ** 2 * dphi
    sol = solvers.direct(J, np.concatenate([_load(el, f1), _load(el, f2)]))
    return _l2(el, sol[:n], dphi), _l2(el, sol[n:], dmu)


def test_ch_linearised_pair_second_order():
    errs = np.array([_ch_error(L) for L in (2, 3, 4)])
    for c in range(2):
        r = _rates(errs[:, c])
        assert r[-1] > 1.8, (errs, r)


def _momentum_error(level):
    """Velocity prediction at rest (u_hat = 0, J_hat = 0: the RBVMS terms vanish), variable rho
    and eta from phi, one component: (rho/dt) v - (1/(2 Re)) div(eta grad v) = f, v = 0 on the
    walls (reading R19: Laplacian form of the viscous term)."""
    mesh = Mesh(*octree.uniform(level))
    el, co = fem.Elem(mesh), fem.Coeffs(PRM)
    n = mesh.n_nodes
    x = mesh.node_xyz
    phi = _phi(x[:, 0], x[:, 1], x[:, 2])
    vs = fem.VMSState(el, co, phi, np.zeros((3, n)), np.full(n, 0.2))
    A = fem.momentum(vs)
    X, Y, Z = _qp_coords(el)
    v = np.sin(PI * X) * np.sin(PI * Y) * np.sin(PI * Z)
    gv = (PI * np.cos(PI * X) * np.sin(PI * Y) * np.sin(PI * Z),
          PI * np.sin(PI * X) * np.cos(PI * Y) * np.sin(PI * Z),
          PI * np.sin(PI * X) * np.sin(PI * Y) * np.cos(PI * Z))
    ph = _phi(X, Y, Z)
    rho = co.alpha * ph + co.beta
    eta = co.gamma * ph + co.xi
    geta = [co.gamma * g for g in _phi_grad(X, Y, Z)]
    f = rho * v / co.dt - (0.5 / co.Re) * (-3 * PI ** 2 * eta * v + sum(geta[d] * gv[d] for d in range(3)))
    A2, b2 = solvers.dirichlet(A, _load(el, f), mesh.boundary)
    vh = spla.spsolve(A2.tocsc(), b2)
    return _l2(el, vh, v)


def test_momentum_at_rest_second_order():
    errs = [_momentum_error(L) for L in (2, 3, 4)]
    r = _rates(errs)
    assert r[-1] > 1.8, (errs, r)


def test_ch_block_second_order_in_time():
    """The CH block of the step (Crank-Nicolson: phi~, mu~ and psi'(phi~) at the midpoint,
    Def. variational_form_sem_disc) is second order in time: with the fluid at rest and no
    gravity or capillary forcing the velocity stays zero, and the step's phi, mu at T = 0.016
    converge to a dt = 2.5e-4 reference at rate 2 on a fixed mesh (self-convergence)."""
    from oracle import step
    w = configs.smooth_uniform(2, seed=0)
    m = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(m.node_xyz)
    prm = dict(w.params.as_dict(), Fr=1e12, We=1e12)
    z = np.zeros_like(f["u"])
    T, res = 0.016, {}
    for dt in (4e-3, 2e-3, 1e-3, 2.5e-4):
        st = step.State(phi=f["phi"].copy(), mu=f["mu"].copy(), u=z.copy(), u_old=z.copy(),
                        p=f["p"].copy())
        for _ in range(int(round(T / dt))):
            st = step.chns_step(m, dict(prm, dt=dt), st)
        res[dt] = st
    ref = res[2.5e-4]
    assert np.abs(ref.u).max() < 1e-12
    for key in ("phi", "mu"):
        errs = [np.linalg.norm(getattr(res[dt], key) - getattr(ref, key)) for dt in (4e-3, 2e-3, 1e-3)]
        r = _rates(errs)
        assert r.min() > 1.85, (key, errs, r)
