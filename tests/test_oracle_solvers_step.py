"""Oracle solver and time-step pins: PCG vs LU, Dirichlet elimination, mass conservation
(Prop. mass_conservation) and energy decay (Sec. 3 energy law) over full steps."""
import numpy as np
import pytest
import scipy.sparse as sp

from chns_workloads import configs
from oracle import fem, solvers, step
from oracle.mesh import Mesh


def test_pcg_matches_lu():
    a, l = configs.random_balanced(0, 1, 4, 0.3)
    m = Mesh(a, l)
    el = fem.Elem(m)
    co = fem.Coeffs(dict(Re=1, We=1, Cn=0.1, Pe=1, Fr=1, rho_ratio=100, eta_ratio=1, dt=1,
                         C_I=6))
    rng = np.random.default_rng(0)
    A = fem.poisson(el, co, np.tanh(3 * rng.standard_normal(m.n_nodes)))
    b = rng.standard_normal(m.n_nodes)
    x, it, rel = solvers.pcg(A, b, rtol=1e-13, mean_zero=True)
    assert rel <= 1e-13
    # reference: pin node 0 and solve the reduced nonsingular system with LU
    bb = b - b.mean()
    Ar = A[1:, 1:]
    xr = np.concatenate([[0.0], solvers.direct(Ar, bb[1:])])
    xr -= xr.mean()
    assert np.abs(x - xr).max() < 1e-9 * np.abs(xr).max()


def test_dirichlet_elimination():
    rng = np.random.default_rng(1)
    n = 30
    B = sp.random(n, n, density=0.3, random_state=1) + 10 * sp.eye(n)
    mask = np.zeros(n, dtype=bool)
    mask[[0, 5, 7]] = True
    g = rng.standard_normal(n)
    b = rng.standard_normal(n)
    A2, b2 = solvers.dirichlet(B, b, mask, g)
    x = solvers.direct(A2, b2)
    assert np.allclose(x[mask], g[mask])
    f = ~mask
    Bd = B.toarray()
    xf = np.linalg.solve(Bd[np.ix_(f, f)], b[f] - Bd[np.ix_(f, mask)] @ g[mask])
    assert np.allclose(x[f], xf)


def _run(w, nsteps):
    m = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(m.node_xyz)
    st = step.State(phi=f["phi"], mu=f["mu"], u=f["u"], u_old=f["u"], p=f["p"])
    el, co = fem.Elem(m), fem.Coeffs(w.params.as_dict())
    masses, energies, logs = [fem.phi_mass(el, st.phi)], [fem.energy(el, co, st.phi, st.u)], []
    for _ in range(nsteps):
        log = []
        st = step.chns_step(m, w.params.as_dict(), st, log=log)
        masses.append(fem.phi_mass(el, st.phi))
        energies.append(fem.energy(el, co, st.phi, st.u))
        logs.append(log)
    return m, st, np.array(masses), np.array(energies), logs


def test_step_conserves_mass_and_dissipates_energy():
    w = configs.smooth_uniform(3, seed=0)
    m, st, ms, es, logs = _run(w, 3)
    # the paper sees ~1e-7..1e-8 drift with iterative solvers; with direct solves it is rounding
    assert np.abs(ms - ms[0]).max() < 1e-12
    assert np.all(np.diff(es) < 0)
    # Newton converges in at most two iterations at this time step (Sec. 6.2)
    assert all(b["newton_its"] <= 2 for lg in logs for b in lg)
    # velocity stays zero on the boundary, pressure has mean zero
    assert np.abs(st.u[:, m.boundary]).max() == 0.0
    assert abs(st.p.mean()) < 1e-12


@pytest.mark.slow
def test_step_on_adaptive_drop_mesh():
    w = configs.rising_drop(3, 5, Cn=0.04)
    m, st, ms, es, logs = _run(w, 1)
    assert m.n_hanging > 0
    assert abs(ms[1] - ms[0]) < 1e-12


def test_chebyshev_preconditioner_is_the_scaled_chebyshev_polynomial():
    """On an eigenvector v of A (D = I) with eigenvalue lam, k steps give z = p(lam) v with
    1 - lam p(lam) = T_k((theta - lam) / delta) / T_k(theta / delta) (library Chebyshev T_k)."""
    from numpy.polynomial import chebyshev as C
    from oracle.solvers import chebyshev_precond
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lams = np.linspace(0.05, 2.0, 12)
    A = Q @ np.diag(lams) @ Q.T
    lmin, lmax = 0.1, 2.2
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    for k in (1, 2, 3, 5):
        for j in (0, 4, 11):
            v = Q[:, j]
            z = chebyshev_precond(A, np.ones(12), v, lmin, lmax, k)
            Tk = lambda t: C.chebval(t, [0] * k + [1])
            p = (1.0 - Tk((theta - lams[j]) / delta) / Tk(theta / delta)) / lams[j]
            assert np.allclose(z, p * v, rtol=1e-12, atol=1e-14), (k, j)


_CH_PRM = dict(Re=35.0, We=2.0, Cn=0.05, Pe=50.0, Fr=1.0, rho_ratio=20.0, eta_ratio=5.0,
               dt=1e-3, C_I=6.0)


def _ch_system(level, prm, seed):
    from chns_workloads import octree
    a, l = octree.uniform(level)
    om = Mesh(a, l, (1.0, 1.0, 1.0))
    el, co = fem.Elem(om), fem.Coeffs(prm)
    rng = np.random.default_rng(seed)
    n = om.n_nodes
    phi = np.tanh(1.5 * rng.standard_normal(n))
    u = 0.3 * rng.standard_normal((3, n))
    J = fem.ch_jacobian(el, co, phi, u)
    ones = np.ones((om.n_elem, 8))
    return n, J.tocsr(), fem.mass(el, ones).tocsr(), fem.stiffness(el, ones).tocsr()


def test_schur_preconditioner_blocks_and_exact_factor():
    """The preconditioner's reading of the CH Jacobian (B = K/(2 Pe Cn), D = -M/2) is the oracle's
    Jacobian, and with the exact Schur complement S = A - B D^-1 C in place of H M^-1 H,
    J P^-1 - I is nilpotent of index 2 (J P^-1 is similar to a unit block-lower-triangular
    matrix), so a sign or scale error in B, D or the factor order breaks the identity."""
    n, J, M, K = _ch_system(2, _CH_PRM, 5)
    k = 0.5 / (_CH_PRM["Pe"] * _CH_PRM["Cn"])
    Jd = J.toarray()
    A, B, C, D = Jd[:n, :n], Jd[:n, n:], Jd[n:, :n], Jd[n:, n:]
    assert np.allclose(B, k * K.toarray(), rtol=0, atol=1e-14 * np.abs(B).max())
    assert np.allclose(D, -0.5 * M.toarray(), rtol=0, atol=1e-14 * np.abs(D).max())
    S = A - B @ np.linalg.solve(D, C)
    s_inv = lambda t: np.linalg.solve(S, t)
    P_inv = np.column_stack([
        solvers.ch_schur_precond(M, K, _CH_PRM["dt"], _CH_PRM["Pe"], _CH_PRM["Cn"], e, s_inv)
        for e in np.eye(2 * n)])
    E = Jd @ P_inv - np.eye(2 * n)
    assert np.linalg.norm(E) > 1e-3                    # the factor is not the inverse ...
    assert np.linalg.norm(E @ E) <= 1e-9 * max(1.0, np.linalg.norm(E) ** 2)  # ... but E^2 = 0


def test_schur_preconditioner_where_the_biharmonic_term_dominates():
    """With H M^-1 H for S and exact inner inverses, GMRES on the CH Newton system of a 16^3 mesh
    with Cn = 0.02, Pe = 1/(3 Cn^2), dt = 2e-2 needs far fewer iterations than with the inverse
    2x2 nodal blocks, and reaches the same solution."""
    import scipy.sparse.linalg as spla
    prm = dict(_CH_PRM, Cn=0.02, Pe=1.0 / (3 * 0.02 ** 2), dt=2e-2)
    n, J, M, K = _ch_system(4, prm, 6)
    b = np.random.default_rng(7).standard_normal(2 * n)
    ref = spla.spsolve(J.tocsc(), b)
    schur = spla.LinearOperator(
        J.shape, matvec=lambda r: solvers.ch_schur_precond(M, K, prm["dt"], prm["Pe"], prm["Cn"], r))
    Jd = J.tocsr()
    diag = Jd.diagonal()
    app, amm, apm, amp = diag[:n], diag[n:], Jd.diagonal(n), Jd.diagonal(-n)
    det = app * amm - apm * amp

    def bj(r):
        x, y = r[:n], r[n:]
        return np.concatenate([(amm * x - apm * y) / det, (-amp * x + app * y) / det])

    jac = spla.LinearOperator(J.shape, matvec=bj)
    its = {}
    for name, P in (("schur", schur), ("block_jacobi", jac)):
        count = [0]
        x, info = spla.gmres(J, b, M=P, rtol=1e-10, restart=30, maxiter=100,
                             callback=lambda _: count.__setitem__(0, count[0] + 1),
                             callback_type="pr_norm")
        its[name] = (count[0], info, np.linalg.norm(x - ref) / np.linalg.norm(ref))
    assert its["schur"][1] == 0 and its["schur"][2] < 1e-7, its
    assert 2 * its["schur"][0] < its["block_jacobi"][0], its  # 28 against 103 here
