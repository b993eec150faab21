"""Temporal order of the oracle's coupled two-block step (oracle/step.py), pinned by manufactured
solutions in the manner of Sec. 6.1 (the residual of a chosen solution is put on the right-hand
sides as a body force), and the paper's Newton behaviour (Sec. 6.2).

The chosen solution lies in the discrete space: a linear, divergence-free velocity with its own
Dirichlet data, a linear pressure and a uniform phase. The Q1 interpolants then reproduce every
spatial term, the strong residual R_m of the RBVMS closure vanishes up to time-discretisation
errors, and the error against the exact solution is the error of the time scheme alone. The
paper reports second order for the velocity and first order for the pressure (Sec. 6.1). Two
plausible mistakes planted in the oracle on the CPU (the printed "+" in the extrapolation
(3u^k + u^{k-1})/2, and the previous pressure p^k dropped from the velocity prediction) break
these pins.

A second test records why the smooth manufactured solution of Sec. 6.1 cannot pin the order on
the coarse meshes the CPU oracle solves: Q1 drops the second derivatives of R_m (reading R8), and
the boxed RBVMS term of the pressure Poisson equation multiplies R_m by 2 tau_m / dt, which tends
to 1 as dt -> 0 at fixed h (tau_m -> dt/2). The error then grows as dt shrinks; on the paper's
512 x 512 mesh tau_m << dt and the term is negligible.
"""
import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

from chns_workloads import configs, octree  # noqa: E402
from oracle import fem, step as ostep  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402

S = sympy
x, y, z, t = S.symbols("x y z t", real=True)
X = (x, y, z)
GHAT = (0, -1, 0)


def _forcing_and_exact(prm, v, p, phi, mu):
    """Body forces of the strong equations (Sec. 3, with p standing for p/We as in reading R3)
    for the exact fields, and the exact fields themselves, as numpy callables."""
    co = fem.Coeffs(prm)
    rho = co.alpha * phi + co.beta
    eta = co.gamma * phi + co.xi
    J = [-(co.alpha / co.Cn) * S.diff(mu, X[j]) for j in range(3)]
    lap = lambda f: sum(S.diff(f, X[j], 2) for j in range(3))
    fv = []
    for i in range(3):
        e = rho * (S.diff(v[i], t) + sum(v[j] * S.diff(v[i], X[j]) for j in range(3)))
        e += (1 / co.Pe) * sum(J[j] * S.diff(v[i], X[j]) for j in range(3))
        e += (co.Cn / co.We) * sum(S.diff(S.diff(phi, X[i]) * S.diff(phi, X[j]), X[j])
                                  for j in range(3))
        e += S.diff(p, X[i])
        e -= (1 / co.Re) * sum(S.diff(eta * S.diff(v[i], X[j]), X[j]) for j in range(3))
        e -= rho * GHAT[i] / co.Fr
        fv.append(e)
    fphi = S.diff(phi, t) + sum(S.diff(v[j] * phi, X[j]) for j in range(3)) - lap(mu) / (co.Pe * co.Cn)
    fmu = mu - (phi ** 3 - phi) + co.Cn ** 2 * lap(phi)
    F = S.lambdify((x, y, z, t), [fv[0], fv[1], fv[2], fphi, fmu], "numpy")
    E = S.lambdify((x, y, z, t), [v[0], v[1], v[2], p, phi, mu], "numpy")

    def bcast(vals, shape):
        return [np.broadcast_to(np.asarray(a, dtype=np.float64), shape) for a in vals]

    def forcing(xq, tt):
        r = bcast(F(xq[..., 0], xq[..., 1], xq[..., 2], tt), xq.shape[:-1])
        return dict(f_v=np.stack(r[:3], axis=-1), f_phi=r[3], f_mu=r[4])

    def exact(xx, tt):
        r = bcast(E(xx[:, 0], xx[:, 1], xx[:, 2], tt), (len(xx),))
        return dict(u=np.stack(r[:3]), p=r[3], phi=r[4], mu=r[5])

    return forcing, exact


def _run(m, prm, forcing, exact, n, T, dirichlet, plus_extrapolation=False):
    dt = T / n
    pr = dict(prm, dt=dt)
    e0 = exact(m.node_xyz, 0.0)
    st = ostep.State(phi=e0["phi"].copy(), mu=e0["mu"].copy(), u=e0["u"].copy(),
                     u_old=exact(m.node_xyz, -dt)["u"], p=e0["p"].copy())
    bc = (lambda xx, tt: exact(xx, tt)["u"]) if dirichlet else None
    for k in range(n):
        if plus_extrapolation:  # (3 u^k - (-u^{k-1})) / 2 = the printed (3 u^k + u^{k-1}) / 2
            st = ostep.State(phi=st.phi, mu=st.mu, u=st.u, u_old=-st.u_old, p=st.p)
        st = ostep.chns_step(m, pr, st, forcing=forcing, t=k * dt, velocity_bc=bc)
    return st


def _err(st, ex, key):
    a, b = getattr(st, key), ex[key]
    if key == "p":
        a, b = a - a.mean(), b - b.mean()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


PRM = dict(Re=10.0, We=1.0, Cn=1.0, Pe=3.0, Fr=1.0, rho_ratio=1 / 0.85, eta_ratio=2.0, dt=0.1,
           C_I=6.0)  # the paper's manufactured-solution groups (Sec. 6.1), density ratio 0.85


def _in_space_case():
    s = S.sin(2 * t) + S.Rational(1, 2)
    v = [(x - S.Rational(1, 2)) * s, -(y - S.Rational(1, 2)) * s, S.Integer(0)]
    p = (x - S.Rational(1, 2) + 2 * (z - S.Rational(1, 2))) * S.cos(3 * t)
    return _forcing_and_exact(PRM, v, p, S.Integer(0), S.Integer(0))


def _errors(ns=(8, 16, 32), **kw):
    a, l = octree.uniform(2)
    m = Mesh(a, l)
    forcing, exact = _in_space_case()
    T = 0.5
    ex = exact(m.node_xyz, T)
    out = []
    for n in ns:
        st = _run(m, PRM, forcing, exact, n, T, dirichlet=True, **kw)
        out.append({k: _err(st, ex, k) for k in ("u", "p")})
    return out


def test_coupled_step_is_second_order_in_velocity_first_in_pressure():
    e = _errors()
    ru = [np.log2(e[i]["u"] / e[i + 1]["u"]) for i in range(2)]
    rp = [np.log2(e[i]["p"] / e[i + 1]["p"]) for i in range(2)]
    assert min(ru) > 1.7, ru
    assert min(rp) > 0.9, rp
    assert e[-1]["u"] < 1e-3 and e[-1]["p"] < 0.1


def test_planted_plus_extrapolation_is_caught():
    e = _errors(plus_extrapolation=True)
    assert e[-1]["p"] > 0.5  # the pressure no longer converges to the exact one


def test_planted_missing_previous_pressure_is_caught(monkeypatch):
    orig = fem.vp_rhs
    monkeypatch.setattr(fem, "vp_rhs", lambda vs, u_k, p_k: orig(vs, u_k, 0.0 * p_k))
    e = _errors()
    ru = [np.log2(e[i]["u"] / e[i + 1]["u"]) for i in range(2)]
    assert max(ru) < 1.4, ru  # first order: the non-incremental projection


def test_smooth_solution_on_a_coarse_mesh_shows_the_small_dt_inconsistency():
    """Sec. 6.1's solution (made zero on the z faces so that no-slip holds) on h = 1/4: the
    pressure error against the exact solution grows as dt shrinks, because the boxed term of the
    pressure Poisson equation approaches -(grad q, R_m / rho) with R_m(exact) = O(1) (the
    second derivatives Q1 drops) when tau_m -> dt/2."""
    g = S.sin(S.pi * z) ** 2
    v = [S.pi * S.sin(S.pi * x) ** 2 * S.sin(2 * S.pi * y) * g * S.sin(t),
         -S.pi * S.sin(2 * S.pi * x) * S.sin(S.pi * y) ** 2 * g * S.sin(t), S.Integer(0)]
    p = S.cos(S.pi * x) * S.sin(S.pi * y) * S.sin(t)
    phi = S.cos(S.pi * x) * S.cos(S.pi * y) * S.sin(t)
    forcing, exact = _forcing_and_exact(PRM, v, p, phi, phi)
    a, l = octree.uniform(2)
    m = Mesh(a, l)
    T = 1.0
    ex = exact(m.node_xyz, T)
    ep = [_err(_run(m, PRM, forcing, exact, n, T, dirichlet=False), ex, "p") for n in (4, 32)]
    assert ep[1] > 1.5 * ep[0] and ep[1] > 1.0, ep
    # tau_m at the finest step is close to dt/2: 2 tau_m / dt above 0.5 everywhere
    el, co = fem.Elem(m), fem.Coeffs(dict(PRM, dt=T / 32))
    vs = fem.VMSState(el, co, np.zeros(m.n_nodes), np.zeros((3, m.n_nodes)), np.zeros(m.n_nodes))
    assert np.min(2.0 * vs.tau / co.dt) > 0.5


def test_newton_converges_in_one_iteration_at_the_paper_tolerance():
    """Sec. 6.2: at the time steps used, the CH Newton iteration converges in a single step. With
    the relative tolerance 1e-6 the exact Newton of the oracle needs one iteration in every block
    after the first step's first block (which relaxes the initial chemical potential), and at
    most two at 1e-10."""
    w = configs.rising_drop(3, 5, Cn=0.04)
    m = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(m.node_xyz)
    for tol, bound_first, bound_rest in ((1e-6, 2, 1), (1e-10, 2, 2)):
        st = ostep.State(phi=f["phi"], mu=f["mu"], u=f["u"], u_old=f["u"], p=f["p"])
        its = []
        for _ in range(2):
            log = []
            st = ostep.chns_step(m, w.params.as_dict(), st, newton_rtol=tol, log=log)
            its += [b["newton_its"] for b in log]
        assert its[0] <= bound_first and max(its[1:]) <= bound_rest, (tol, its)


def test_planted_missing_advection_in_the_closure_residual_is_caught(monkeypatch):
    """R_m enters the velocity prediction, the pressure Poisson and the velocity update right-hand
    sides through the RBVMS closure; without its advection term it no longer vanishes at the
    exact solution and the velocity loses its second order."""
    orig = fem.VMSState.residual_m

    def no_advection(self, v, u_k, p_k):
        out = orig(self, v, u_k, p_k)
        vt = 0.5 * (v + u_k)
        for i in range(3):
            out[..., i] -= self.rho * np.sum(self.uh * self.el.grad(vt[i]), axis=-1)
        return out

    monkeypatch.setattr(fem.VMSState, "residual_m", no_advection)
    e = _errors()
    ru = [np.log2(e[i]["u"] / e[i + 1]["u"]) for i in range(2)]
    assert max(ru) < 1.2, ru
    assert e[-1]["p"] > 0.5
