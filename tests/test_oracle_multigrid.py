"""Oracle geometric multigrid pins (oracle/multigrid.py): the coarsening of Sec. 5.4, the
prolongation (child interpolation) and restriction, the level operators and the V-cycle.

Each pin is fixed by something other than the oracle itself: octree validity and leaf counts,
exact reproduction of linear fields, a brute-force point evaluation of the coarse function, the
Galerkin identity P^T A_f P = A_c of nested conforming spaces with exact quadrature, and the
algebraic properties of a symmetric V-cycle. A planted mistake in P (one weight changed) is
shown to break the Galerkin identity."""
import numpy as np
import pytest
import scipy.sparse as sp

from chns_workloads import configs, octree
from chns_workloads.octree import MAXD
from oracle import fem, multigrid as mg
from oracle.mesh import Mesh

PRM = dict(Re=35.0, We=2.0, Cn=0.05, Pe=50.0, Fr=1.0, rho_ratio=20.0, eta_ratio=5.0, dt=1e-3,
           C_I=6.0)


def _trees():
    return {
        "uniform3": octree.uniform(3),
        "random1": configs.random_balanced(1, 2, 5, 0.2),
        "random0": configs.random_balanced(0, 1, 4, 0.3),
        "drop": (lambda w: (w.anchors, w.levels))(configs.rising_drop(3, 5, Cn=0.04)),
    }


TREES = _trees()


@pytest.mark.parametrize("name", list(TREES))
def test_coarsen_gives_balanced_octree(name):
    a, l = TREES[name]
    a = np.asarray(a, dtype=np.int64)
    l = np.asarray(l, dtype=np.int64)
    ac, lc = mg.coarsen(a, l)
    L = l.max()
    n_fine = int(np.sum(l == L))
    assert n_fine % 8 == 0
    assert len(lc) == len(l) - 7 * n_fine // 8
    assert lc.max() == L - 1
    # covering, disjoint, Morton ordered and 2:1 balanced (independent checker of the inputs)
    keys = octree.morton_key(ac)
    assert np.all(np.diff(keys.astype(np.float64)) > 0)
    vol = np.sum((np.int64(1) << (3 * (MAXD - lc))).astype(np.float64))
    assert vol == float(1 << (3 * MAXD))
    assert octree.is_balanced(ac.astype(np.uint32), lc.astype(np.uint8))
    Mesh(ac, lc)  # builds (no chained hanging constraints)


def test_hierarchy_ends_at_coarsest_level():
    a, l = TREES["drop"]
    ms = mg.hierarchy(a, l, coarsest_level=2)
    assert [int(m.levels.max()) for m in ms] == [5, 4, 3, 2]
    assert ms[-1].n_nodes == 125
    assert all(ms[i + 1].n_nodes < ms[i].n_nodes for i in range(len(ms) - 1))


@pytest.mark.parametrize("name", ["random1", "random0", "drop"])
def test_prolongation_reproduces_linear_fields(name):
    a, l = TREES[name]
    ext = (1.0, 2.0, 0.5)
    ms = mg.hierarchy(a, l, ext, coarsest_level=1)
    c = np.array([0.3, -1.2, 0.7, 2.1])
    f = lambda x: c[0] + c[1] * x[:, 0] + c[2] * x[:, 1] + c[3] * x[:, 2]
    for lf in range(len(ms) - 1):
        P = mg.prolongation(ms[lf], ms[lf + 1])
        assert P.shape == (ms[lf].n_nodes, ms[lf + 1].n_nodes)
        assert np.abs(P @ f(ms[lf + 1].node_xyz) - f(ms[lf].node_xyz)).max() < 1e-13
        assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0)
        # weights are dyadic: products of 1, 1/2 and the hanging weights 1/2, 1/4
        assert np.all(P.data * 64.0 == np.round(P.data * 64.0))
        # every coarse leaf gives the same row for a fine node on its boundary (continuity)
        assert mg.prolongation_consistency(ms[lf], ms[lf + 1]) < 1e-15


def _point_value(coarse, uc, x):
    """Brute force: find a coarse leaf whose closed box holds the integer point x and evaluate
    the trilinear interpolant of its corner values (hanging corners through coarse.P)."""
    full = coarse.P @ uc
    lo = coarse.anchors
    hi = lo + coarse.side[:, None]
    inside = np.all((lo <= x) & (x <= hi), axis=1)
    e = np.nonzero(inside)[0][0]
    t = (x - lo[e]) / float(coarse.side[e])
    val = 0.0
    for a in range(8):
        bits = [(a >> d) & 1 for d in range(3)]
        w = np.prod([t[d] if bits[d] else 1.0 - t[d] for d in range(3)])
        val += w * full[coarse.e2p[e, a]]
    return val


def test_prolongation_matches_point_evaluation():
    a, l = TREES["random1"]
    ms = mg.hierarchy(a, l, coarsest_level=1)
    rng = np.random.default_rng(3)
    for lf in range(len(ms) - 1):
        f, c = ms[lf], ms[lf + 1]
        uc = rng.standard_normal(c.n_nodes)
        P = mg.prolongation(f, c)
        got = P @ uc
        idx = rng.choice(f.n_nodes, size=min(200, f.n_nodes), replace=False)
        want = np.array([_point_value(c, uc, f.node_int[i]) for i in idx])
        assert np.abs(got[idx] - want).max() < 1e-13


@pytest.mark.parametrize("name,ext", [("random1", (1.0, 1.0, 1.0)), ("drop", (1.0, 4.0, 1.0))])
def test_galerkin_identity_constant_coefficient(name, ext):
    """V_c is a subspace of V_f and 2x2x2 Gauss is exact for Q1 stiffness and mass on boxes, so
    P^T K_f P = K_c and P^T M_f P = M_c to rounding."""
    a, l = TREES[name]
    ms = mg.hierarchy(a, l, ext, coarsest_level=2)
    for lf in range(len(ms) - 1):
        f, c = ms[lf], ms[lf + 1]
        P = mg.prolongation(f, c)
        ef, ec = fem.Elem(f), fem.Elem(c)
        for op in (fem.stiffness, fem.mass):
            Af = op(ef, np.ones((f.n_elem, 8)))
            Ac = op(ec, np.ones((c.n_elem, 8)))
            G = (P.T @ Af @ P).tocsr()
            assert abs(G - Ac).max() < 1e-12 * abs(Ac).max()


def test_planted_prolongation_error_breaks_galerkin_identity():
    a, l = TREES["random1"]
    ms = mg.hierarchy(a, l, coarsest_level=3)
    f, c = ms[0], ms[1]
    P = mg.prolongation(f, c).tolil()
    i, j = [(i, j) for i, row in enumerate(P.rows) for j in row if P[i, j] == 0.5][0]
    P[i, j] = 0.25  # one half-weight halved
    P = P.tocsr()
    ef, ec = fem.Elem(f), fem.Elem(c)
    Af = fem.stiffness(ef, np.ones((f.n_elem, 8)))
    Ac = fem.stiffness(ec, np.ones((c.n_elem, 8)))
    assert abs((P.T @ Af @ P) - Ac).max() > 1e-3 * abs(Ac).max()


def test_injection_is_the_fine_node_at_the_same_point():
    a, l = TREES["drop"]
    ms = mg.hierarchy(a, l, coarsest_level=2)
    for lf in range(len(ms) - 1):
        inj = mg.injection(ms[lf], ms[lf + 1])
        assert np.array_equal(ms[lf].node_int[inj], ms[lf + 1].node_int)


def test_start_vector_is_exact_integer_hash():
    s = mg.start_vector(5)
    want = [((i * 2654435761) % (1 << 32)) / float(1 << 32) - 0.5 for i in range(5)]
    assert np.array_equal(s, np.array(want))


def test_power_estimate_bounds_spectrum():
    a, l = TREES["random0"]
    m = Mesh(a, l)
    phi = np.tanh(3.0 * (m.node_xyz[:, 0] - 0.4))
    A = fem.poisson(fem.Elem(m), fem.Coeffs(PRM), phi)
    d = A.diagonal()
    lam = mg.power_lmax(A, 1.0 / d, 40)
    Ds = sp.diags(1.0 / np.sqrt(d))
    true = np.linalg.eigvalsh((Ds @ A @ Ds).toarray()).max()
    assert 0.9 * true <= lam <= true * (1 + 1e-12)


def _vcycle(name="drop", ext=(1.0, 1.0, 1.0), coarsest=2, degree=3):
    a, l = TREES[name]
    ms = mg.hierarchy(a, l, ext, coarsest_level=coarsest)
    m = ms[0]
    x = m.node_xyz
    phi = np.tanh((np.linalg.norm(x - 0.5, axis=1) - 0.3) / 0.06)
    return ms, mg.VCycle(ms, PRM, phi, degree=degree)


def test_vcycle_single_level_is_exact_solve():
    a, l = octree.uniform(2)
    ms = mg.hierarchy(a, l, coarsest_level=2)
    assert len(ms) == 1
    phi = np.linspace(-1, 1, ms[0].n_nodes)
    B = mg.VCycle(ms, PRM, phi)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(ms[0].n_nodes)
    r -= r.mean()
    z = B(r)
    assert abs(z.mean()) < 1e-12
    assert np.linalg.norm(B.A[0] @ z - r) < 1e-10 * np.linalg.norm(r)


def test_vcycle_symmetric_and_contracting():
    ms, B = _vcycle()
    A = B.A[0]
    n = ms[0].n_nodes
    rng = np.random.default_rng(1)
    r1, r2 = rng.standard_normal(n), rng.standard_normal(n)
    r1 -= r1.mean()
    r2 -= r2.mean()
    assert abs(r1 @ B(r2) - r2 @ B(r1)) < 1e-10 * abs(r1 @ B(r2))
    # error propagation E = I - B A contracts a mean-free error in the energy norm
    e = rng.standard_normal(n)
    e -= e.mean()
    en = lambda v: np.sqrt(v @ (A @ v))
    e1 = e - B(A @ e)
    assert en(e1) < 0.5 * en(e)


def test_planted_smoother_order_breaks_symmetry():
    """Post-smoothing from zero on the new residual (instead of correcting z) makes the cycle
    non-symmetric: the symmetry pin catches a misplaced smoothing step."""
    ms, B = _vcycle()

    def bad_cycle(l, r):
        if l == len(B.A) - 1:
            return np.linalg.solve(B.coarse_reg, r)
        z = B.smooth(l, r)
        zc = bad_cycle(l + 1, B.P[l].T @ (r - B.A[l] @ z))
        return z + B.P[l] @ zc + 0.5 * B.smooth(l, r)

    n = ms[0].n_nodes
    rng = np.random.default_rng(2)
    r1, r2 = rng.standard_normal(n), rng.standard_normal(n)
    r1 -= r1.mean()
    r2 -= r2.mean()
    sym = abs(r1 @ bad_cycle(0, r2) - r2 @ bad_cycle(0, r1)) / abs(r1 @ bad_cycle(0, r2))
    assert sym > 1e-6


def test_fcg_with_vcycle_solves_and_beats_jacobi():
    from oracle import solvers
    ms, B = _vcycle("drop", (1.0, 4.0, 1.0))
    A = B.A[0]
    n = ms[0].n_nodes
    b = np.random.default_rng(4).standard_normal(n)
    b -= b.mean()
    x, it, rel = mg.fcg_mg(A, b, B, rtol=1e-10)
    xj, itj, _ = solvers.pcg(A, b, rtol=1e-10, mean_zero=True)
    assert rel <= 1e-10
    assert np.linalg.norm(x - xj) <= 1e-7 * np.linalg.norm(xj)
    assert it * 4 < itj


def test_shifted_vcycle_preconditions_h_of_the_schur_preconditioner():
    """For H = M/sqrt(dt) + Cn sqrt(k) K (the inner operator of solvers.ch_schur_precond) the
    cycle is symmetric and CG with it converges in a few iterations, far fewer than Jacobi."""
    from oracle import solvers
    a, l = TREES["drop"]
    ms = mg.hierarchy(a, l, (1.0, 1.0, 1.0), coarsest_level=2)
    Cn, dt = 0.02, 1e-3
    Pe = 1.0 / (3 * Cn ** 2)
    k = 0.5 / (Pe * Cn)
    sa, sb = 1.0 / np.sqrt(dt), Cn * np.sqrt(k)
    B = mg.VCycle(ms, PRM, shift=(sa, sb))
    m = ms[0]
    el = fem.Elem(m)
    ones = np.ones((m.n_elem, 8))
    H = (fem.mass(el, ones) / np.sqrt(dt) + Cn * np.sqrt(k) * fem.stiffness(el, ones)).tocsr()
    assert abs(B.A[0] - H).max() < 1e-14 * abs(H).max()
    rng = np.random.default_rng(3)
    r1, r2 = rng.standard_normal(m.n_nodes), rng.standard_normal(m.n_nodes)
    assert abs(r1 @ B(r2) - r2 @ B(r1)) < 1e-10 * abs(r1 @ B(r2))
    # exact on the coarsest level (no null space: no 1 1^T term)
    Bc = mg.VCycle(ms[-1:], PRM, shift=(sa, sb))
    rc = rng.standard_normal(ms[-1].n_nodes)
    assert np.linalg.norm(Bc.A[0] @ Bc(rc) - rc) < 1e-10 * np.linalg.norm(rc)
    b = rng.standard_normal(m.n_nodes)
    x, it, rel = mg.fcg_mg(H, b - b.mean(), B, rtol=1e-10)
    _, itj, _ = solvers.pcg(H, b - b.mean(), rtol=1e-10)
    assert rel <= 1e-10 and it * 3 < itj
