"""Pins of the learned-preconditioner oracle: gradients by central finite differences, layer
identities and adjointness, and the properties of the grid transfer."""
import numpy as np
import pytest

from chns_workloads import configs
from oracle import learned as L
from oracle.mesh import Mesh


def _net(D=8, C=4, seed=0):
    P = L.init_params(C=C, seed=seed)
    rng = np.random.default_rng(seed + 1)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    x = rng.standard_normal((2, D, D, D))
    t = rng.standard_normal((D, D, D))
    return P, x, t


def test_backward_matches_finite_differences():
    P, x, t = _net()
    out, cache = L.forward(P, x)
    _, g = L.loss_and_grad(out, t)
    G = L.backward(P, cache, g)
    rng = np.random.default_rng(3)
    eps = 1e-6
    for k in P:
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in P[k].shape)
            old = P[k][idx]
            P[k][idx] = old + eps
            lp, _ = L.loss_and_grad(L.forward(P, x)[0], t)
            P[k][idx] = old - eps
            lm, _ = L.loss_and_grad(L.forward(P, x)[0], t)
            P[k][idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - G[k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, G[k][idx])


def test_delta_kernel_is_identity_and_shift():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 6, 6, 6))
    W = np.zeros((27, 3, 3))
    W[L.TAPS.index((0, 0, 0))] = np.eye(3)
    assert np.allclose(L.conv3(x, W, np.zeros(3)), x)
    W = np.zeros((27, 3, 3))
    W[L.TAPS.index((1, 0, 0))] = np.eye(3)          # y(x) = x(x + 1) with zero padding
    y = L.conv3(x, W, np.zeros(3))
    assert np.allclose(y[:, :, :, :-1], x[:, :, :, 1:]) and np.allclose(y[:, :, :, -1], 0)


def test_pool_up_adjoint():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 8, 8, 8))
    b = rng.standard_normal((2, 4, 4, 4))
    assert np.isclose(np.sum(L.pool(a) * b), np.sum(a * L.pool_backward(b)))
    assert np.isclose(np.sum(L.up(b) * a), np.sum(b * L.up_backward(a)))
    assert np.allclose(L.pool(np.ones((1, 4, 4, 4))), 1.0)


@pytest.mark.parametrize("D", [4, 8])
def test_grid_transfer(D):
    a, l = configs.random_balanced(2, 1, 4, 0.3)
    m = Mesh(a, l)
    Pg = L.grid_prolongation(m.node_int, m.extent, D)
    assert np.allclose(Pg.sum(axis=1), 1.0)                 # partition of unity
    # exact for fields linear in each coordinate between the outermost cell centres
    c = (np.arange(D) + 0.5) / D
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    f = lambda x, y, z: 0.3 + x - 2 * y + 0.5 * z
    xyz = m.node_xyz
    inner = np.all((xyz >= c[0]) & (xyz <= c[-1]), axis=1)
    got = Pg @ f(xx, yy, zz).ravel()
    assert np.abs(got[inner] - f(*xyz[inner].T)).max() < 1e-12
    # restriction is the adjoint
    r = np.random.default_rng(0).standard_normal(m.n_nodes)
    g = np.random.default_rng(1).standard_normal(D ** 3)
    assert np.isclose((Pg.T @ r) @ g, r @ (Pg @ g))


def test_bf16_round_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    a = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 8, 1000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, 65504.0]])
    ref = torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16_round(a), ref)
    # ties go to the even neighbour
    assert L.bf16_round(1.0 + 2.0 ** -8) == 1.0 and L.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_flatten_roundtrip():
    P = L.init_params(C=16, seed=2)
    v = L.flatten(P)
    assert len(v) == 27 * 16 * 2 + 16 + 6 * (27 * 256 + 16) + 17
    Q = L.unflatten(v)
    assert all(np.array_equal(P[k], Q[k]) for k in P)


def _mesh_and_grid(D=8):
    a, l = configs.random_balanced(3, 1, 4, 0.3)
    m = Mesh(a, l)
    return m, L.grid_prolongation(m.node_int, m.extent, D)


def test_constant_network_gives_scaled_constant_correction():
    """All conv weights and biases zero, out.b = c: out = c everywhere, so the correction is
    s(r) * out_scale * c at every node (P_g has unit row sums)."""
    D = 8
    m, Pg = _mesh_and_grid(D)
    P = L.init_params(C=4, seed=0)
    for k in P:
        P[k] = np.zeros_like(P[k])
    P["out.b"] = np.array([0.7])
    r = np.random.default_rng(0).standard_normal(m.n_nodes)
    lr = np.zeros((D, D, D))
    c = L.coarse_correction(P, Pg, r, lr, D, 3.0)
    s = np.sqrt(r @ r / D ** 3)
    assert np.allclose(c, s * 3.0 * 0.7, rtol=1e-13)


def test_correction_is_positively_homogeneous_and_zero_net_gives_jacobi():
    D = 8
    m, Pg = _mesh_and_grid(D)
    P, _, _ = _net(D=D, C=4, seed=4)
    rng = np.random.default_rng(1)
    r = rng.standard_normal(m.n_nodes)
    lr = rng.standard_normal((D, D, D))
    c1 = L.coarse_correction(P, Pg, r, lr, D, 2.0)
    c2 = L.coarse_correction(P, Pg, 3.5 * r, lr, D, 2.0)
    assert np.allclose(c2, 3.5 * c1, rtol=1e-12, atol=0)
    assert np.array_equal(L.coarse_correction(P, Pg, 0 * r, lr, D, 2.0), np.zeros(m.n_nodes))
    Z = {k: np.zeros_like(v) for k, v in P.items()}
    dinv = rng.uniform(0.5, 2.0, m.n_nodes)
    A = np.eye(m.n_nodes) * 3.0
    assert np.allclose(L.precondition(Z, Pg, A, r, lr, D, 2.0, dinv), (2.0 / 3.0) * dinv * r,
                       rtol=1e-15, atol=0)
    # with a network, the Jacobi step acts on what the correction leaves
    z = L.precondition(P, Pg, A, r, lr, D, 2.0, dinv, omega=0.5)
    assert np.allclose(z, c1 + 0.5 * dinv * (r - 3.0 * c1), rtol=1e-12)


def test_training_target_of_constant_error():
    """Constants are the Poisson null space: a constant error gives a zero target, adding one
    changes nothing; the cell mean of a constant is that constant where nodes reach."""
    D = 8
    m, Pg = _mesh_and_grid(D)
    n = m.n_nodes
    reached = (Pg.T @ np.ones(n)).reshape(D, D, D) > 0
    cm = L.cell_mean(Pg, np.full(n, 2.5), D)
    assert np.allclose(cm[reached], 2.5) and np.all(cm[~reached] == 0)
    assert np.allclose(L.training_target(Pg, np.full(n, 2.5), 0.5, D), 0.0, atol=1e-14)
    e = np.random.default_rng(0).standard_normal(n)
    t = L.training_target(Pg, e, 0.5, D)
    assert np.allclose(L.training_target(Pg, e + 7.0, 0.5, D), t, atol=1e-12)
    assert np.allclose(L.training_target(Pg, 3.0 * e, 1.5, D), t, atol=1e-12)
    assert np.allclose(t, L.cell_mean(Pg, e - e.mean(), D) / 0.5)


def test_fcg_with_fixed_preconditioner_equals_pcg():
    """With a fixed SPD preconditioner the Polak-Ribiere beta equals Fletcher-Reeves (r_new is
    M-orthogonal to r_old), so flexible CG reproduces Jacobi-PCG."""
    from oracle import fem, solvers
    a, l = configs.random_balanced(2, 1, 4, 0.3)
    m = Mesh(a, l)
    co = fem.Coeffs(dict(Re=1, We=1, Cn=0.1, Pe=1, Fr=1, rho_ratio=10.0, eta_ratio=1.0, dt=1.0,
                         C_I=6.0))
    phi = np.tanh(3 * np.random.default_rng(0).standard_normal(m.n_nodes))
    A = fem.poisson(fem.Elem(m), co, phi) + 1e-3 * fem.mass(fem.Elem(m), np.ones((m.n_elem, 8)))
    b = np.random.default_rng(1).standard_normal(m.n_nodes)
    dinv = 1.0 / A.diagonal()
    x1, it1, _ = solvers.pcg(A, b, rtol=1e-10)
    x2, it2, _ = L.fcg(A, b, lambda r: dinv * r, rtol=1e-10)
    assert abs(it1 - it2) <= 1 and np.allclose(x1, x2, rtol=0, atol=1e-8 * np.abs(x1).max())


def test_energy_loss_gradient_matches_finite_differences():
    """dL/d(out) of the energy loss against central differences through a linear output layer:
    perturbing out.b by t shifts out by t everywhere, so dL/d(out.b) = sum of dL/d(out)."""
    from oracle import fem
    D = 8
    m, Pg = _mesh_and_grid(D)
    co = fem.Coeffs(dict(Re=1, We=1, Cn=0.1, Pe=1, Fr=1, rho_ratio=10.0, eta_ratio=1.0, dt=1.0,
                         C_I=6.0))
    rng = np.random.default_rng(3)
    A = fem.poisson(fem.Elem(m), co, np.tanh(rng.standard_normal(m.n_nodes)))
    e = rng.standard_normal(m.n_nodes)
    e -= e.mean()
    P, x, _ = _net(D=D, C=4, seed=6)
    loss, gout, _ = L.energy_loss_and_grad(P, Pg, A, e, x, 0.7, D, 1.3)
    eps = 1e-6
    P["out.b"] = P["out.b"] + eps
    lp = L.energy_loss_and_grad(P, Pg, A, e, x, 0.7, D, 1.3)[0]
    P["out.b"] = P["out.b"] - 2 * eps
    lm = L.energy_loss_and_grad(P, Pg, A, e, x, 0.7, D, 1.3)[0]
    assert abs((lp - lm) / (2 * eps) - gout.sum()) <= 1e-6 * max(1.0, abs(gout.sum()))
    Z = {k: np.zeros_like(v) for k, v in P.items()}
    assert np.isclose(L.energy_loss_and_grad(Z, Pg, A, e, x, 0.7, D, 1.3)[0], 1.0, rtol=1e-13)
