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
