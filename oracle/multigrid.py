"""Oracle geometric multigrid for the pressure-Poisson operator on the octree.

TEST INFRASTRUCTURE ONLY (see the package header).

Not part of the paper's solver stack (PETSc algebraic multigrid, App. A). The paper names a
geometric multigrid on the octree as the remedy for the cost of its AMG setup (Sec. 7,
"Scaling", the component breakdown, and the Conclusions). The pieces below are built from the
paper's octree operations and a standard V-cycle:

* coarsening: every leaf at the finest level is replaced by its parent. This is the one-level
  coarsening of the intergrid transfer (Sec. 5.4, "Traversal-based Intergrid Transfers"). A leaf
  at the finest level always has its seven siblings as leaves, so the parents tile the same
  region and the coarse list is again a complete, 2:1-balanced octree;
* prolongation P (coarse -> fine): the coarse finite-element function, including its hanging
  constraints, evaluated at the fine nodes. This is the child interpolation of Sec. 5.4. Every
  fine node sits on the half-size lattice {0, 1/2, 1}^3 of a coarse leaf, where the trilinear
  weights are products of 1, 1/2 and 0;
* restriction R = P^T;
* level operators: the Poisson operator (grad q, (1/rho(phi~*)) grad p) rediscretised on each
  level, with phi~ injected (a coarse node is always a fine node);
* smoother: `degree` steps of the Chebyshev iteration on D^-1 A (solvers.chebyshev_precond) on
  [lmax / smooth_range, lmax], lmax = lmax_factor x the power estimate of the largest
  eigenvalue of D^-1 A (`power_its` iterations from a fixed start vector, `start_vector`);
* coarsest level: the exact mean-zero solution, (A + 1 1^T / n)^-1 r (pure Neumann);
* the same cycle for the constant-coefficient operator sa (q, p) + sb (grad q, grad p) with
  sa > 0 (the inner operator H of the Cahn-Hilliard Schur-complement preconditioner,
  solvers.ch_schur_precond), whose coarsest level is solved exactly without the 1 1^T term;
* V-cycle: pre-smoothing from zero, residual, restriction, recursion, prolongation, and
  post-smoothing on the new residual with the same polynomial, so that the cycle is a
  symmetric linear operator.

Pins (tests/test_oracle_multigrid.py): the coarse list is a valid balanced octree with the
expected leaf count; P reproduces globally linear fields and agrees with a brute-force point
evaluation of the coarse function; the coarse operator equals the Galerkin product P^T A P for
constant coefficients (exact quadrature, nested spaces); the V-cycle is symmetric, is the exact
solve on a one-level hierarchy, and contracts the error.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .mesh import MAXD, Mesh, _pkey

# 27 points of the half-size lattice of a leaf (x fastest) and the trilinear weights of its 8
# corners there: N_a(xi) = prod_d (1 - xi_d or xi_d) with xi_d in {0, 1/2, 1}
LATTICE = np.array([[i, j, k] for k in range(3) for j in range(3) for i in range(3)],
                   dtype=np.int64)
_XI = LATTICE.astype(np.float64) / 2.0
_BITS = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int64)
LATTICE_W = np.prod(np.where(_BITS[None, :, :] == 1, _XI[:, None, :], 1.0 - _XI[:, None, :]),
                    axis=2)                                        # (27, 8)


def coarsen(anchors, levels):
    """Replace every leaf of the finest level by its parent; Morton order is kept (the parent of
    a run of eight siblings takes the place of the first)."""
    a = np.asarray(anchors, dtype=np.int64)
    lv = np.asarray(levels, dtype=np.int64)
    L = int(lv.max())
    if L == 0:
        raise ValueError("a single root leaf cannot be coarsened")
    fine = lv == L
    side_parent = np.int64(1) << (MAXD - (L - 1))
    pa = a.copy()
    pa[fine] = (a[fine] // side_parent) * side_parent
    pl = lv.copy()
    pl[fine] = L - 1
    # keep the first occurrence of each parent (the sibling with the smallest Morton key comes
    # first in a Morton-ordered list)
    keep = np.ones(len(lv), dtype=bool)
    fi = np.nonzero(fine)[0]
    key = _pkey(pa[fi])
    _, first = np.unique(key, return_index=True)
    drop = np.ones(len(fi), dtype=bool)
    drop[first] = False
    keep[fi[drop]] = False
    return pa[keep], pl[keep]


def hierarchy(anchors, levels, extent=(1.0, 1.0, 1.0), coarsest_level=2):
    """Meshes from the fine one down: coarsen until the finest leaf level is <= coarsest_level."""
    a = np.asarray(anchors, dtype=np.int64)
    lv = np.asarray(levels, dtype=np.int64)
    meshes = [Mesh(a, lv, extent)]
    while int(lv.max()) > coarsest_level:
        a, lv = coarsen(a, lv)
        meshes.append(Mesh(a, lv, extent))
    return meshes


def prolongation(fine: Mesh, coarse: Mesh) -> sp.csr_matrix:
    """P (N_fine x N_coarse): the coarse finite-element function evaluated at the fine nodes.

    For each coarse leaf C and each of its 27 half-size lattice points that is a fine node, the
    value is sum_a N_a(xi) u_C(a), with the corner values u_C(a) taken through the coarse
    mesh's hanging constraints (coarse.P). A fine node on the boundary of several coarse leaves
    takes the row of the first; the coarse function is continuous, so all of them agree (the
    tests check this)."""
    Ec = coarse.n_elem
    half = coarse.side // 2                                           # (Ec,)
    pts = coarse.anchors[:, None, :] + half[:, None, None] * LATTICE[None, :, :]   # (Ec, 27, 3)
    fkey = _pkey(fine.node_int)
    order = np.argsort(fkey)
    skey = fkey[order]
    q = _pkey(pts.reshape(-1, 3))
    pos = np.minimum(np.searchsorted(skey, q), len(skey) - 1)
    hit = skey[pos] == q
    fine_idx = np.where(hit, order[pos], -1)                          # (Ec*27,)
    # rows of (C, k): sum_a W[k, a] e_{corner point a of C}, then through coarse.P
    rows = np.repeat(np.arange(Ec * 27), 8)
    cols = np.repeat(coarse.e2p, 27, axis=0).reshape(-1)
    vals = np.tile(LATTICE_W, (Ec, 1)).reshape(-1)
    T = sp.csr_matrix((vals, (rows, cols)), shape=(Ec * 27, len(coarse.points)))
    Q = (T @ coarse.P).tocsr()                                        # (Ec*27, N_c)
    sel = np.nonzero(hit)[0]
    fi = fine_idx[sel]
    _, first = np.unique(fi, return_index=True)
    if len(first) != fine.n_nodes:
        raise ValueError("a fine node lies on no coarse leaf's half-size lattice")
    S = sp.csr_matrix((np.ones(len(first)), (fi[first], sel[first])), shape=(fine.n_nodes, Ec * 27))
    P = (S @ Q).tocsr()
    P.eliminate_zeros()
    return P


def prolongation_consistency(fine: Mesh, coarse: Mesh) -> float:
    """Largest difference between the rows that different coarse leaves give for the same fine
    node (zero when the coarse function is continuous across leaves)."""
    Ec = coarse.n_elem
    half = coarse.side // 2
    pts = coarse.anchors[:, None, :] + half[:, None, None] * LATTICE[None, :, :]
    fkey = _pkey(fine.node_int)
    order = np.argsort(fkey)
    skey = fkey[order]
    q = _pkey(pts.reshape(-1, 3))
    pos = np.minimum(np.searchsorted(skey, q), len(skey) - 1)
    hit = skey[pos] == q
    rows = np.repeat(np.arange(Ec * 27), 8)
    cols = np.repeat(coarse.e2p, 27, axis=0).reshape(-1)
    vals = np.tile(LATTICE_W, (Ec, 1)).reshape(-1)
    Q = (sp.csr_matrix((vals, (rows, cols)), shape=(Ec * 27, len(coarse.points))) @ coarse.P).tocsr()
    P = prolongation(fine, coarse)
    sel = np.nonzero(hit)[0]
    D = Q[sel] - P[order[pos[sel]]]
    return float(abs(D).max()) if D.nnz else 0.0


def injection(fine: Mesh, coarse: Mesh) -> np.ndarray:
    """Index of the fine node at each coarse node's position."""
    fkey = _pkey(fine.node_int)
    order = np.argsort(fkey)
    skey = fkey[order]
    q = _pkey(coarse.node_int)
    pos = np.minimum(np.searchsorted(skey, q), len(skey) - 1)
    if np.any(skey[pos] != q):
        raise ValueError("a coarse node is not a fine node")
    return order[pos]


def start_vector(n: int) -> np.ndarray:
    """Fixed start of the power iteration: s_i = (i * 2654435761 mod 2^32) / 2^32 - 1/2, in exact
    integer arithmetic (the same values on any machine)."""
    i = np.arange(n, dtype=np.uint64)
    h = (i * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)
    return h.astype(np.float64) / 4294967296.0 - 0.5


def power_lmax(A, dinv, iters):
    """Estimate of the largest eigenvalue of D^-1 A: v <- D^-1 A v / ||D^-1 A v|| from
    v = D^-1 s / ||D^-1 s||; returns the last norm."""
    v = dinv * start_vector(A.shape[0])
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = dinv * (A @ v)
        lam = float(np.linalg.norm(w))
        v = w / lam
    return lam


class VCycle:
    """The V-cycle preconditioner z = B r of the Poisson operator for the coefficient phi~ of
    the fine mesh."""

    def __init__(self, meshes, prm, phi_t=None, degree=3, power_its=12, smooth_range=15.0,
                 lmax_factor=1.1, constant_coefficient=False, shift=None):
        """shift = (sa, sb): the level operators are sa M + sb K instead of the Poisson
        operator with coefficient phi_t."""
        self.meshes = meshes
        self.degree = degree
        co = fem.Coeffs(prm)
        self.P = [prolongation(meshes[l], meshes[l + 1]) for l in range(len(meshes) - 1)]
        self.inj = [injection(meshes[l], meshes[l + 1]) for l in range(len(meshes) - 1)]
        if shift is None:
            phis = [np.asarray(phi_t, dtype=np.float64)]
            for l in range(len(meshes) - 1):
                phis.append(phis[-1][self.inj[l]])
            self.phi = phis
        self.A, self.dinv, self.lmax, self.lmin = [], [], [], []
        for l, m in enumerate(meshes):
            el = fem.Elem(m)
            ones = np.ones((m.n_elem, 8))
            if shift is not None:
                A = shift[0] * fem.mass(el, ones) + shift[1] * fem.stiffness(el, ones)
            elif constant_coefficient:
                A = fem.stiffness(el, ones)
            else:
                A = fem.poisson(el, co, phis[l])
            self.A.append(A.tocsr())
            d = A.diagonal()
            self.dinv.append(1.0 / d)
            lam = power_lmax(A, 1.0 / d, power_its)
            self.lmax.append(lmax_factor * lam)
            self.lmin.append(lmax_factor * lam / smooth_range)
        Ac = self.A[-1].toarray()
        n = Ac.shape[0]
        self.coarse_reg = Ac if shift is not None else Ac + np.full((n, n), 1.0 / n)

    def smooth(self, l, r):
        from .solvers import chebyshev_precond
        return chebyshev_precond(self.A[l], self.dinv[l], r, self.lmin[l], self.lmax[l],
                                 self.degree)

    def cycle(self, l, r):
        if l == len(self.A) - 1:
            return np.linalg.solve(self.coarse_reg, r)
        A = self.A[l]
        z = self.smooth(l, r)
        zc = self.cycle(l + 1, self.P[l].T @ (r - A @ z))
        z = z + self.P[l] @ zc
        return z + self.smooth(l, r - A @ z)

    def __call__(self, r):
        return self.cycle(0, np.asarray(r, dtype=np.float64))


def fcg_mg(A, b, B, rtol=1e-8, maxit=1000, x0=None):
    """Flexible CG (Polak-Ribiere beta) preconditioned by B on the mean-zero Poisson system;
    returns (x, iterations, relative residual)."""
    b = np.asarray(b, dtype=np.float64) - np.mean(b)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = b - A @ x
    r -= r.mean()
    bn = np.linalg.norm(b)
    z = B(r)
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.linalg.norm(r) / bn
    while rel > rtol and it < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r_old = r.copy()
        r = r - alpha * q
        z = B(r)
        beta = (z @ (r - r_old)) / rz
        rz = r @ z
        p = z + beta * p
        it += 1
        rel = np.linalg.norm(r) / bn
    return x - x.mean(), it, rel
