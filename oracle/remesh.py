"""Oracle adaptive remeshing and intergrid transfer on the octree.

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 5.4 ("Traversal-based Intergrid Transfers") changes the mesh locally by one level at most
per remesh and moves the fields from the current mesh A to the new mesh B in three cases: a
leaf of both meshes copies its values, a leaf of A refined in B gives its children the values of
its own shape functions at their nodes, and leaves of A coarsened in B give their parent its
corner values. The scaling runs (Sec. 7) refine the band |phi| <= 0.95 around the interface and
coarsen away from it. Written out here:

* ``flags``: the band test of a leaf uses the finite-element phase phi_h of A at the leaf's 8
  corners and its centre (the 9 points of the initial refinement, reading R21): the leaf is in
  the band when the smallest |phi_h| there is <= threshold. In the band and below ``lmax`` it is
  flagged for refinement (+1); out of the band and above ``lmin`` it is a coarsening candidate
  (-1); otherwise 0.
* ``new_leaves``: a +1 leaf is replaced by its 8 children; the 8 children of one parent, all
  leaves and all flagged -1, are replaced by the parent; the other leaves stay. The list is then
  made 2:1 balanced by splitting leaves that touch a leaf more than one level finer, until none
  does (the unique coarsest balanced refinement), and sorted in Morton order.
* ``transfer``: the value at every node of B is the finite-element function of A (hanging
  constraints included) evaluated at the node's position, by locating a leaf of A that contains
  it and evaluating that leaf's trilinear interpolant. The function is continuous, so any leaf
  containing the point gives the same value. This is each of the three cases above: at a node
  of a copied leaf the point is a node of A; at a child node it is the parent's shape functions;
  the corners of a coarsened parent are nodes of A, so the parent takes A's values there (the
  "projection" of coarsened leaves read as this nodal injection, which is why the paper finds
  the coarsening transfer not mass conserving, Sec. 6.2).

Pins (tests/test_oracle_remesh.py): flags of a linear phase against the closed form of its
9-point minimum; the new list is a valid balanced octree, equal to the input generators'
independent ripple balance, with the expected leaf counts on uniform trees; the transfer
reproduces linear fields, is the identity at nodes shared by A and B (a refine-then-coarsen round
trip returns the original values exactly), and equals the multigrid oracle's prolongation, built
from lattice points instead of point location, when B is A with its finest level refined.
"""
from __future__ import annotations

import numpy as np

from .mesh import CORNER_BITS, MAXD, Mesh, _morton


def phase_at_corners_and_centre(mesh: Mesh, phi: np.ndarray) -> np.ndarray:
    """(E, 9) values of phi_h at each leaf's 8 corners (through the hanging constraints) and at
    its centre (the trilinear interpolant there is the mean of the corner values)."""
    ue = mesh.element_values(phi)
    return np.concatenate([ue, ue.mean(axis=1, keepdims=True)], axis=1)


def flags(mesh: Mesh, phi: np.ndarray, threshold: float, lmin: int, lmax: int) -> np.ndarray:
    v = np.abs(phase_at_corners_and_centre(mesh, phi)).min(axis=1)
    band = v <= threshold
    out = np.zeros(mesh.n_elem, dtype=np.int8)
    out[band & (mesh.levels < lmax)] = 1
    out[~band & (mesh.levels > lmin)] = -1
    return out


def _children(anchor, level):
    half = np.int64(1) << np.int64(MAXD - level - 1)
    return [anchor + half * CORNER_BITS[c] for c in range(8)]


def _touch_violations(a, lv):
    """Indices of leaves that touch (closed boxes intersect) a leaf more than one level finer."""
    side = np.int64(1) << (MAXD - lv)
    lo, hi = a, a + side[:, None]
    bad = []
    for i in range(len(lv)):
        touch = np.all((lo <= hi[i]) & (hi >= lo[i]), axis=1)
        if np.any(lv[touch] > lv[i] + 1):
            bad.append(i)
    return bad


def balance(anchors, levels):
    """Split leaves touching a leaf more than one level finer until the list is 2:1 balanced
    (brute force over all pairs; small meshes only). Returns Morton-sorted leaves."""
    a = [np.asarray(x, dtype=np.int64) for x in np.asarray(anchors, dtype=np.int64)]
    lv = list(np.asarray(levels, dtype=np.int64))
    while True:
        A, L = np.array(a), np.array(lv)
        bad = set(_touch_violations(A, L))
        if not bad:
            break
        a2, l2 = [], []
        for i in range(len(L)):
            if i in bad:
                a2 += _children(A[i], L[i])
                l2 += [L[i] + 1] * 8
            else:
                a2.append(A[i])
                l2.append(L[i])
        a, lv = a2, l2
    A, L = np.array(a, dtype=np.int64), np.array(lv, dtype=np.int64)
    order = np.argsort(_morton(A), kind="stable")
    return A[order], L[order]


def new_leaves(mesh: Mesh, fl: np.ndarray):
    a, lv = mesh.anchors, mesh.levels
    E = mesh.n_elem
    # sibling groups: leaves sharing a parent at the same level
    merged = np.zeros(E, dtype=bool)
    par = a & ~((np.int64(1) << (MAXD - lv + 1))[:, None] - 1)
    groups = {}
    for i in range(E):
        if fl[i] == -1:
            groups.setdefault((int(lv[i]),) + tuple(int(v) for v in par[i]), []).append(i)
    out_a, out_l = [], []
    for key, members in groups.items():
        if len(members) == 8:
            merged[members] = True
            out_a.append(np.array(key[1:], dtype=np.int64))
            out_l.append(key[0] - 1)
    for i in range(E):
        if merged[i]:
            continue
        if fl[i] == 1:
            out_a += _children(a[i], lv[i])
            out_l += [lv[i] + 1] * 8
        else:
            out_a.append(a[i])
            out_l.append(lv[i])
    return balance(np.array(out_a), np.array(out_l))


def locate(mesh: Mesh, pts: np.ndarray, chunk: int = 256) -> np.ndarray:
    """Index of the first leaf (in Morton order) whose closed box contains each integer point."""
    lo = mesh.anchors
    hi = mesh.anchors + mesh.side[:, None]
    out = np.empty(len(pts), dtype=np.int64)
    for s in range(0, len(pts), chunk):
        p = pts[s:s + chunk]
        inside = np.all((lo[None, :, :] <= p[:, None, :]) & (p[:, None, :] <= hi[None, :, :]), axis=2)
        if not np.all(inside.any(axis=1)):
            raise ValueError("a point lies in no leaf")
        out[s:s + chunk] = np.argmax(inside, axis=1)
    return out


def transfer(a: Mesh, b: Mesh, u: np.ndarray) -> np.ndarray:
    """Nodal values on b of the finite-element function u of a (u: (N_a,) or (k, N_a))."""
    u = np.asarray(u, dtype=np.float64)
    single = u.ndim == 1
    U = u[None, :] if single else u
    e = locate(a, b.node_int)
    xi = (b.node_int - a.anchors[e]).astype(np.float64) / a.side[e][:, None].astype(np.float64)
    w = np.prod(np.where(CORNER_BITS[None, :, :] == 1, xi[:, None, :], 1.0 - xi[:, None, :]),
                axis=2)                                                    # (N_b, 8)
    out = np.stack([np.sum(w * a.element_values(Uk)[e], axis=1) for Uk in U])
    return out[0] if single else out
