"""Oracle mesh: nodes, hanging nodes and the prolongation P of a 2:1-balanced octree.

TEST INFRASTRUCTURE ONLY (see the package header).

Follows Sec. 5.3 ("Identification of unique, independent nodes"): the corners of every leaf are
emitted and de-duplicated by integer coordinate; a corner that lies in the interior of an edge
or a face of another (coarser) leaf is *hanging* and is not a degree of freedom. Its value is
interpolated from the immediate parent's nodes (caption of Fig. "traversal"): the two ends of
the coarse edge (weights 1/2) or the four corners of the coarse face (weights 1/4). With the
full 2:1 balance the parents of a hanging node are never hanging themselves.

Independent nodes are numbered in Morton order of their integer coordinates.

Pins: node counts of uniform meshes, partition of unity and exact reproduction of linear fields
by P (tests/test_oracle_mesh.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MAXD = 20
CORNER_BITS = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int64)


def _pkey(c: np.ndarray) -> np.ndarray:
    """Unique int64 key of integer points with coordinates in [0, 2**MAXD]."""
    m = np.int64((1 << MAXD) + 1)
    c = np.asarray(c, dtype=np.int64)
    return (c[..., 2] * m + c[..., 1]) * m + c[..., 0]


def _morton(c: np.ndarray) -> np.ndarray:
    """Morton key (x lowest) of points with 21-bit coordinates, by a plain bit loop."""
    c = np.asarray(c, dtype=np.uint64)
    key = np.zeros(len(c), dtype=np.uint64)
    for b in range(MAXD + 1):
        for d in range(3):
            bit = (c[:, d] >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(3 * b + d)
    return key


class Mesh:
    """Leaves -> (points, hanging constraints, P, element-to-point map, boundary flags)."""

    def __init__(self, anchors, levels, extent=(1.0, 1.0, 1.0)):
        self.anchors = np.asarray(anchors, dtype=np.int64)
        self.levels = np.asarray(levels, dtype=np.int64)
        self.extent = np.asarray(extent, dtype=np.float64)
        E = len(self.levels)
        self.n_elem = E
        side = np.int64(1) << (MAXD - self.levels)            # (E,)
        self.side = side
        # element sizes in physical units
        self.h = (side[:, None].astype(np.float64) / float(1 << MAXD)) * self.extent[None, :]

        # ---- all corners, de-duplicated
        corners = self.anchors[:, None, :] + side[:, None, None] * CORNER_BITS[None, :, :]
        keys = _pkey(corners).reshape(-1)
        ukeys, inv = np.unique(keys, return_inverse=True)
        self.e2p = inv.reshape(E, 8)
        pts = np.zeros((len(ukeys), 3), dtype=np.int64)
        pts[self.e2p.reshape(-1)] = corners.reshape(-1, 3)
        self.points = pts
        NP = len(ukeys)

        # ---- hanging points: corners that are an edge midpoint or face centre of some leaf
        half = side // 2
        cand, parents = [], []
        for d in range(3):                      # edges along axis d
            o1, o2 = [e for e in range(3) if e != d]
            for b1 in (0, 1):
                for b2 in (0, 1):
                    base = self.anchors.copy()
                    base[:, o1] += b1 * side
                    base[:, o2] += b2 * side
                    mid = base.copy()
                    mid[:, d] += half
                    end = base.copy()
                    end[:, d] += side
                    cand.append(mid)
                    parents.append(np.stack([base, end, base, end], axis=1))
        n_edge_cand = len(cand)
        for d in range(3):                      # faces normal to axis d
            o1, o2 = [e for e in range(3) if e != d]
            for b in (0, 1):
                base = self.anchors.copy()
                base[:, d] += b * side
                ctr = base.copy()
                ctr[:, o1] += half
                ctr[:, o2] += half
                cs = []
                for c1 in (0, 1):
                    for c2 in (0, 1):
                        q = base.copy()
                        q[:, o1] += c1 * side
                        q[:, o2] += c2 * side
                        cs.append(q)
                cand.append(ctr)
                parents.append(np.stack(cs, axis=1))
        kind = np.concatenate([np.full(E, 2 if i < n_edge_cand else 4) for i in range(len(cand))])
        cand = np.concatenate(cand)
        parents = np.concatenate(parents)
        ck = _pkey(cand)
        pos = np.searchsorted(ukeys, ck)
        pos = np.minimum(pos, NP - 1)
        hit = ukeys[pos] == ck
        hp = pos[hit]
        hkind = kind[hit]
        hpar = parents[hit]
        hanging = np.zeros(NP, dtype=bool)
        hanging[hp] = True
        nparent = np.zeros(NP, dtype=np.int64)
        parent_pts = np.full((NP, 4), -1, dtype=np.int64)
        # record parents (identical from every leaf that reports the same point)
        par_idx = np.searchsorted(ukeys, _pkey(hpar))
        if np.any(ukeys[np.minimum(par_idx, NP - 1)] != _pkey(hpar)):
            raise ValueError("hanging-node parent is not a mesh point (tree not 2:1 balanced?)")
        for i in range(len(hp)):
            p = hp[i]
            pp = np.unique(par_idx[i, :hkind[i]])
            if nparent[p] == 0:
                nparent[p] = len(pp)
                parent_pts[p, :len(pp)] = pp
            elif nparent[p] != len(pp) or np.any(parent_pts[p, :len(pp)] != pp):
                raise ValueError("inconsistent hanging constraints")
        if np.any(hanging[parent_pts[hanging][:, :2].reshape(-1)]):
            raise ValueError("chained hanging constraint (tree not 2:1 balanced)")
        self.hanging = hanging
        self.nparent = nparent
        self.parent_pts = parent_pts

        # ---- independent nodes in Morton order of their coordinates
        ind_pts = np.nonzero(~hanging)[0]
        order = np.argsort(_morton(pts[ind_pts]), kind="stable")
        ind_pts = ind_pts[order]
        N = len(ind_pts)
        self.n_nodes = N
        self.n_hanging = int(hanging.sum())
        p2n = np.full(NP, -1, dtype=np.int64)
        p2n[ind_pts] = np.arange(N)
        self.ind_pts = ind_pts
        self.p2n = p2n

        # ---- prolongation P: point values from independent node values
        rows, cols, vals = [ind_pts], [np.arange(N)], [np.ones(N)]
        hp_all = np.nonzero(hanging)[0]
        for k in (2, 4):
            sel = hp_all[nparent[hp_all] == k]
            for j in range(k):
                rows.append(sel)
                cols.append(p2n[parent_pts[sel, j]])
                vals.append(np.full(len(sel), 1.0 / k))
        self.P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(NP, N))

        # ---- node coordinates and boundary flags
        self.node_int = pts[ind_pts]
        self.node_xyz = self.node_int.astype(np.float64) / float(1 << MAXD) * self.extent[None, :]
        full = np.int64(1) << MAXD
        self.boundary = np.any((self.node_int == 0) | (self.node_int == full), axis=1)

    # ------------------------------------------------------------------ helpers
    def element_values(self, nodal: np.ndarray) -> np.ndarray:
        """Gather nodal values (N,) to element corners (E, 8) through P (hanging interpolation)."""
        return (self.P @ nodal)[self.e2p]

    def assemble_matrix(self, Ae: np.ndarray) -> sp.csr_matrix:
        """A = P^T (sum_e scatter(A_e)) P for element matrices Ae (E, 8, 8)."""
        E = self.n_elem
        r = np.repeat(self.e2p, 8, axis=1).reshape(-1)
        c = np.tile(self.e2p, (1, 8)).reshape(-1)
        NP = len(self.points)
        K = sp.csr_matrix((Ae.reshape(-1), (r, c)), shape=(NP, NP))
        return (self.P.T @ K @ self.P).tocsr()

    def assemble_vector(self, be: np.ndarray) -> np.ndarray:
        """b = P^T (sum_e scatter(b_e)) for element vectors be (E, 8)."""
        NP = len(self.points)
        v = np.bincount(self.e2p.reshape(-1), weights=be.reshape(-1), minlength=NP)
        return self.P.T @ v
