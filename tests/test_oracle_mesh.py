"""Oracle mesh pins: node counts, hanging-node constraints, prolongation (Sec. 5.3)."""
import numpy as np
import pytest

from chns_workloads import configs, octree
from chns_workloads.octree import MAXD
from oracle.mesh import Mesh


@pytest.mark.parametrize("L", [1, 2, 3])
def test_uniform_counts(L):
    a, l = octree.uniform(L)
    m = Mesh(a, l)
    assert m.n_nodes == (2 ** L + 1) ** 3
    assert m.n_hanging == 0
    assert m.boundary.sum() == (2 ** L + 1) ** 3 - (2 ** L - 1) ** 3


def test_one_refined_octant_counts():
    # level-1 cube with the octant at the origin split once more: 27 coarse nodes and 19 new
    # points in the refined octant, of which 12 hang on the three interior coarse faces
    # (3 face centres + 9 distinct edge midpoints) and 7 are independent
    a, l = octree.uniform(1)
    keep = np.any(a != 0, axis=1)
    kids = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)]) << (MAXD - 2)
    a2 = np.concatenate([a[keep], kids.astype(np.uint32)])
    l2 = np.concatenate([l[keep], np.full(8, 2, dtype=np.uint8)])
    a2, l2 = octree.morton_sort(a2, l2)
    m = Mesh(a2, l2)
    assert m.n_hanging == 12
    assert m.n_nodes == 34
    assert np.sum(m.nparent == 4) == 3 and np.sum(m.nparent == 2) == 9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_prolongation_reproduces_linear(seed):
    a, l = configs.random_balanced(seed, 1, 4, 0.3)
    m = Mesh(a, l, extent=(1.0, 2.0, 0.5))
    assert m.n_hanging > 0
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(4)
    f = lambda x: c[0] + x[:, 0] * c[1] + x[:, 1] * c[2] + x[:, 2] * c[3]
    pts = m.points / float(1 << MAXD) * m.extent
    assert np.abs(m.P @ f(m.node_xyz) - f(pts)).max() < 1e-13
    # partition of unity, and parents are never hanging
    assert np.allclose(m.P.sum(axis=1), 1.0)
    assert not np.any(m.hanging[m.parent_pts[m.hanging][:, :2].ravel()])


def test_node_order_is_morton():
    a, l = configs.random_balanced(4, 1, 4, 0.3)
    m = Mesh(a, l)
    k = octree.morton_key(m.node_int)
    assert np.all(np.diff(k.astype(np.float64)) > 0)
