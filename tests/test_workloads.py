"""Input generators: octree construction, 2:1 balance, Morton order (Sec. 5.2)."""
import numpy as np
import pytest

from chns_workloads import configs, octree
from chns_workloads.octree import MAXD


def _volume(levels):
    return float(np.sum(8.0 ** (-levels.astype(np.float64))))


def _check_tree(a, l):
    assert abs(_volume(l) - 1.0) < 1e-12
    k = octree.morton_key(a.astype(np.int64))
    assert np.all(np.diff(k.astype(np.float64)) > 0)          # strictly Morton sorted
    s = (np.int64(1) << (MAXD - l.astype(np.int64)))
    assert np.all(a.astype(np.int64) % s[:, None] == 0)        # anchors aligned to their size


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_balanced(seed):
    a, l = configs.random_balanced(seed, 1, 4, 0.3)
    _check_tree(a, l)
    assert octree.is_balanced(a, l)


def test_balance_refines_unbalanced_input():
    # refine deeply only the octants whose upper corner is the cube centre: the finest of them
    # touch level-1 octants, so the input is unbalanced
    def pred(anchors, level):
        return np.all(anchors + (1 << (MAXD - level)) == (1 << (MAXD - 1)), axis=1)
    a, l = octree.build_octree(pred, 1, 5)
    assert not octree.is_balanced(a, l)
    b, m = octree.balance21(a, l)
    _check_tree(b, m)
    assert octree.is_balanced(b, m)
    # every original leaf is covered by leaves at least as fine
    for i in range(len(a)):
        lo = a[i].astype(np.int64)
        hi = lo + (1 << (MAXD - int(l[i])))
        inside = np.all((b >= lo) & (b < hi), axis=1)
        assert np.all(m[inside] >= l[i])


def test_balance_idempotent():
    a, l = configs.random_balanced(5, 1, 4, 0.3)
    b, m = octree.balance21(a, l)
    assert np.array_equal(a, b) and np.array_equal(l, m)


def test_uniform():
    a, l = octree.uniform(3)
    assert len(a) == 512
    _check_tree(a, l)


def test_rising_drop_mesh_shape():
    w = configs.rising_drop(3, 5, Cn=0.04)
    _check_tree(w.anchors, w.levels)
    assert w.levels.min() == 3 and w.levels.max() == 5
