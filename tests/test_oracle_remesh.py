"""Pins of the oracle's remeshing and intergrid transfer (oracle/remesh.py, Sec. 5.4) against
what the geometry and the finite-element space fix, independently of the oracle's own code."""
import numpy as np
import pytest

from chns_workloads import configs, octree
from oracle import multigrid, remesh
from oracle.mesh import MAXD, Mesh


def _vol(levels):
    return float(np.sum(8.0 ** (-np.asarray(levels, dtype=np.float64))))


def test_flags_of_a_linear_phase_match_the_closed_form():
    """phi = (x - x0) / w is reproduced exactly by Q1 (and its centre value is the mean of the
    corners), so the 9-point minimum of |phi| on a leaf is min(|x_lo - x0|, |x_hi - x0|,
    |x_mid - x0|) / w from the leaf's geometry alone."""
    a, l = octree.balance21(*configs.random_balanced(3, 1, 4, 0.4))
    m = Mesh(a, l)
    x0, w, thr = 0.3719, 0.05, 0.95
    phi = (m.node_xyz[:, 0] - x0) / w
    fl = remesh.flags(m, phi, thr, 2, 4)
    h = m.side.astype(np.float64) / (1 << MAXD)
    xl = m.anchors[:, 0].astype(np.float64) / (1 << MAXD)
    d = np.minimum(np.minimum(np.abs(xl - x0), np.abs(xl + h - x0)), np.abs(xl + h / 2 - x0)) / w
    assert np.min(np.abs(d - thr)) > 1e-9  # no near-ties
    band = d <= thr
    want = np.where(band & (m.levels < 4), 1, np.where(~band & (m.levels > 2), -1, 0))
    assert np.array_equal(fl, want)
    assert (fl == 1).any() and (fl == -1).any() and (fl == 0).any()


def test_uniform_refine_and_coarsen_counts():
    a, l = octree.uniform(3)
    m = Mesh(a, l)
    a2, l2 = remesh.new_leaves(m, np.ones(m.n_elem, dtype=np.int8))
    assert len(l2) == 8 ** 4 and np.all(l2 == 4)
    a3, l3 = remesh.new_leaves(m, -np.ones(m.n_elem, dtype=np.int8))
    assert len(l3) == 8 ** 2 and np.all(l3 == 2)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_new_leaves_are_the_coarsest_balanced_refinement(seed):
    """Random flags on a random balanced tree: the result is 2:1 balanced (brute force), covers
    the cube, changes every old leaf by one level at most before balancing, and equals the input
    generators' ripple balance (an independent algorithm) applied to the same split/merge list."""
    a, l = octree.balance21(*configs.random_balanced(seed, 1, 4, 0.35))
    m = Mesh(a, l)
    rng = np.random.default_rng(seed)
    fl = rng.integers(-1, 2, m.n_elem).astype(np.int8)
    fl[m.levels >= 5] = np.minimum(fl[m.levels >= 5], 0)
    fl[m.levels <= 1] = np.maximum(fl[m.levels <= 1], 0)
    na, nl = remesh.new_leaves(m, fl)
    assert octree.is_balanced(na, nl)
    assert abs(_vol(nl) - 1.0) < 1e-12
    # the ripple balance of the input generators on the unbalanced split/merge list
    ua, ul = _split_merge(m, fl)
    ra, rl = octree.balance21(ua, ul)
    assert np.array_equal(np.asarray(ra, dtype=np.int64), na)
    assert np.array_equal(np.asarray(rl, dtype=np.int64), nl)


def _split_merge(m, fl):
    """The split/merge list before balancing, restated from Sec. 5.4 with plain loops."""
    out = []
    done = np.zeros(m.n_elem, dtype=bool)
    for i in range(m.n_elem):
        if done[i]:
            continue
        lv = int(m.levels[i])
        s = 1 << (MAXD - lv)
        ps = 2 * s
        pa = (m.anchors[i] // ps) * ps
        sib = [j for j in range(i, min(i + 8, m.n_elem))
               if m.levels[j] == lv and np.all((m.anchors[j] // ps) * ps == pa)]
        if lv > 0 and np.all(m.anchors[i] == pa) and len(sib) == 8 and all(fl[j] == -1 for j in sib):
            out.append((pa, lv - 1))
            done[sib] = True
            continue
        if fl[i] == 1:
            h = s // 2
            for c in range(8):
                out.append((m.anchors[i] + h * np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1]),
                            lv + 1))
        else:
            out.append((m.anchors[i], lv))
        done[i] = True
    return (np.array([o[0] for o in out], dtype=np.int64),
            np.array([o[1] for o in out], dtype=np.int64))


def test_transfer_reproduces_linear_fields():
    a, l = octree.balance21(*configs.random_balanced(4, 1, 4, 0.35))
    m = Mesh(a, l)
    rng = np.random.default_rng(4)
    fl = rng.integers(-1, 2, m.n_elem).astype(np.int8)
    fl[m.levels >= 5] = 0
    fl[m.levels <= 1] = np.maximum(fl[m.levels <= 1], 0)
    b = Mesh(*remesh.new_leaves(m, fl))
    c = np.array([0.3, -1.2, 0.7])
    u = m.node_xyz @ c + 0.25
    got = remesh.transfer(m, b, u)
    assert np.max(np.abs(got - (b.node_xyz @ c + 0.25))) < 1e-14


def test_refine_then_coarsen_round_trip_is_exact():
    a, l = octree.balance21(*configs.random_balanced(5, 1, 3, 0.4))
    m = Mesh(a, l)
    b = Mesh(*remesh.new_leaves(m, np.ones(m.n_elem, dtype=np.int8)))
    c = Mesh(*remesh.new_leaves(b, -np.ones(b.n_elem, dtype=np.int8)))
    assert np.array_equal(c.anchors, m.anchors) and np.array_equal(c.levels, m.levels)
    u = np.random.default_rng(5).standard_normal(m.n_nodes)
    back = remesh.transfer(b, c, remesh.transfer(m, b, u))
    assert np.array_equal(back, u)


def test_transfer_equals_multigrid_prolongation():
    """B = A with its finest level refined is A's multigrid fine mesh turned around: coarsening B
    gives A back, and the multigrid oracle's prolongation P(B <- A), built from the half-size
    lattice of each coarse leaf, equals the transfer built from point location."""
    a, l = octree.balance21(*configs.random_balanced(6, 1, 4, 0.35))
    fine = Mesh(a, l)
    ca, cl = multigrid.coarsen(a, l)
    coarse = Mesh(ca, cl)
    u = np.random.default_rng(6).standard_normal(coarse.n_nodes)
    P = multigrid.prolongation(fine, coarse)
    assert np.max(np.abs(remesh.transfer(coarse, fine, u) - P @ u)) < 1e-14


def test_planted_transposed_weights_are_caught(monkeypatch):
    """A plausible slip, the weights of xi and 1 - xi exchanged, fails the linear pin."""
    a, l = octree.balance21(*configs.random_balanced(4, 1, 3, 0.4))
    m = Mesh(a, l)
    b = Mesh(*remesh.new_leaves(m, np.ones(m.n_elem, dtype=np.int8)))
    orig = remesh.CORNER_BITS
    monkeypatch.setattr(remesh, "CORNER_BITS", 1 - orig)
    u = m.node_xyz[:, 0]
    assert np.max(np.abs(remesh.transfer(m, b, u) - b.node_xyz[:, 0])) > 0.1
