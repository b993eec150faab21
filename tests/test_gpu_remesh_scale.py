"""Remeshing at the size the bench runs it (the rising drop on levels 5-8, 314,672 leaves, band
|phi| <= 0.95): the GPU's band flags equal the oracle's, its new leaf list equals the input
generators' ripple 2:1 balance of the same split/merge list (an implementation independent of
both the library's and the oracle's; on small meshes the oracle's brute-force balance is pinned
to it), and the transferred fields equal the oracle's finite-element evaluation at 1,500 sampled
new nodes (1e-13)."""
import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs, octree  # noqa: E402
from oracle import remesh as orem  # noqa: E402
from oracle.mesh import CORNER_BITS, MAXD, Mesh as OMesh  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import Mesh  # noqa: E402

THR = 0.95


@functools.lru_cache(maxsize=None)
def _case():
    w = configs.rising_drop(5, 8)
    om = OMesh(w.anchors, w.levels, w.extent)
    gm = Mesh(w.anchors, w.levels, w.extent)
    phi = w.init(om.node_xyz)["phi"]
    return w, om, gm, phi


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _split_merge(a, lv, fl):
    """The split/merge list of Sec. 5.4 before balancing (vectorised over the leaves): runs of 8
    sibling leaves that are all -1 become their parent, +1 leaves become their 8 children."""
    n = len(lv)
    s = np.int64(1) << (MAXD - lv)
    first = np.zeros(n, dtype=bool)
    ok = (lv > 0) & np.all(a % (2 * s)[:, None] == 0, axis=1) & (np.arange(n) + 7 < n)
    idx = np.nonzero(ok)[0]
    good = np.ones(len(idx), dtype=bool)
    for c in range(8):
        j = idx + c
        good &= (lv[j] == lv[idx]) & (fl[j] == -1)
        good &= np.all(a[j] == a[idx] + s[idx, None] * CORNER_BITS[c][None, :], axis=1)
    first[idx[good]] = True
    merged = np.zeros(n, dtype=bool)
    for c in range(8):
        merged[np.nonzero(first)[0] + c] = True
    keep = ~merged & (fl != 1)
    ref = ~merged & (fl == 1)
    half = s[ref] // 2
    kids = [a[ref] + half[:, None] * CORNER_BITS[c][None, :] for c in range(8)]
    out_a = np.concatenate([a[keep], a[first]] + kids)
    out_l = np.concatenate([lv[keep], lv[first] - 1] + [lv[ref] + 1] * 8)
    return out_a, out_l


def test_flags_and_leaves_at_bench_size():
    w, om, gm, phi = _case()
    v = np.abs(orem.phase_at_corners_and_centre(om, phi)).min(axis=1)
    assert np.min(np.abs(v - THR)) > 1e-9  # no near-ties
    ref = orem.flags(om, phi, THR, 5, 8)
    fl = torch.empty(gm.n_elem, dtype=torch.int8, device="cuda")
    capi.chns_remesh_flags(gm.handle, _dev(phi), THR, 5, 8, fl)
    assert np.array_equal(fl.cpu().numpy(), ref)
    ua, ul = _split_merge(om.anchors, om.levels, ref)
    ra, rl = octree.balance21(ua, ul)
    nm = Mesh(handle=capi.chns_mesh_remesh(gm.handle, _dev(phi), THR, 5, 8))
    a, l = nm.leaves()
    assert len(l) == len(rl) > gm.n_elem
    assert np.array_equal(a.astype(np.int64), np.asarray(ra, dtype=np.int64))
    assert np.array_equal(l.astype(np.int64), np.asarray(rl, dtype=np.int64))


def test_transfer_at_bench_size_on_sampled_nodes():
    w, om, gm, phi = _case()
    nm = Mesh(handle=capi.chns_mesh_remesh(gm.handle, _dev(phi), THR, 5, 8))
    rng = np.random.default_rng(71)
    U = rng.standard_normal((2, om.n_nodes))
    src = [_dev(U[i]) for i in range(2)]
    dst = [torch.empty(nm.n_nodes, dtype=torch.float64, device="cuda") for _ in range(2)]
    capi.chns_transfer(gm.handle, nm.handle, src, dst)
    got = np.stack([d.cpu().numpy() for d in dst])
    sel = rng.choice(nm.n_nodes, 1500, replace=False)
    pts = nm.node_int[sel].astype(np.int64)
    e = orem.locate(om, pts, chunk=64)
    xi = (pts - om.anchors[e]).astype(np.float64) / om.side[e][:, None].astype(np.float64)
    wgt = np.prod(np.where(CORNER_BITS[None, :, :] == 1, xi[:, None, :], 1.0 - xi[:, None, :]),
                  axis=2)
    for i in range(2):
        ref = np.sum(wgt * om.element_values(U[i])[e], axis=1)
        assert np.max(np.abs(got[i][sel] - ref)) <= 1e-13 * np.max(np.abs(U[i]))
