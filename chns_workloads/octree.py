"""Seeded octree workloads: top-down refinement from a predicate, 2:1 balance, Morton order.

This module produces *inputs* (leaf lists) for both the CUDA library and the CPU oracle.
It holds none of the finite-element arithmetic of the method.

Conventions
-----------
* ``MAXD`` = 20: anchors are integer coordinates in units of 2**-MAXD of the unit cube.
* A leaf is (anchor[3] uint32, level uint8); its side is 2**(MAXD-level) units.
* Leaves are returned in Morton (Z-order) order of their anchors, the space-filling-curve order
  in which the paper partitions and traverses octants (Sec. 5.2).
* Balance is the full 2:1 condition: two leaves that touch (through a face, an edge or a
  corner) differ by at most one level (Sec. 5.2, "2:1 balancing").
"""
from __future__ import annotations

import numpy as np

MAXD = 20

_OFFS27 = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)],
                   dtype=np.int64)


def _part1by2(v: np.ndarray) -> np.ndarray:
    """Spread the low 21 bits of v so that bit i lands at bit 3*i."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_key(xyz: np.ndarray) -> np.ndarray:
    """Morton key of integer points (n,3), x in the lowest bit of each triple. Coordinates < 2**21."""
    xyz = np.asarray(xyz)
    return (_part1by2(xyz[:, 0]) | (_part1by2(xyz[:, 1]) << np.uint64(1))
            | (_part1by2(xyz[:, 2]) << np.uint64(2)))


def _key(c: np.ndarray, level: int) -> np.ndarray:
    n = np.int64(1) << np.int64(level)
    return (c[:, 2].astype(np.int64) * n + c[:, 1]) * n + c[:, 0]


def _unkey(k: np.ndarray, level: int) -> np.ndarray:
    n = np.int64(1) << np.int64(level)
    return np.stack([k % n, (k // n) % n, k // (n * n)], axis=1).astype(np.int64)


def build_octree(refine, lmin: int, lmax: int) -> tuple[np.ndarray, np.ndarray]:
    """Top-down construction (Sec. 5.2): refine every octant below ``lmin``, and octants for
    which ``refine(anchor_units, level)`` is true below ``lmax``.

    ``refine`` takes an (m,3) int64 array of anchors (units of 2**-MAXD) and the level, and
    returns a bool array of length m. Returns (anchors uint32 (n,3), levels uint8 (n,)),
    not yet balanced and not yet sorted.
    """
    if not (0 <= lmin <= lmax < MAXD):
        raise ValueError("need 0 <= lmin <= lmax < MAXD")
    octs = np.zeros((1, 3), dtype=np.int64)
    out_a, out_l = [], []
    for lev in range(0, lmax + 1):
        if lev < lmin:
            split = np.ones(len(octs), dtype=bool)
        elif lev == lmax:
            split = np.zeros(len(octs), dtype=bool)
        else:
            split = np.asarray(refine(octs, lev), dtype=bool)
        out_a.append(octs[~split])
        out_l.append(np.full((~split).sum(), lev, dtype=np.uint8))
        par = octs[split]
        if len(par) == 0:
            break
        half = np.int64(1) << np.int64(MAXD - lev - 1)
        kids = [par + np.array([(c & 1) * half, ((c >> 1) & 1) * half, ((c >> 2) & 1) * half])
                for c in range(8)]
        octs = np.concatenate(kids, axis=0)
    return np.concatenate(out_a).astype(np.uint32), np.concatenate(out_l)


def balance21(anchors: np.ndarray, levels: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Refine leaves until the tree is 2:1 balanced across faces, edges and corners.

    Works on the set of *split* octants per level: if an octant P at level l is split, each of
    its 26 same-level neighbours N inside the domain must exist as an octant, i.e. parent(N)
    must be split as well. Levels are processed from fine to coarse so that requirements
    ripple upward. Returns the balanced leaves in Morton order.
    """
    anchors = np.asarray(anchors, dtype=np.int64)
    levels = np.asarray(levels, dtype=np.int64)
    lmax = int(levels.max()) if len(levels) else 0
    split: list[np.ndarray] = [np.zeros(0, dtype=np.int64) for _ in range(lmax + 1)]
    for L in range(1, lmax + 1):
        sel = anchors[levels == L]
        if len(sel) == 0:
            continue
        for l in range(L):
            split[l] = np.concatenate([split[l], _key(sel >> (MAXD - l), l)])
    split = [np.unique(s) for s in split]
    for l in range(lmax - 1, 0, -1):
        if len(split[l]) == 0:
            continue
        c = _unkey(split[l], l)
        nb = (c[:, None, :] + _OFFS27[None, :, :]).reshape(-1, 3)
        inside = np.all((nb >= 0) & (nb < (1 << l)), axis=1)
        req = np.unique(_key(nb[inside] >> 1, l - 1))
        split[l - 1] = np.union1d(split[l - 1], req)
    out_a, out_l = [], []
    if len(split[0]) == 0:
        return np.zeros((1, 3), dtype=np.uint32), np.zeros(1, dtype=np.uint8)
    for l in range(lmax + 1):
        if len(split[l]) == 0:
            continue
        c = _unkey(split[l], l)
        kids = np.concatenate([2 * c + np.array([ch & 1, (ch >> 1) & 1, (ch >> 2) & 1])
                               for ch in range(8)], axis=0)
        kk = _key(kids, l + 1)
        nxt = split[l + 1] if l + 1 <= lmax else np.zeros(0, dtype=np.int64)
        leaf = ~np.isin(kk, nxt)
        out_a.append(kids[leaf] << (MAXD - l - 1))
        out_l.append(np.full(leaf.sum(), l + 1, dtype=np.uint8))
    return morton_sort(np.concatenate(out_a).astype(np.uint32), np.concatenate(out_l))


def morton_sort(anchors: np.ndarray, levels: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    order = np.argsort(morton_key(np.asarray(anchors, dtype=np.int64)), kind="stable")
    return np.ascontiguousarray(anchors[order]), np.ascontiguousarray(levels[order])


def uniform(level: int) -> tuple[np.ndarray, np.ndarray]:
    """All 8**level octants of one level, Morton-sorted."""
    n = 1 << level
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    a = (g.reshape(-1, 3).astype(np.int64) << (MAXD - level)).astype(np.uint32)
    return morton_sort(a, np.full(len(a), level, dtype=np.uint8))


def octant_corner_points(anchors: np.ndarray, levels: np.ndarray, extent) -> np.ndarray:
    """Physical coordinates (n, 9, 3) of the 8 corners and the centre of each octant."""
    a = np.asarray(anchors, dtype=np.float64)
    s = (2.0 ** (MAXD - np.asarray(levels, dtype=np.float64)))[:, None]
    pts = [a + s * np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1]) for c in range(8)]
    pts.append(a + 0.5 * s)
    p = np.stack(pts, axis=1) / float(1 << MAXD)
    return p * np.asarray(extent, dtype=np.float64)[None, None, :]


def refine_band(phi_fn, extent, threshold: float):
    """Refinement predicate of the form 'min over corners and centre of |phi| < threshold'."""
    def pred(anchors, level):
        lev = np.full(len(anchors), level)
        pts = octant_corner_points(anchors, lev, extent)
        v = np.abs(phi_fn(pts.reshape(-1, 3))).reshape(len(anchors), 9)
        return v.min(axis=1) < threshold
    return pred


def is_balanced(anchors: np.ndarray, levels: np.ndarray) -> bool:
    """Brute-force check of the full 2:1 condition (for tests on small trees)."""
    a = np.asarray(anchors, dtype=np.int64)
    lv = np.asarray(levels, dtype=np.int64)
    s = np.int64(1) << (MAXD - lv)
    lo, hi = a, a + s[:, None]
    n = len(a)
    for i in range(n):
        touch = np.all((lo <= hi[i]) & (hi >= lo[i]), axis=1)
        touch[i] = False
        if np.any(np.abs(lv[touch] - lv[i]) > 1):
            return False
    return True
