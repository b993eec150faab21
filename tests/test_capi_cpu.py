"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/chns.h declares, and rejects invalid leaf lists before touching the device."""
import os
import re

import numpy as np
import pytest

from chns_workloads import octree
from chns_workloads.octree import MAXD


def _header_functions(root):
    src = open(os.path.join(root, "include", "chns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chns_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(root):
    from paper_2107_05123_gb300 import capi
    declared = _header_functions(root)
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(capi.LIB, name), name
    assert set(declared) == set(capi.DECLARED)
    assert "sm_103a" in capi.chns_version()


def _expect(status, fn):
    from paper_2107_05123_gb300 import capi
    with pytest.raises(capi.ChnsError) as ei:
        fn()
    assert ei.value.status == status


def test_rejects_invalid_leaves():
    from paper_2107_05123_gb300 import capi
    a, l = octree.uniform(2)
    # unsorted
    _expect(capi.EINVAL, lambda: capi.chns_mesh_create(a[::-1].copy(), l[::-1].copy()))
    # missing a leaf (not covering)
    _expect(capi.EINVAL, lambda: capi.chns_mesh_create(a[1:], l[1:]))
    # misaligned anchor
    b = a.copy()
    b[3, 0] += 1
    _expect(capi.EINVAL, lambda: capi.chns_mesh_create(b, l))
    # level out of range
    _expect(capi.EINVAL, lambda: capi.chns_mesh_create(np.zeros((1, 3), np.uint32),
                                                       np.array([MAXD], np.uint8)))
    # bad extent
    _expect(capi.EINVAL, lambda: capi.chns_mesh_create(a, l, (1.0, 0.0, 1.0)))


def test_rejects_unbalanced_leaves():
    from paper_2107_05123_gb300 import capi

    def pred(anchors, level):
        return np.all(anchors + (1 << (MAXD - level)) == (1 << (MAXD - 1)), axis=1)
    a, l = octree.build_octree(pred, 1, 4)
    a, l = octree.morton_sort(a, l)
    assert not octree.is_balanced(a, l)
    _expect(capi.EUNBALANCED, lambda: capi.chns_mesh_create(a, l))
