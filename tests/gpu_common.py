"""Shared setup of the GPU parity tests: the same seeded leaf lists and fields go to the CUDA
library (through the C ABI) and to the CPU oracle; every expected value comes from the oracle."""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

from chns_workloads import configs, octree
from chns_workloads.octree import MAXD
from oracle import fem, solvers
from oracle.mesh import Mesh as OMesh

PRM = dict(Re=35.0, We=2.0, Cn=0.05, Pe=50.0, Fr=1.0, rho_ratio=20.0, eta_ratio=5.0, dt=1e-3,
           C_I=6.0)


def _one_refined():
    a, l = octree.uniform(1)
    keep = np.any(a != 0, axis=1)
    kids = (np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)]) << (MAXD - 2))
    a2 = np.concatenate([a[keep], kids.astype(np.uint32)])
    l2 = np.concatenate([l[keep], np.full(8, 2, dtype=np.uint8)])
    return octree.morton_sort(a2, l2)


LEAVES = {
    "uniform2": (lambda: octree.uniform(2), (1.0, 1.0, 1.0)),
    "one_refined": (_one_refined, (1.0, 1.0, 1.0)),
    "random0_box": (lambda: configs.random_balanced(0, 1, 4, 0.3), (1.0, 2.0, 0.5)),
    "random1": (lambda: configs.random_balanced(1, 2, 5, 0.2), (1.0, 1.0, 1.0)),
    "drop_l3_5": (lambda: (lambda w: (w.anchors, w.levels))(configs.rising_drop(3, 5, Cn=0.04)),
                  (1.0, 1.0, 1.0)),
}
SMALL = list(LEAVES)


@functools.lru_cache(maxsize=None)
def meshes(name):
    from paper_2107_05123_gb300.session import Mesh
    f, ext = LEAVES[name]
    a, l = f()
    return OMesh(a, l, ext), Mesh(a, l, ext)


def fields(n, seed):
    rng = np.random.default_rng(seed)
    return dict(phi=1.2 * np.tanh(1.5 * rng.standard_normal(n)),
                u=rng.standard_normal((3, n)), mu=rng.standard_normal(n),
                x=rng.standard_normal((3, n)))


def dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda",
                           dtype=dtype or torch.float64)


def bf16_round(a):
    """Round to bfloat16 (round to nearest even) and back, on the host."""
    import torch
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def f32_round(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dirichlet_matrix(A, mask):
    keep = sp.diags((~mask).astype(np.float64))
    return (keep @ A @ keep + sp.diags(mask.astype(np.float64))).tocsr()


def oracle_operator(om, op, prm, phi, u=None, mu=None):
    """The oracle's assembled matrix of an operator over all its components."""
    from paper_2107_05123_gb300 import capi
    el, co = fem.Elem(om), fem.Coeffs(prm)
    if op == capi.OP_POISSON:
        return fem.poisson(el, co, phi)
    if op == capi.OP_MASS:
        A = dirichlet_matrix(fem.mass_rho(el, co, phi), om.boundary)
        return sp.block_diag([A, A, A]).tocsr()
    if op == capi.OP_CH:
        return fem.ch_jacobian(el, co, phi, u)
    if op == capi.OP_MOMENTUM:
        vs = fem.VMSState(el, co, phi, u, mu)
        A = dirichlet_matrix(fem.momentum(vs), om.boundary)
        return sp.block_diag([A, A, A]).tocsr()
    raise ValueError(op)


def relerr(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))
