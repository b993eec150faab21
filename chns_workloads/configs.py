"""The synthetic workloads: meshes (leaf lists), physical parameters and initial fields.

Each workload is a leaf list (Morton order, 2:1 balanced), a box extent, a parameter set and a
function that evaluates the initial fields at physical node coordinates. Node coordinates are
not produced here: the oracle and the CUDA library each enumerate nodes from the leaf list
themselves, and both evaluate these closed forms at the points they find.

Physical parameters follow Sec. 3 (non-dimensional groups; 1/Pe = 3 Cn^2 where the workload
does not fix Pe) and the density/viscosity ratios rho_+/rho_-, eta_+/eta_- with the phase
phi = +1 as the reference fluid.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from . import fields, octree


@dataclass
class Params:
    Re: float
    We: float
    Cn: float
    Pe: float
    Fr: float
    rho_ratio: float   # rho_+ / rho_-  (phase +1 over phase -1)
    eta_ratio: float   # eta_+ / eta_-
    dt: float
    C_I: float = 6.0

    def as_dict(self):
        return dict(Re=self.Re, We=self.We, Cn=self.Cn, Pe=self.Pe, Fr=self.Fr,
                    rho_ratio=self.rho_ratio, eta_ratio=self.eta_ratio, dt=self.dt, C_I=self.C_I)


@dataclass
class Workload:
    name: str
    anchors: np.ndarray
    levels: np.ndarray
    extent: tuple
    params: Params
    init: Callable  # x (n,3) physical -> dict(phi, mu, u (3,n), p)
    steps: int = 1
    info: dict = field(default_factory=dict)

    @property
    def n_elem(self):
        return len(self.levels)


def _smooth_init(seed, Cn):
    def init(x):
        phi, lap = fields.smooth_phi(x)
        return dict(phi=phi, mu=fields.chem_potential(phi, lap, Cn),
                    u=fields.fourier_curl_velocity(x, seed), p=np.zeros(len(x)))
    return init


def _drops_init(centres, radii, Cn):
    def init(x):
        phi, lap = fields.drops_phi(x, centres, radii, Cn)
        return dict(phi=phi, mu=fields.chem_potential(phi, lap, Cn),
                    u=np.zeros((3, len(x))), p=np.zeros(len(x)))
    return init


def smooth_uniform(level: int = 4, seed: int = 0) -> Workload:
    """Uniform octree of one level on the unit cube, smooth phase field, random
    divergence-free velocity (Fourier modes k <= 2), fluid parameters of moderate contrast."""
    a, l = octree.uniform(level)
    p = Params(Re=100.0, We=10.0, Cn=0.1, Pe=100.0, Fr=1.0, rho_ratio=10.0, eta_ratio=10.0,
               dt=1e-3)
    return Workload(f"smooth_uniform_l{level}", a, l, (1.0, 1.0, 1.0), p,
                    _smooth_init(seed, p.Cn), steps=1)


def drop_octree(centres, radii, Cn, lmin, lmax, threshold=0.9):
    phi_fn = lambda x: fields.drops_phi(x, centres, radii, Cn)[0]
    a, l = octree.build_octree(octree.refine_band(phi_fn, (1, 1, 1), threshold), lmin, lmax)
    return octree.balance21(a, l)


def rising_drop(lmin: int = 5, lmax: int = 8, Cn: float = 0.01) -> Workload:
    """A drop of radius 0.15 at (0.5, 0.5, 0.3) (phi = -1 inside), fluid at rest, density ratio
    1000, viscosity ratio 100; adaptive levels lmin..lmax refined where |phi| < 0.9."""
    c, r = np.array([[0.5, 0.5, 0.3]]), np.array([0.15])
    a, l = drop_octree(c, r, Cn, lmin, lmax)
    p = Params(Re=35.0, We=1.0, Cn=Cn, Pe=1.0 / (3 * Cn * Cn), Fr=1.0, rho_ratio=1000.0,
               eta_ratio=100.0, dt=5e-4)
    return Workload(f"rising_drop_l{lmin}-{lmax}", a, l, (1.0, 1.0, 1.0), p,
                    _drops_init(c, r, Cn), steps=10, info=dict(centres=c, radii=r))


def rayleigh_taylor(lmin: int = 6, lmax: int = 10, Cn: float = 0.005) -> Workload:
    """Perturbed interface y = 2 + 0.05 cos(2 pi x) cos(2 pi z) in the box [0,1]x[0,4]x[0,1]
    (the unit octree scaled per axis by (1, 4, 1)); heavy phase on top, density ratio 3."""
    ext = (1.0, 4.0, 1.0)
    phi_fn = lambda x: fields.rt_phi(x, Cn)[0]
    a, l = octree.build_octree(octree.refine_band(phi_fn, ext, 0.9), lmin, lmax)
    a, l = octree.balance21(a, l)
    p = Params(Re=1000.0, We=1000.0, Cn=Cn, Pe=1.0 / (3 * Cn * Cn), Fr=1.0, rho_ratio=3.0,
               eta_ratio=1.0, dt=2.5e-4)

    def init(x):
        phi, lap = fields.rt_phi(x, Cn)
        return dict(phi=phi, mu=fields.chem_potential(phi, lap, Cn),
                    u=np.zeros((3, len(x))), p=np.zeros(len(x)))
    return Workload(f"rayleigh_taylor_l{lmin}-{lmax}", a, l, ext, p, init, steps=20)


def many_drops(seed: int = 0, n: int = 8, rmin: float = 0.05, rmax: float = 0.12,
               lmin: int = 5, lmax: int = 8, Cn: float = 0.01) -> Workload:
    """Seeded non-overlapping drops (phi = -1 inside) with the rising-drop parameters."""
    c, r = fields.sample_drops(seed, n, rmin, rmax)
    a, l = drop_octree(c, r, Cn, lmin, lmax)
    p = Params(Re=35.0, We=1.0, Cn=Cn, Pe=1.0 / (3 * Cn * Cn), Fr=1.0, rho_ratio=1000.0,
               eta_ratio=100.0, dt=5e-4)
    return Workload(f"drops{n}_s{seed}_l{lmin}-{lmax}", a, l, (1.0, 1.0, 1.0), p,
                    _drops_init(c, r, Cn), steps=1, info=dict(centres=c, radii=r))


def shear_velocity(x, U=1.0):
    """The linear shear u = U (2y - 1, 0, 0) of the unit cube: the walls y = 0 and y = 1 move
    with -U and +U, the faces x = 0 and x = 1 see the profile flow in and out (zero net flux)."""
    u = np.zeros((3, len(x)))
    u[0] = U * (2.0 * x[:, 1] - 1.0)
    return u


def breakup(lmin: int = 6, lmax: int = 11, Cn: float = 0.002, n: int = 64, seed: int = 0,
            U: float = 1.0) -> Workload:
    """Many-drop breakup: n seeded non-overlapping drops of radius 0.02-0.08 (phi = -1 inside) in
    the unit cube under the shear u = U (2y - 1, 0, 0), imposed as velocity Dirichlet data on
    every face and taken as the initial velocity; density ratio 100, viscosity ratio 50,
    Re 2000, We 50, Fr 1, dt 1e-4; levels lmin..lmax refined where |phi| < 0.9."""
    c, r = fields.sample_drops(seed, n, 0.02, 0.08)
    phi_fn = lambda x: np.tanh(fields.nearest_drop(x, c, r)[1] / (np.sqrt(2.0) * Cn))
    a, l = octree.build_octree(octree.refine_band(phi_fn, (1, 1, 1), 0.9), lmin, lmax)
    a, l = octree.balance21(a, l)
    p = Params(Re=2000.0, We=50.0, Cn=Cn, Pe=1.0 / (3 * Cn * Cn), Fr=1.0, rho_ratio=100.0,
               eta_ratio=50.0, dt=1e-4)

    def init(x):
        phi, lap = fields.drops_phi_nearest(x, c, r, Cn)
        return dict(phi=phi, mu=fields.chem_potential(phi, lap, Cn), u=shear_velocity(x, U),
                    p=np.zeros(len(x)))
    return Workload(f"breakup{n}_s{seed}_l{lmin}-{lmax}", a, l, (1.0, 1.0, 1.0), p, init,
                    steps=50, info=dict(centres=c, radii=r,
                                        velocity_bc=lambda x, t: shear_velocity(x, U)))


def random_balanced(seed: int, lmin: int = 1, lmax: int = 4, frac: float = 0.3):
    """A small random 2:1-balanced octree (for hanging-node tests): refine a random fraction
    of octants at each level, then balance."""
    rng = np.random.default_rng(seed)
    pred = lambda anchors, level: rng.random(len(anchors)) < frac
    a, l = octree.build_octree(pred, lmin, lmax)
    return octree.balance21(a, l)
