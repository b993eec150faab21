"""Seeded synthetic initial conditions (closed forms evaluated at given physical points).

Inputs only: these functions describe initial phase fields, chemical potentials and velocities
of the synthetic workloads. They hold none of the discretisation.

The interface profile is tanh(d / (sqrt(2) Cn)), the planar equilibrium of the chemical
potential mu = psi'(phi) - Cn^2 lap(phi) of Sec. 3 (psi' = phi^3 - phi), with the signed distance
d > 0 in the phase phi = +1 (the continuous, heavier fluid) and d < 0 inside drops (phi = -1).
(The 3D Rayleigh-Taylor setup of Sec. 6.4 prints tanh(sqrt(2) d / Cn), twice as steep; started
from it, a drop at density ratio 1000 releases the non-equilibrium capillary force in its first
steps.) The initial chemical potential is the pointwise closed form of mu, evaluated
analytically; for the equilibrium profile only the curvature part remains.
"""
from __future__ import annotations

import numpy as np


def _tanh_profile(d, grad_d_sq, lap_d, Cn):
    """phi = tanh(k d) with k = 1/(sqrt(2) Cn); returns phi and its Laplacian."""
    k = 1.0 / (np.sqrt(2.0) * Cn)
    t = np.tanh(k * d)
    s2 = 1.0 - t * t
    lap = k * s2 * lap_d - 2.0 * k * k * t * s2 * grad_d_sq
    return t, lap


def chem_potential(phi, lap_phi, Cn):
    """Closed-form mu = phi^3 - phi - Cn^2 lap(phi) of an analytic initial phase field."""
    return phi ** 3 - phi - Cn * Cn * lap_phi


# ---------------------------------------------------------------- config: manufactured smooth field
def smooth_phi(x):
    """phi = 0.5 sin(2 pi x) cos(2 pi y) cos(2 pi z) and its Laplacian."""
    tp = 2.0 * np.pi
    phi = 0.5 * np.sin(tp * x[:, 0]) * np.cos(tp * x[:, 1]) * np.cos(tp * x[:, 2])
    return phi, -3.0 * tp * tp * phi


def fourier_curl_velocity(x, seed: int, kmax: int = 2):
    """Divergence-free velocity u = curl A, A_c = sum_k a_{c,k} prod_d sin^2(pi k_d x_d),
    k in {1..kmax}^3, a ~ N(0,1) from numpy default_rng(seed). u and grad u vanish on the
    boundary of the unit cube."""
    rng = np.random.default_rng(seed)
    ks = [(kx, ky, kz) for kz in range(1, kmax + 1) for ky in range(1, kmax + 1)
          for kx in range(1, kmax + 1)]
    a = rng.standard_normal((3, len(ks)))
    pi = np.pi
    dA = np.zeros((3, 3, len(x)))  # dA[c, d] = dA_c/dx_d
    for m, k in enumerate(ks):
        s2 = [np.sin(pi * k[d] * x[:, d]) ** 2 for d in range(3)]
        ds2 = [pi * k[d] * np.sin(2 * pi * k[d] * x[:, d]) for d in range(3)]
        for d in range(3):
            prod = ds2[d].copy()
            for e in range(3):
                if e != d:
                    prod = prod * s2[e]
            for c in range(3):
                dA[c, d] += a[c, m] * prod
    u = np.stack([dA[2, 1] - dA[1, 2], dA[0, 2] - dA[2, 0], dA[1, 0] - dA[0, 1]], axis=0)
    return u


# ---------------------------------------------------------------- drops and interfaces
def drops_phi(x, centres, radii, Cn):
    """phi = min_i tanh((|x-c_i| - R_i)/(sqrt(2) Cn)) (phi = -1 inside drops) and its Laplacian
    taken from the drop that attains the minimum."""
    best_phi = None
    best_lap = None
    for c, R in zip(np.atleast_2d(centres), np.atleast_1d(radii)):
        r = np.linalg.norm(x - np.asarray(c)[None, :], axis=1)
        r_safe = np.maximum(r, 1e-300)
        phi, lap = _tanh_profile(r - R, 1.0, 2.0 / r_safe, Cn)
        if best_phi is None:
            best_phi, best_lap = phi, lap
        else:
            m = phi < best_phi
            best_phi = np.where(m, phi, best_phi)
            best_lap = np.where(m, lap, best_lap)
    return best_phi, best_lap


def rt_phi(x, Cn, y0=2.0, amp=0.05):
    """Perturbed planar interface y = y0 + amp cos(2 pi x) cos(2 pi z); phi = +1 above."""
    tp = 2.0 * np.pi
    cx, cz = np.cos(tp * x[:, 0]), np.cos(tp * x[:, 2])
    sx, sz = np.sin(tp * x[:, 0]), np.sin(tp * x[:, 2])
    d = x[:, 1] - y0 - amp * cx * cz
    g2 = 1.0 + (amp * tp * sx * cz) ** 2 + (amp * tp * cx * sz) ** 2
    lapd = 2.0 * amp * tp * tp * cx * cz
    return _tanh_profile(d, g2, lapd, Cn)


def nearest_drop(x, centres, radii, chunk: int = 1 << 20):
    """Index of the drop with the smallest signed distance |x - c_i| - R_i at each point and that
    distance, for many points and drops (squared distances through one matrix product per chunk
    of points)."""
    c = np.atleast_2d(np.asarray(centres, dtype=np.float64))
    R = np.atleast_1d(np.asarray(radii, dtype=np.float64))
    cc = np.sum(c * c, axis=1)
    idx = np.empty(len(x), dtype=np.int64)
    dmin = np.empty(len(x))
    for s in range(0, len(x), chunk):
        xs = np.asarray(x[s:s + chunk], dtype=np.float64)
        d2 = np.sum(xs * xs, axis=1)[:, None] - 2.0 * (xs @ c.T) + cc[None, :]
        d = np.sqrt(np.maximum(d2, 0.0)) - R[None, :]
        i = np.argmin(d, axis=1)
        idx[s:s + chunk] = i
        dmin[s:s + chunk] = d[np.arange(len(xs)), i]
    return idx, dmin


def drops_phi_nearest(x, centres, radii, Cn):
    """The phase of many drops, phi = tanh(d / (sqrt(2) Cn)) with d the smallest signed distance
    to a drop (tanh is increasing, so this is the minimum over drops of each drop's profile), and
    its Laplacian from that nearest drop, with r evaluated exactly for it."""
    c = np.atleast_2d(np.asarray(centres, dtype=np.float64))
    R = np.atleast_1d(np.asarray(radii, dtype=np.float64))
    i, _ = nearest_drop(x, c, R)
    r = np.linalg.norm(x - c[i], axis=1)
    return _tanh_profile(r - R[i], 1.0, 2.0 / np.maximum(r, 1e-300), Cn)


def sample_drops(seed: int, n: int, rmin: float, rmax: float, margin: float = 0.02,
                 max_tries: int = 100000):
    """Non-overlapping drops in the unit cube by rejection sampling (seeded)."""
    rng = np.random.default_rng(seed)
    cs, rs = [], []
    tries = 0
    while len(cs) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place drops")
        R = rng.uniform(rmin, rmax)
        c = rng.uniform(R + margin, 1.0 - R - margin, size=3)
        if all(np.linalg.norm(c - c2) > R + r2 + margin for c2, r2 in zip(cs, rs)):
            cs.append(c)
            rs.append(R)
    return np.array(cs), np.array(rs)
