"""Oracle linear and nonlinear solvers.

TEST INFRASTRUCTURE ONLY (see the package header).

* ``pcg``: textbook preconditioned conjugate gradients with a Jacobi (diagonal) preconditioner,
  stopping on ||r||_2 / ||b||_2 <= rtol. With ``mean_zero`` the right-hand side and the result
  are projected to discrete mean zero (pure-Neumann pressure, reading R7).
* ``dirichlet``: row/column elimination with identity rows for velocity (H^1_0, Sec. 4).
* ``direct`` and ``gmres``: library sparse LU (SuperLU) and GMRES used as solver steps.
* ``chebyshev_precond``: the Chebyshev iteration for D^-1 A z = D^-1 r from z = 0 on an interval
  [lmin, lmax] (three-term recurrence), i.e. z = p(D^-1 A) D^-1 r; the polynomial preconditioner
  beside Jacobi in the build's Krylov row (not in the paper, whose PETSc solves use AMG/ASM).
* ``newton``: plain Newton on the CH residual (Appendix A uses Newton; Sec. 6.2 reports one
  iteration at the time steps used).
* ``ch_schur_precond``: the block upper-triangular preconditioner of the CH Newton Jacobian
  [A B; C D] (Def. weak_VMS_disc_CH linearised: B = K/(2 Pe Cn), D = -M/2) on the Schur
  complement of D, approximated by H M^-1 H, H = M/sqrt(dt) + Cn sqrt(k) K, with exact inner
  inverses (sparse LU); the build's CH preconditioner for fine meshes, not in the paper (whose
  PETSc solves use algebraic multigrid).

Pins: pcg against sparse LU on SPD systems; dirichlet elimination against a reduced solve; the
Chebyshev polynomial against its closed form; the Schur preconditioner with the exact Schur
complement makes (J P^-1 - I)^2 vanish (tests/test_oracle_solvers_step.py).

"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def pcg(A, b, x0=None, rtol=1e-8, maxit=100000, diag=None, mean_zero=False):
    """Jacobi-PCG. Returns (x, iterations, final relative residual)."""
    b = np.asarray(b, dtype=np.float64).copy()
    if mean_zero:
        b -= b.mean()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    dinv = 1.0 / (A.diagonal() if diag is None else diag)
    r = b - A @ x
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.linalg.norm(r) / bn
    while rel > rtol and it < maxit:
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        rel = np.linalg.norm(r) / bn
    if mean_zero:
        x -= x.mean()
    return x, it, rel


def dirichlet(A, b, mask, g=None):
    """Eliminate Dirichlet rows/columns (mask True) with data g (default 0): returns (A', b')
    with identity rows on the boundary and the known columns moved to the right-hand side."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    g = np.zeros(n) if g is None else np.asarray(g, dtype=np.float64)
    keep = (~mask).astype(np.float64)
    Dk = sp.diags(keep)
    b2 = keep * (b - A @ (g * mask)) + mask * g
    A2 = Dk @ A @ Dk + sp.diags(mask.astype(np.float64))
    return A2.tocsr(), b2


def direct(A, b):
    return spla.spsolve(sp.csc_matrix(A), b)


def gmres(A, b, x0=None, rtol=1e-12, restart=50, maxiter=2000):
    M = sp.diags(1.0 / A.diagonal())
    x, info = spla.gmres(A, b, x0=x0, rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter, M=M)
    if info != 0:
        raise RuntimeError(f"gmres did not converge (info={info})")
    return x


def newton(residual, jacobian, x0, rtol=1e-10, atol=1e-13, maxit=20, linsolve=direct):
    """Plain Newton: x <- x - J(x)^{-1} F(x) until ||F|| <= max(rtol ||F(x0)||, atol)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    F = residual(x)
    f0 = np.linalg.norm(F)
    its = 0
    while np.linalg.norm(F) > max(rtol * f0, atol) and its < maxit:
        x = x - linsolve(jacobian(x), F)
        F = residual(x)
        its += 1
    return x, its, float(np.linalg.norm(F))


def chebyshev_precond(A, dinv, r, lmin, lmax, degree):
    """z after `degree` Chebyshev steps for D^-1 A z = D^-1 r from z = 0 on [lmin, lmax]."""
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho_old = 1.0 / sigma
    d = dinv * r / theta
    z = d.copy()
    for _ in range(1, degree):
        rho = 1.0 / (2.0 * sigma - rho_old)
        d = rho * rho_old * d + (2.0 * rho / delta) * dinv * (r - A @ z)
        z = z + d
        rho_old = rho
    return z


def ch_schur_precond(M, K, dt, Pe, Cn, r, s_inv=None):
    """z = P^-1 r for P = [S~ B; 0 D] with B = k K, k = 1/(2 Pe Cn), D = -M/2 and
    S~^-1 = H^-1 M H^-1, H = M/sqrt(dt) + Cn sqrt(k) K (s_inv, a callable, replaces S~^-1).
    r and z hold [phi; mu]: z_mu = D^-1 r_mu, z_phi = S~^-1 (r_phi - B z_mu)."""
    n = M.shape[0]
    r = np.asarray(r, dtype=np.float64)
    k = 0.5 / (Pe * Cn)
    z_mu = -2.0 * spla.spsolve(M.tocsc(), r[n:])
    t = r[:n] - k * (K @ z_mu)
    if s_inv is None:
        H = (M / np.sqrt(dt) + Cn * np.sqrt(k) * K).tocsc()
        z_phi = spla.spsolve(H, M @ spla.spsolve(H, t))
    else:
        z_phi = s_inv(t)
    return np.concatenate([z_phi, z_mu])
