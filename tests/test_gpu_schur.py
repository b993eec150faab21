"""GPU parity of the Cahn-Hilliard Schur-complement preconditioner (flexible GMRES): the solution
of the CH Newton system agrees with the oracle's direct solve, the mixed-precision solve reaches
the FP64 residual the oracle's matrix confirms, and where the biharmonic part dominates (small
Cn h^-1 relative to dt) it needs far fewer iterations than the 2x2 nodal block-Jacobi
preconditioner."""
import numpy as np
import pytest

from gpu_common import PRM, dev, fields, meshes, oracle_operator, relerr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2107_05123_gb300 import capi  # noqa: E402
from oracle import solvers  # noqa: E402


def _system(prm, seed):
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, seed)
    f["phi"] = np.tanh(f["phi"])
    A = oracle_operator(om, capi.OP_CH, prm, f["phi"], f["u"], f["mu"])
    b = f["x"][:2].ravel().copy()
    coef = capi.make_coef(dev(f["phi"]), [dev(f["u"][i]) for i in range(3)], dev(f["mu"]))
    return om, gm, A, b, coef


def _solve(gm, prm, coef, b, pc, inner=capi.FP64, rtol=1e-12, max_it=20000, inner_its=0):
    x = torch.zeros(2 * gm.n_nodes, dtype=torch.float64, device="cuda")
    s = capi.make_solver(capi.KSP_GMRES, pc, rtol, max_it, 30, inner, 1e-3, 40,
                         inner_its=inner_its)
    st = capi.chns_krylov_solve(gm.handle, capi.OP_CH, capi.make_params(prm), coef, dev(b), x, s,
                                check=False)
    return x.cpu().numpy(), st


@pytest.mark.parametrize("kernel", [capi.APPLY_PATCH, capi.APPLY_STREAM])
def test_schur_mixed_precision_through_either_apply_kernel(kernel):
    """The FP32 shifted operator of the preconditioner runs through the per-patch or the
    persistent pipelined kernel (the automatic choice on large meshes); both reach the FP64
    residual the oracle's matrix confirms."""
    om, gm, A, b, coef = _system(PRM, 94)
    capi.chns_mesh_set_apply_config(gm.handle, kernel, 0)
    try:
        x, st = _solve(gm, PRM, coef, b, capi.PC_SCHUR, inner=capi.FP32, rtol=1e-10)
    finally:
        capi.chns_mesh_set_apply_config(gm.handle, capi.APPLY_AUTO, 0)
    assert st.status == capi.OK
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.05e-10


@pytest.mark.parametrize("inner_its", [0, 6])
def test_schur_solve_fp64_matches_oracle(inner_its):
    om, gm, A, b, coef = _system(PRM, 91)
    ref = solvers.direct(A, b)
    x, st = _solve(gm, PRM, coef, b, capi.PC_SCHUR, inner_its=inner_its)
    assert st.status == capi.OK
    assert st.rel_residual <= 1e-12
    assert relerr(x, ref) < 1e-8


def test_schur_mixed_precision_reaches_fp64_residual():
    om, gm, A, b, coef = _system(PRM, 92)
    x, st = _solve(gm, PRM, coef, b, capi.PC_SCHUR, inner=capi.FP32, rtol=1e-10)
    assert st.status == capi.OK and st.refinements >= 1
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.05e-10


def test_schur_beats_block_jacobi_where_the_biharmonic_term_dominates():
    stiff = dict(PRM, Cn=0.02, Pe=1.0 / (3 * 0.02 ** 2), dt=2e-2)
    om, gm, A, b, coef = _system(stiff, 93)
    ref = solvers.direct(A, b)
    xs, ss = _solve(gm, stiff, coef, b, capi.PC_SCHUR, rtol=1e-10)
    xj, sj = _solve(gm, stiff, coef, b, capi.PC_JACOBI, rtol=1e-10, max_it=3000)
    assert ss.status == capi.OK
    assert relerr(xs, ref) < 1e-6
    assert ss.iterations * 2 < sj.iterations, (ss.iterations, sj.iterations)


def test_schur_rejects_other_operators_and_long_restarts():
    om, gm = meshes("drop_l3_5")
    x = torch.zeros(gm.n_nodes, dtype=torch.float64, device="cuda")
    b = torch.ones(gm.n_nodes, dtype=torch.float64, device="cuda")
    ph = torch.zeros(gm.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.ChnsError):
        capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, capi.make_params(PRM),
                               capi.make_coef(ph), b, x,
                               capi.make_solver(capi.KSP_CG, capi.PC_SCHUR, 1e-8))
    x2 = torch.zeros(2 * gm.n_nodes, dtype=torch.float64, device="cuda")
    b2 = torch.ones(2 * gm.n_nodes, dtype=torch.float64, device="cuda")
    z = [ph, ph, ph]
    with pytest.raises(capi.ChnsError):
        capi.chns_krylov_solve(gm.handle, capi.OP_CH, capi.make_params(PRM),
                               capi.make_coef(ph, z, ph), b2, x2,
                               capi.make_solver(capi.KSP_GMRES, capi.PC_SCHUR, 1e-8, 100, 40))
