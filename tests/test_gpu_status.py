"""Failure statuses of the Krylov solve through the C ABI, with the failures made on the host:
a right-hand side holding a NaN gives CHNS_ENAN, and an iteration limit reached before the
tolerance gives CHNS_ENOTCONV with the last iterate left in x (that iterate is checked against
the oracle's matrix: its residual is below the starting one). No kernel is made to fault."""
import numpy as np
import pytest

from gpu_common import PRM, dev, fields, meshes, oracle_operator

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2107_05123_gb300 import capi  # noqa: E402


def _rhs(om, seed):
    b = np.random.default_rng(seed).standard_normal(om.n_nodes)
    return b - b.mean()


@pytest.mark.parametrize("inner", [capi.FP64, capi.FP32])
def test_nan_in_rhs_gives_enan(inner):
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 3)
    b = _rhs(om, 4)
    b[om.n_nodes // 3] = np.nan
    x = torch.zeros(om.n_nodes, dtype=torch.float64, device="cuda")
    st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, capi.make_params(PRM),
                                capi.make_coef(dev(f["phi"])), dev(b), x,
                                capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-8, 200, 30,
                                                 inner, check_every=1), check=False)
    assert st.status == capi.ENAN
    assert "NaN" in capi.LIB.chns_last_error().decode()


@pytest.mark.parametrize("ksp,op", [(capi.KSP_CG, capi.OP_POISSON),
                                    (capi.KSP_GMRES, capi.OP_CH)])
def test_iteration_limit_gives_enotconv_with_last_iterate(ksp, op):
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 5)
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, PRM, f["phi"], f["u"], f["mu"])
    b = np.random.default_rng(6).standard_normal(nc * om.n_nodes)
    if op == capi.OP_POISSON:
        b -= b.mean()
    x = torch.zeros(nc * om.n_nodes, dtype=torch.float64, device="cuda")
    coef = capi.make_coef(dev(f["phi"]), [dev(f["u"][i]) for i in range(3)], dev(f["mu"]))
    st = capi.chns_krylov_solve(gm.handle, op, capi.make_params(PRM), coef, dev(b), x,
                                capi.make_solver(ksp, capi.PC_JACOBI, 1e-12, 3, 30, capi.FP64,
                                                 check_every=1), check=False)
    assert st.status == capi.ENOTCONV
    assert st.iterations == 3
    xh = x.cpu().numpy()
    assert np.linalg.norm(xh) > 0.0  # the last iterate is kept, not cleared
    r = np.linalg.norm(b - A @ xh) / np.linalg.norm(b)
    assert r < 1.0
    assert abs(r - st.rel_residual) <= 1e-8 * max(r, 1e-300) + 1e-12
