"""Operator applies in double-float arithmetic (CHNS_FP64_DF: FP64 arrays, the Poisson and mass
element arithmetic in pairs of FP32 numbers; the CH and momentum applies stay FP64) against the
oracle, solves whose refinement residuals use them, and a time step with them in the pressure
and velocity-update solves. Double-float operations carry relative errors of about 1e-14
(measured on the CPU with the same algorithms: addition 6e-15 of |a| + |b|, product 1.3e-14,
reciprocal 1.2e-14, reciprocal square root 4e-14), so the apply bound is 1e-11 (FP64: 1e-12)."""
import numpy as np
import pytest

from gpu_common import PRM, dev, fields, meshes, oracle_operator, relerr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs  # noqa: E402
from oracle import step as ostep  # noqa: E402
from oracle.mesh import Mesh as OMesh  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import DeviceState, Mesh, default_step_params  # noqa: E402

OPS = [capi.OP_POISSON, capi.OP_MASS, capi.OP_CH, capi.OP_MOMENTUM]
APPLY = {capi.OP_POISSON: capi.chns_apply_poisson, capi.OP_MASS: capi.chns_apply_mass,
         capi.OP_CH: capi.chns_apply_ch, capi.OP_MOMENTUM: capi.chns_apply_momentum}


@pytest.mark.parametrize("op", OPS)
def test_double_float_applies_match_oracle(op):
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 31 + op)
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, PRM, f["phi"], f["u"], f["mu"])
    x = f["x"][:nc].ravel()
    coef = capi.make_coef(dev(f["phi"]), [dev(f["u"][i]) for i in range(3)], dev(f["mu"]))
    y = torch.zeros(nc * gm.n_nodes, dtype=torch.float64, device="cuda")
    APPLY[op](gm.handle, capi.make_params(PRM), coef, dev(x), y, capi.FP64_DF)
    assert relerr(y.cpu().numpy(), A @ x) < 1e-11


@pytest.mark.parametrize("op", [capi.OP_POISSON, capi.OP_MASS])
def test_solves_with_double_float_refinement_reach_the_fp64_residual(op):
    """Mixed-precision CG whose refinement residuals use the double-float applies reaches the
    relative residual 1e-10 measured with the oracle's matrix."""
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 41 + op)
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, PRM, f["phi"], f["u"], f["mu"])
    b = A @ f["x"][:nc].ravel()
    coef = capi.make_coef(dev(f["phi"]), [dev(f["u"][i]) for i in range(3)], dev(f["mu"]))
    x = torch.zeros(nc * gm.n_nodes, dtype=torch.float64, device="cuda")
    s = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-10, 20000, 30, capi.FP32, 1e-6,
                         fp64_apply=capi.FP64_DF)
    st = capi.chns_krylov_solve(gm.handle, op, capi.make_params(PRM), coef, dev(b), x, s)
    r = b - A @ x.cpu().numpy()
    if op == capi.OP_POISSON:
        r = r - r.mean()
    assert st.refinements >= 1
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)


def test_step_with_double_float_refinement_matches_oracle():
    w = configs.rising_drop(3, 5)  # density ratio 1000, viscosity ratio 100, Cn 0.01, We 1
    om = OMesh(w.anchors, w.levels, w.extent)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(om.node_xyz)
    prm = w.params.as_dict()
    ref = ostep.chns_step(om, prm, ostep.State(phi=f["phi"], mu=f["mu"], u=f["u"], u_old=f["u"],
                                               p=f["p"]), newton_rtol=1e-13)
    ds = DeviceState(dict(phi=f["phi"], mu=f["mu"], u=f["u"], p=f["p"]))
    sp = default_step_params(rtol=1e-12, newton_rtol=1e-13, inner=capi.FP32)
    sp.pp.fp64_apply = capi.FP64_DF
    sp.vu.fp64_apply = capi.FP64_DF
    capi.chns_step(gm.handle, ds.c, capi.make_params(prm), sp)
    got = ds.host()
    for k in ("phi", "mu", "u"):
        assert relerr(got[k], getattr(ref, k)) < 1e-8, k
    assert relerr(got["p"] - got["p"].mean(), ref.p - ref.p.mean()) < 1e-8


def test_unknown_fp64_apply_precision_is_rejected():
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 51)
    coef = capi.make_coef(dev(f["phi"]))
    b = torch.ones(gm.n_nodes, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    s = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-8, 100, 30, capi.FP32, 1e-6,
                         fp64_apply=capi.FP32)
    with pytest.raises(capi.ChnsError):
        capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, capi.make_params(PRM), coef, b, x, s)
