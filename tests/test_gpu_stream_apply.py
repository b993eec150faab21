"""GPU parity of the persistent, pipelined patch apply (CHNS_APPLY_STREAM) against the oracle.

Small grids (1, 3, 7 CTAs) make every CTA walk several patches, so the three-stage pipeline
(slot table of patch k+2, node values of patch k+1, compute of patch k) and its buffer rotation
run on meshes the oracle assembles in seconds; max_ctas = 0 gives one patch per CTA. The FP32
applies are compared with the oracle evaluated on the same FP32-rounded inputs (1e-5, as for the
per-patch kernel), and the two kernels with each other (1e-6: only the order of additions into
shared nodes differs)."""
import numpy as np
import pytest

from gpu_common import LEAVES, PRM, dev, f32_round, fields, oracle_operator, relerr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import Mesh  # noqa: E402
from oracle.mesh import Mesh as OMesh  # noqa: E402

APPLY = {capi.OP_POISSON: capi.chns_apply_poisson, capi.OP_MASS: capi.chns_apply_mass}


def _pair(name):
    f, ext = LEAVES[name]
    a, l = f()
    return OMesh(a, l, ext), Mesh(a, l, ext)


def _apply(gm, op, ph, x, kernel, max_ctas):
    capi.chns_mesh_set_apply_config(gm.handle, kernel, max_ctas)
    nc = capi.OP_NCOMP[op]
    y = torch.zeros(nc * gm.n_nodes, dtype=torch.float32, device="cuda")
    APPLY[op](gm.handle, capi.make_params(PRM), capi.make_coef(ph), dev(x, torch.float32), y,
              capi.FP32)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("op", [capi.OP_POISSON, capi.OP_MASS])
@pytest.mark.parametrize("name", ["random1", "drop_l3_5", "random0_box"])
def test_stream_apply_matches_oracle(name, op):
    om, gm = _pair(name)
    f = fields(om.n_nodes, 71 + op)
    nc = capi.OP_NCOMP[op]
    x = f32_round(f["x"][:nc].ravel())
    phi = f32_round(f["phi"])
    A = oracle_operator(om, op, PRM, phi, f["u"], f["mu"])
    ref = A @ x
    ph = dev(phi, torch.float32)
    y_patch = _apply(gm, op, ph, x, capi.APPLY_PATCH, 0)
    assert relerr(y_patch, ref) < 1e-5
    for max_ctas in (1, 3, 7, 0):
        y = _apply(gm, op, ph, x, capi.APPLY_STREAM, max_ctas)
        assert relerr(y, ref) < 1e-5, max_ctas
        assert relerr(y, y_patch) < 1e-6, max_ctas
    gm.close()


@pytest.mark.parametrize("max_ctas", [1, 5])
def test_stream_cg_reaches_fp64_residual(max_ctas):
    """The pressure solve with the CG update fused into the pipelined apply (FP32 inner CG,
    FP64 refinement) reaches the FP64 residual the oracle's matrix confirms, and agrees with the
    oracle's solution."""
    from oracle import solvers
    om, gm = _pair("drop_l3_5")
    capi.chns_mesh_set_apply_config(gm.handle, capi.APPLY_STREAM, max_ctas)
    f = fields(om.n_nodes, 81)
    f["phi"] = np.tanh(f["phi"])
    A = oracle_operator(om, capi.OP_POISSON, PRM, f["phi"])
    b = f["x"][0].copy()
    b -= b.mean()
    ref, _, _ = solvers.pcg(A, b, rtol=1e-13, mean_zero=True)
    x = torch.zeros(gm.n_nodes, dtype=torch.float64, device="cuda")
    s = capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-10, 20000, 30,
                         inner_precision=capi.FP32, inner_rtol=1e-6, check_every=8)
    st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, capi.make_params(PRM),
                                capi.make_coef(dev(f["phi"])), dev(b), x, s)
    xs = x.cpu().numpy()
    assert st.refinements >= 1
    assert np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1.05e-10
    xs = xs - xs.mean()
    assert relerr(xs, ref - ref.mean()) < 1e-8
    gm.close()


def test_apply_config_rejects_bad_arguments():
    om, gm = _pair("uniform2")
    with pytest.raises(Exception):
        capi.chns_mesh_set_apply_config(gm.handle, 7, 0)
    with pytest.raises(Exception):
        capi.chns_mesh_set_apply_config(gm.handle, capi.APPLY_STREAM, -1)
    capi.chns_mesh_set_apply_config(gm.handle, capi.APPLY_AUTO, 0)
    gm.close()
