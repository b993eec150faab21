"""GPU parity at the sizes and physics the bench runs (through the C ABI, against the oracle).

* the rising-drop mesh of the bench (levels 5-8, 314,672 leaves): mesh tables bit-exact; the four
  FP64 applies (1e-12) and FP32 applies with the launch
  configuration chosen automatically, on the workload's physics (density ratio 1000, viscosity
  ratio 100, Cn 0.01, We 1); one pressure-Poisson solve (1e-8);
* the Rayleigh-Taylor mesh on levels 6-9 (1.43e6 leaves, the bench workload one level coarser):
  mesh tables bit-exact and the FP32 Poisson apply, where the automatic choice is the
  persistent pipelined kernel (at least 16 patches per SM), against the oracle's matrix;
* one time step with the rising drop's parameters (Cn 0.01, density ratio 1000) on a levels 3-5
  drop, against the oracle's step (1e-8 per field, FP64).
The oracle assembles every matrix on the host (tens of seconds at these sizes).

FP32 applies are compared on the FP32-rounded inputs against the floating-point bound of a sum of
products, || y - A x || <= 1e-5 || |A| |x| ||: with density ratio 1000 the coefficient 1/rho spans
three decades, the rows of the Poisson operator cancel, and the error relative to || A x || alone
reaches 1.5e-5 although each entry is within a few hundred FP32 roundings of its terms."""
import functools

import numpy as np
import pytest

from gpu_common import dev, f32_round, oracle_operator, relerr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs  # noqa: E402
from oracle import fem, solvers, step as ostep  # noqa: E402
from oracle.mesh import Mesh as OMesh  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import DeviceState, Mesh, default_step_params  # noqa: E402

OPS = [capi.OP_POISSON, capi.OP_MASS, capi.OP_CH, capi.OP_MOMENTUM]
APPLY = {capi.OP_POISSON: capi.chns_apply_poisson, capi.OP_MASS: capi.chns_apply_mass,
         capi.OP_CH: capi.chns_apply_ch, capi.OP_MOMENTUM: capi.chns_apply_momentum}


@functools.lru_cache(maxsize=None)
def _drop():
    w = configs.rising_drop(5, 8)
    om = OMesh(w.anchors, w.levels, w.extent)
    gm = Mesh(w.anchors, w.levels, w.extent)
    return w, om, gm


@functools.lru_cache(maxsize=None)
def _fields(n_seed):
    w, om, gm = _drop()
    rng = np.random.default_rng(n_seed)
    f0 = w.init(om.node_xyz)
    # the drop's phase and chemical potential, a small seeded velocity
    return dict(phi=f0["phi"], mu=f0["mu"], u=0.05 * rng.standard_normal((3, om.n_nodes)),
                x=rng.standard_normal((3, om.n_nodes)))


def _check_mesh(om, gm):
    assert gm.n_elem == om.n_elem and gm.n_nodes == om.n_nodes
    assert gm.n_hanging == om.n_hanging
    assert np.array_equal(gm.node_int.astype(np.int64), om.node_int)
    assert np.array_equal(gm.boundary, om.boundary)


def test_drop_mesh_matches_oracle():
    w, om, gm = _drop()
    assert gm.n_elem == 314672
    _check_mesh(om, gm)


@pytest.mark.parametrize("op", OPS)
def test_drop_applies_fp64_and_fp32(op):
    w, om, gm = _drop()
    prm = w.params.as_dict()
    f = _fields(40 + op)
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, prm, f["phi"], f["u"], f["mu"])
    x = f["x"][:nc].ravel()
    coef = capi.make_coef(dev(f["phi"]), [dev(f["u"][i]) for i in range(3)], dev(f["mu"]))
    y = torch.zeros(nc * gm.n_nodes, dtype=torch.float64, device="cuda")
    APPLY[op](gm.handle, capi.make_params(prm), coef, dev(x), y, capi.FP64)
    assert relerr(y.cpu().numpy(), A @ x) < 1e-12
    # FP32 on the rounded inputs
    phi32, u32, mu32 = f32_round(f["phi"]), f32_round(f["u"]), f32_round(f["mu"])
    A32 = oracle_operator(om, op, prm, phi32, u32, mu32)
    x32 = f32_round(x)
    c32 = capi.make_coef(dev(phi32, torch.float32), [dev(u32[i], torch.float32) for i in range(3)],
                         dev(mu32, torch.float32))
    y32 = torch.zeros(nc * gm.n_nodes, dtype=torch.float32, device="cuda")
    APPLY[op](gm.handle, capi.make_params(prm), c32, dev(x32, torch.float32), y32, capi.FP32)
    assert _fp32_err(y32, A32, x32) < 1e-5


def _fp32_err(y, A, x):
    y = y.double().cpu().numpy()
    return float(np.linalg.norm(y - A @ x) / np.linalg.norm(abs(A) @ abs(x)))


def test_drop_pressure_solve_matches_oracle():
    w, om, gm = _drop()
    prm = w.params.as_dict()
    f = _fields(50)
    el, co = fem.Elem(om), fem.Coeffs(prm)
    z = np.zeros((3, om.n_nodes))
    b = fem.pp_rhs(fem.VMSState(el, co, f["phi"], z, f["mu"]), f["u"], z, np.zeros(om.n_nodes))
    A = fem.poisson(el, co, f["phi"])
    ref, _, _ = solvers.pcg(A, b, rtol=1e-12, mean_zero=True)
    x = torch.zeros(gm.n_nodes, dtype=torch.float64, device="cuda")
    st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, capi.make_params(prm),
                                capi.make_coef(dev(f["phi"])), dev(b), x,
                                capi.make_solver(capi.KSP_CG, capi.PC_JACOBI, 1e-12, 20000, 30,
                                                 check_every=8))
    assert st.status == capi.OK
    assert relerr(x.cpu().numpy(), ref) < 1e-8


def test_rayleigh_taylor_levels_6_9_mesh_and_pipelined_poisson_apply():
    w = configs.rayleigh_taylor(6, 9, 0.005)
    om = OMesh(w.anchors, w.levels, w.extent)
    gm = Mesh(w.anchors, w.levels, w.extent)
    _check_mesh(om, gm)
    prm = w.params.as_dict()
    phi = f32_round(w.init(om.node_xyz)["phi"])
    x = f32_round(np.random.default_rng(60).standard_normal(om.n_nodes))
    A = fem.poisson(fem.Elem(om), fem.Coeffs(prm), phi)
    y = torch.zeros(gm.n_nodes, dtype=torch.float32, device="cuda")
    capi.chns_mesh_set_apply_config(gm.handle, capi.APPLY_AUTO, 0)
    capi.chns_apply_poisson(gm.handle, capi.make_params(prm), capi.make_coef(dev(phi, torch.float32)),
                            dev(x, torch.float32), y, capi.FP32)
    assert _fp32_err(y, A, x) < 1e-5
    # the same through the one-CTA-per-patch kernel
    y2 = torch.zeros_like(y)
    capi.chns_mesh_set_apply_config(gm.handle, capi.APPLY_PATCH, 0)
    capi.chns_apply_poisson(gm.handle, capi.make_params(prm), capi.make_coef(dev(phi, torch.float32)),
                            dev(x, torch.float32), y2, capi.FP32)
    assert _fp32_err(y2, A, x) < 1e-5


def test_step_with_rising_drop_parameters_matches_oracle():
    w = configs.rising_drop(3, 5)  # Cn 0.01, density ratio 1000, viscosity ratio 100, We 1
    om = OMesh(w.anchors, w.levels, w.extent)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(om.node_xyz)
    prm = w.params.as_dict()
    ref = ostep.chns_step(om, prm, ostep.State(phi=f["phi"], mu=f["mu"], u=f["u"], u_old=f["u"],
                                               p=f["p"]), newton_rtol=1e-13)
    ds = DeviceState(dict(phi=f["phi"], mu=f["mu"], u=f["u"], p=f["p"]))
    st = capi.chns_step(gm.handle, ds.c, capi.make_params(prm),
                        default_step_params(rtol=1e-12, newton_rtol=1e-13))
    got = ds.host()
    for k in ("phi", "mu", "u"):
        assert relerr(got[k], getattr(ref, k)) < 1e-8, k
    assert relerr(got["p"] - got["p"].mean(), ref.p - ref.p.mean()) < 1e-8
    assert abs(st.phi_mass_after - st.phi_mass_before) < 1e-11
