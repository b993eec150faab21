"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded
inputs. Tolerances: FP64 applies and right-hand sides 1e-12 (relative 2-norm); FP64 solves
compared at rtol 1e-12 on both sides to 1e-8; FP32 applies against the oracle evaluated on the
FP32/BF16-rounded inputs to 1e-5 (a few hundred FP32 operations per entry, unit roundoff 6e-8)."""
import numpy as np
import pytest

from gpu_common import (PRM, SMALL, bf16_round, dev, f32_round, fields, meshes, oracle_operator,
                        relerr)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2107_05123_gb300 import capi  # noqa: E402
from oracle import fem, solvers  # noqa: E402

OPS = [capi.OP_POISSON, capi.OP_MASS, capi.OP_CH, capi.OP_MOMENTUM]
APPLY = {capi.OP_POISSON: capi.chns_apply_poisson, capi.OP_MASS: capi.chns_apply_mass,
         capi.OP_CH: capi.chns_apply_ch, capi.OP_MOMENTUM: capi.chns_apply_momentum}


@pytest.mark.parametrize("name", SMALL)
def test_mesh_matches_oracle(name):
    om, gm = meshes(name)
    assert gm.n_elem == om.n_elem
    assert gm.n_nodes == om.n_nodes
    assert gm.n_hanging == om.n_hanging
    assert np.array_equal(gm.node_int.astype(np.int64), om.node_int)
    assert np.array_equal(gm.boundary, om.boundary)


def _coef(f, dtype):
    return [dev(f["phi"], dtype), [dev(f["u"][i], dtype) for i in range(3)], dev(f["mu"], dtype)]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("name", SMALL)
def test_apply_fp64(name, op):
    om, gm = meshes(name)
    f = fields(om.n_nodes, 11 + op)
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, PRM, f["phi"], f["u"], f["mu"])
    x = f["x"][:nc].ravel()
    ph, u, mu = _coef(f, torch.float64)
    y = torch.zeros(nc * gm.n_nodes, dtype=torch.float64, device="cuda")
    APPLY[op](gm.handle, capi.make_params(PRM), capi.make_coef(ph, u, mu), dev(x), y)
    assert relerr(y.cpu().numpy(), A @ x) < 1e-12


@pytest.mark.parametrize("prec", [capi.FP32, capi.FP32_BF16COEF])
@pytest.mark.parametrize("op", OPS)
def test_apply_reduced_precision(op, prec):
    """The oracle sees exactly the rounded inputs the kernel sees. In BF16 coefficient storage the
    phase field is stored as bfloat16(1 + phi~) (the C ABI's convention)."""
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 21 + op)
    nc = capi.OP_NCOMP[op]
    x = f32_round(f["x"][:nc].ravel())
    if prec == capi.FP32_BF16COEF:
        s16 = bf16_round(1.0 + f["phi"])
        phi, u, mu = s16 - 1.0, bf16_round(f["u"]), bf16_round(f["mu"])
        cdt, ph = torch.bfloat16, dev(s16).to(torch.bfloat16)
    else:
        phi, u, mu = f32_round(f["phi"]), f32_round(f["u"]), f32_round(f["mu"])
        cdt, ph = torch.float32, dev(phi).to(torch.float32)
    A = oracle_operator(om, op, PRM, phi, u, mu)
    uu = [dev(u[i]).to(cdt) for i in range(3)]
    mm = dev(mu).to(cdt)
    y = torch.zeros(nc * gm.n_nodes, dtype=torch.float32, device="cuda")
    APPLY[op](gm.handle, capi.make_params(PRM), capi.make_coef(ph, uu, mm),
              dev(x, torch.float32), y, prec)
    assert relerr(y.double().cpu().numpy(), A @ x) < 1e-5


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("name", ["one_refined", "random1", "drop_l3_5"])
def test_diagonal_fp64(name, op):
    om, gm = meshes(name)
    f = fields(om.n_nodes, 31 + op)
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, PRM, f["phi"], f["u"], f["mu"])
    ph, u, mu = _coef(f, torch.float64)
    d = torch.zeros(nc * gm.n_nodes, dtype=torch.float64, device="cuda")
    capi.chns_operator_diagonal(gm.handle, op, capi.make_params(PRM), capi.make_coef(ph, u, mu), d)
    assert relerr(d.cpu().numpy(), A.diagonal()) < 1e-12


@pytest.mark.parametrize("name", ["random0_box", "drop_l3_5"])
def test_rhs_fp64(name):
    om, gm = meshes(name)
    N = om.n_nodes
    rng = np.random.default_rng(41)
    el, co = fem.Elem(om), fem.Coeffs(PRM)
    phi, phik = 1.2 * np.tanh(rng.standard_normal(N)), np.tanh(rng.standard_normal(N))
    mu, muk = rng.standard_normal(N), rng.standard_normal(N)
    u, uk, v = (rng.standard_normal((3, N)) for _ in range(3))
    pk, pn = rng.standard_normal(N), rng.standard_normal(N)
    prm = capi.make_params(PRM)
    # CH residual
    f = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    capi.chns_residual_ch(gm.handle, prm, dev(phi), dev(mu), dev(phik), dev(muk),
                          [dev(u[i]) for i in range(3)], f)
    fp, fm = fem.ch_residual(el, co, phi, mu, phik, muk, u)
    assert relerr(f.cpu().numpy(), np.concatenate([fp, fm])) < 1e-12
    # VMS right-hand sides
    vs = fem.VMSState(el, co, phi, u, mu)
    coef = capi.make_coef(dev(phi), [dev(u[i]) for i in range(3)], dev(mu))
    ukd = [dev(uk[i]) for i in range(3)]
    vd = [dev(v[i]) for i in range(3)]
    b = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    capi.chns_rhs_momentum(gm.handle, prm, coef, ukd, dev(pk), b)
    ref = fem.vp_rhs(vs, uk, pk)
    ref[:, om.boundary] = 0.0
    assert relerr(b.cpu().numpy(), ref.ravel()) < 1e-12
    bp = torch.zeros(N, dtype=torch.float64, device="cuda")
    capi.chns_rhs_poisson(gm.handle, prm, coef, vd, ukd, dev(pk), bp)
    assert relerr(bp.cpu().numpy(), fem.pp_rhs(vs, v, uk, pk)) < 1e-12
    capi.chns_rhs_velocity_update(gm.handle, prm, coef, vd, ukd, dev(pk), dev(pn), b)
    ref = fem.vu_rhs(vs, v, uk, pk, pn)
    ref[:, om.boundary] = 0.0
    assert relerr(b.cpu().numpy(), ref.ravel()) < 1e-12
    # phi mass
    assert abs(capi.chns_phi_mass(gm.handle, dev(phi)) - fem.phi_mass(el, phi)) < 1e-12


@pytest.mark.parametrize("op,ksp", [(capi.OP_POISSON, capi.KSP_CG), (capi.OP_MASS, capi.KSP_CG),
                                    (capi.OP_CH, capi.KSP_GMRES),
                                    (capi.OP_MOMENTUM, capi.KSP_GMRES)])
def test_solve_fp64(op, ksp):
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 51 + op)
    f["phi"] = np.tanh(f["phi"])
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, PRM, f["phi"], f["u"], f["mu"])
    b = f["x"][:nc].ravel().copy()
    if op in (capi.OP_MASS, capi.OP_MOMENTUM):
        b.reshape(nc, -1)[:, om.boundary] = 0.0
    if op == capi.OP_POISSON:
        ref, _, _ = solvers.pcg(A, b, rtol=1e-13, mean_zero=True)
    else:
        ref = solvers.direct(A, b)
    x = torch.zeros(nc * gm.n_nodes, dtype=torch.float64, device="cuda")
    s = capi.make_solver(ksp, capi.PC_JACOBI, 1e-12, 20000, 30)
    st = capi.chns_krylov_solve(gm.handle, op, capi.make_params(PRM),
                                capi.make_coef(*_coef(f, torch.float64)), dev(b), x, s)
    assert st.rel_residual <= 1e-12
    assert relerr(x.cpu().numpy(), ref) < 1e-8


@pytest.mark.parametrize("inner", [capi.FP32, capi.FP32_BF16COEF])
@pytest.mark.parametrize("op,ksp", [(capi.OP_POISSON, capi.KSP_CG), (capi.OP_CH, capi.KSP_GMRES),
                                    (capi.OP_MOMENTUM, capi.KSP_GMRES)])
def test_solve_mixed_precision_reaches_fp64_residual(op, ksp, inner):
    """FP32 inner Krylov + FP64 refinement: the oracle's own matrix confirms ||b - A x|| / ||b||."""
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 61 + op)
    f["phi"] = np.tanh(f["phi"])
    nc = capi.OP_NCOMP[op]
    A = oracle_operator(om, op, PRM, f["phi"], f["u"], f["mu"])
    b = f["x"][:nc].ravel().copy()
    if op in (capi.OP_MASS, capi.OP_MOMENTUM):
        b.reshape(nc, -1)[:, om.boundary] = 0.0
    if op == capi.OP_POISSON:
        b -= b.mean()
    x = torch.zeros(nc * gm.n_nodes, dtype=torch.float64, device="cuda")
    s = capi.make_solver(ksp, capi.PC_JACOBI, 1e-10, 20000, 30, inner, 1e-3, 30)
    st = capi.chns_krylov_solve(gm.handle, op, capi.make_params(PRM),
                                capi.make_coef(*_coef(f, torch.float64)), dev(b), x, s)
    xs = x.cpu().numpy()
    assert st.refinements >= 1
    assert np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1.05e-10
