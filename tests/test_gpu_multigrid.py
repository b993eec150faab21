"""GPU parity of the geometric multigrid (csrc/multigrid.cu) against the oracle
(oracle/multigrid.py) through the C ABI: the level hierarchy, the transfers P and R = P^T, the
injected coefficients, the Chebyshev intervals, one V-cycle, and the flexible-CG solves with the
V-cycle preconditioner (FP64, and FP32 inside FP64 refinement) inside a solve and a time step.

Tolerances: the transfers have dyadic weights (exact in both), so they agree to the summation
order (1e-14); the V-cycle in FP64 agrees to 1e-10 (power estimates from the same integer start
vector, the coarsest solve by an explicit inverse on the GPU and an LU solve in the oracle, both
of a matrix with condition number below 1e5); solves are compared at rtol 1e-12 to 1e-8."""
import numpy as np
import pytest

from gpu_common import PRM, dev, meshes, relerr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs  # noqa: E402
from oracle import fem, multigrid as omg, solvers  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import Mesh  # noqa: E402

CASES = ["drop_l3_5", "random1", "random0_box"]


def _phi(x):
    return 1.1 * np.tanh((np.linalg.norm(x - np.array([0.5, 0.45, 0.5]), axis=1) - 0.3) / 0.06)


class _Pair:
    def __init__(self, name, degree=3, coarsest=2):
        om, gm = meshes(name)
        self.om, self.gm = om, gm
        self.oms = omg.hierarchy(om.anchors, om.levels, om.extent, coarsest_level=coarsest)
        self.mg = capi.chns_mg_create(gm.handle, coarsest_level=coarsest, degree=degree)
        self.phi = _phi(om.node_xyz)
        self.degree = degree

    def close(self):
        capi.chns_mg_destroy(self.mg)


@pytest.fixture(params=CASES)
def pair(request):
    p = _Pair(request.param)
    yield p
    p.close()


def test_hierarchy_matches_oracle(pair):
    nodes, elems = capi.chns_mg_levels(pair.mg)
    assert list(nodes) == [m.n_nodes for m in pair.oms]
    assert list(elems) == [m.n_elem for m in pair.oms]


def test_transfers_match_oracle(pair):
    rng = np.random.default_rng(5)
    for l in range(len(pair.oms) - 1):
        P = omg.prolongation(pair.oms[l], pair.oms[l + 1])
        xc = rng.standard_normal(P.shape[1])
        xf = torch.zeros(P.shape[0], dtype=torch.float64, device="cuda")
        capi.chns_mg_prolong(pair.mg, l, dev(xc), xf)
        assert relerr(xf.cpu().numpy(), P @ xc) < 1e-14
        yf = rng.standard_normal(P.shape[0])
        yc = torch.zeros(P.shape[1], dtype=torch.float64, device="cuda")
        capi.chns_mg_restrict(pair.mg, l, dev(yf), yc)
        assert relerr(yc.cpu().numpy(), P.T @ yf) < 1e-14


def test_setup_matches_oracle(pair):
    phi_d = dev(pair.phi)
    capi.chns_mg_setup(pair.mg, capi.make_params(PRM), phi_d, capi.FP64)
    B = omg.VCycle(pair.oms, PRM, pair.phi, degree=pair.degree)
    for l, m in enumerate(pair.oms):
        got = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
        capi.chns_mg_coefficient(pair.mg, l, got)
        assert np.array_equal(got.cpu().numpy(), B.phi[l])
    lam = capi.chns_mg_lambda(pair.mg, len(pair.oms), capi.FP64)
    for l in range(len(pair.oms) - 1):
        assert abs(lam[l] - B.lmax[l]) <= 1e-10 * B.lmax[l]


def test_vcycle_fp64_matches_oracle(pair):
    phi_d = dev(pair.phi)
    capi.chns_mg_setup(pair.mg, capi.make_params(PRM), phi_d, capi.FP64)
    B = omg.VCycle(pair.oms, PRM, pair.phi, degree=pair.degree)
    rng = np.random.default_rng(8)
    for _ in range(2):
        r = rng.standard_normal(pair.om.n_nodes)
        r -= r.mean()
        z = torch.zeros_like(dev(r))
        capi.chns_mg_vcycle(pair.mg, dev(r), z, capi.FP64)
        assert relerr(z.cpu().numpy(), B(r)) < 1e-10


def test_vcycle_fp32_close_to_oracle(pair):
    phi32 = dev(pair.phi, torch.float32)
    capi.chns_mg_setup(pair.mg, capi.make_params(PRM), phi32, capi.FP32)
    B = omg.VCycle(pair.oms, PRM, phi32.double().cpu().numpy(), degree=pair.degree)
    r = np.random.default_rng(9).standard_normal(pair.om.n_nodes)
    r -= r.mean()
    r32 = dev(r, torch.float32)
    z = torch.zeros_like(r32)
    capi.chns_mg_vcycle(pair.mg, r32, z, capi.FP32)
    assert relerr(z.double().cpu().numpy(), B(r32.double().cpu().numpy())) < 1e-4


@pytest.mark.parametrize("inner", [capi.FP64, capi.FP32])
def test_fcg_multigrid_solve(pair, inner):
    om, gm = pair.om, pair.gm
    A = fem.poisson(fem.Elem(om), fem.Coeffs(PRM), pair.phi)
    b = np.random.default_rng(10).standard_normal(om.n_nodes)
    b -= b.mean()
    ref, itj, _ = solvers.pcg(A, b, rtol=1e-12, mean_zero=True)
    x = torch.zeros(om.n_nodes, dtype=torch.float64, device="cuda")
    s = capi.make_solver(capi.KSP_FCG, capi.PC_MULTIGRID, 1e-12 if inner == capi.FP64 else 1e-10,
                         500, 30, inner, 1e-6, 30, check_every=1, mg=pair.mg)
    st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, capi.make_params(PRM),
                                capi.make_coef(dev(pair.phi)), dev(b), x, s)
    xh = x.cpu().numpy()
    tol = 1e-8 if inner == capi.FP64 else 1e-6
    assert relerr(xh, ref) < tol
    assert np.linalg.norm(b - A @ xh) <= (1e-12 if inner == capi.FP64 else 1e-10) * 1.01 * np.linalg.norm(b)
    assert st.iterations * 2 < itj


def test_multigrid_in_time_step_matches_jacobi():
    """One rising-drop step (levels 3-5, density ratio 1000) with the pressure Poisson solves
    preconditioned by the V-cycle agrees with the same step under Jacobi-PCG."""
    from paper_2107_05123_gb300.session import DeviceState, default_step_params
    w = configs.rising_drop(3, 5, Cn=0.04)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f0 = w.init(gm.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    mg = capi.chns_mg_create(gm.handle)
    try:
        out = {}
        for name in ("jacobi", "mg"):
            ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
            sp = default_step_params(rtol=1e-11, inner=capi.FP64)
            if name == "mg":
                sp.pp = capi.make_solver(capi.KSP_FCG, capi.PC_MULTIGRID, 1e-11, 500, 30,
                                         capi.FP64, check_every=1, mg=mg)
            st = capi.chns_step(gm.handle, ds.c, prm, sp)
            out[name] = (ds.host(), [st.pp[l].iterations for l in range(2)])
        (a, ia), (b, ib) = out["jacobi"], out["mg"]
        for k in ("phi", "mu", "p", "u"):
            assert relerr(b[k], a[k]) < 1e-8, k
        assert max(ib) * 4 < min(ia)
    finally:
        capi.chns_mg_destroy(mg)


def _h_shift(prm):
    k = 0.5 / (prm["Pe"] * prm["Cn"])
    return 1.0 / np.sqrt(prm["dt"]), prm["Cn"] * np.sqrt(k)


def test_shifted_vcycle_matches_oracle_beside_the_poisson_setup(pair):
    """The hierarchy keeps the Poisson and the shifted (sa M + sb K) setups side by side: after
    both setups each V-cycle matches its oracle cycle."""
    sa, sb = _h_shift(PRM)
    prm = capi.make_params(PRM)
    phi_d = dev(pair.phi)
    capi.chns_mg_setup(pair.mg, prm, phi_d, capi.FP64)
    capi.chns_mg_setup_shifted(pair.mg, prm, sa, sb, capi.FP64)
    Bp = omg.VCycle(pair.oms, PRM, pair.phi, degree=pair.degree)
    Bs = omg.VCycle(pair.oms, PRM, shift=(sa, sb), degree=pair.degree)
    lam = capi.chns_mg_lambda(pair.mg, len(pair.oms), capi.FP64, op=capi.MG_SHIFTED)
    for l in range(len(pair.oms) - 1):
        assert abs(lam[l] - Bs.lmax[l]) <= 1e-10 * Bs.lmax[l]
    rng = np.random.default_rng(12)
    r = rng.standard_normal(pair.om.n_nodes)
    z = torch.zeros_like(dev(r))
    capi.chns_mg_vcycle(pair.mg, dev(r), z, capi.FP64, op=capi.MG_SHIFTED)
    assert relerr(z.cpu().numpy(), Bs(r)) < 1e-10
    r -= r.mean()
    capi.chns_mg_vcycle(pair.mg, dev(r), z, capi.FP64, op=capi.MG_POISSON)
    assert relerr(z.cpu().numpy(), Bp(r)) < 1e-10


@pytest.mark.parametrize("inner", [capi.FP64, capi.FP32])
def test_schur_with_multigrid_inner_solves(inner):
    """The CH Newton system with the Schur-complement preconditioner whose H^-1 is one V-cycle:
    the solution agrees with the oracle's direct solve (FP64) or reaches the FP64 residual
    (mixed precision), in no more GMRES iterations than with 20 inner CG iterations."""
    from gpu_common import fields, oracle_operator
    stiff = dict(PRM, Cn=0.02, Pe=1.0 / (3 * 0.02 ** 2), dt=2e-2)
    om, gm = meshes("drop_l3_5")
    f = fields(om.n_nodes, 93)
    f["phi"] = np.tanh(f["phi"])
    A = oracle_operator(om, capi.OP_CH, stiff, f["phi"], f["u"], f["mu"])
    b = f["x"][:2].ravel().copy()
    coef = capi.make_coef(dev(f["phi"]), [dev(f["u"][i]) for i in range(3)], dev(f["mu"]))
    mg = capi.chns_mg_create(gm.handle)
    try:
        rtol = 1e-12 if inner == capi.FP64 else 1e-10
        its = {}
        for name, hier in (("cg", None), ("mg", mg)):
            x = torch.zeros(2 * gm.n_nodes, dtype=torch.float64, device="cuda")
            s = capi.make_solver(capi.KSP_GMRES, capi.PC_SCHUR, rtol, 2000, 30, inner, 1e-3, 40,
                                 mg=hier)
            st = capi.chns_krylov_solve(gm.handle, capi.OP_CH, capi.make_params(stiff), coef,
                                        dev(b), x, s)
            its[name] = st.iterations
            xh = x.cpu().numpy()
            assert np.linalg.norm(b - A @ xh) <= 1.05 * rtol * np.linalg.norm(b)
            if inner == capi.FP64:
                assert relerr(xh, solvers.direct(A, b)) < 1e-8
        assert its["mg"] <= its["cg"], its
    finally:
        capi.chns_mg_destroy(mg)
