"""GPU parity of the learned preconditioner against oracle/learned.py: grid transfer, network
forward (bfloat16 activations, FP32 accumulation) and backward, Adam; flexible CG with the
learned correction; and the gain of a network trained on solver-generated pairs over Jacobi-PCG.

Tolerances. The network stores every activation (and, in the backward pass, every gradient
after the ReLU mask) in bfloat16, with relative spacing 2^-8. The oracle rounds the same tensors
at the same points, but it sums in FP64 where the kernels sum in FP32 in another order, so an
element whose exact value lies within ~1e-6 relative of a rounding boundary can round to the
neighbouring bfloat16 value (an error of 2^-8 on that element). A few such flips per layer move
the network's output by well under 1% in norm; the tests allow 1% (forward) and 2% (gradients,
whose chain passes through twice as many rounded tensors) in relative L2 norm."""
import numpy as np
import pytest

from chns_workloads import configs
from oracle import fem, learned as L
from tests.gpu_common import PRM, dev, meshes, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2107_05123_gb300 import capi as c
    return c


def _oracle_params(flat):
    P = L.unflatten(np.asarray(flat, dtype=np.float64))
    for name in L.LAYERS:                      # conv weights are used in bfloat16
        P[name + ".W"] = L.bf16_round(P[name + ".W"])
    return P


def _randomised_net(capi, D, seed):
    net = capi.chns_learned_create(D, 0, seed)
    p = capi.chns_learned_get_params(net)
    rng = np.random.default_rng(seed)
    P = L.unflatten(p.astype(np.float64))
    for name in L.LAYERS:
        P[name + ".b"] = 0.05 * rng.standard_normal(P[name + ".b"].shape)
    P["out.b"] = np.array([0.1])
    capi.chns_learned_set_params(net, L.flatten(P).astype(np.float32))
    return net, capi.chns_learned_get_params(net)


@pytest.mark.parametrize("D", [8, 16, 32])
def test_forward_matches_oracle(capi, D):
    import torch
    net, flat = _randomised_net(capi, D, 1)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, D, D, D)).astype(np.float32)
    out = torch.zeros(D ** 3, device="cuda", dtype=torch.float32)
    capi.chns_learned_forward(net, dev(x, torch.float32), out)
    torch.cuda.synchronize()
    ref, _ = L.forward(_oracle_params(flat), x.astype(np.float64), round_act=L.bf16_round)
    err = relerr(out.cpu().numpy(), ref.ravel())
    capi.chns_learned_destroy(net)
    assert err < 1e-2, err


@pytest.mark.parametrize("D", [8, 16])
def test_backward_matches_oracle(capi, D):
    import torch
    net, flat = _randomised_net(capi, D, 3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, D, D, D)).astype(np.float32)
    gout = (rng.standard_normal((D, D, D)) / D ** 3).astype(np.float32)
    out = torch.zeros(D ** 3, device="cuda", dtype=torch.float32)
    grad = torch.zeros(len(flat), device="cuda", dtype=torch.float32)
    capi.chns_learned_forward(net, dev(x, torch.float32), out)
    capi.chns_learned_backward(net, dev(gout, torch.float32), grad)
    torch.cuda.synchronize()
    P = _oracle_params(flat)
    _, cache = L.forward(P, x.astype(np.float64), round_act=L.bf16_round)
    G = L.backward(P, cache, gout.astype(np.float64), round_grad=L.bf16_round)
    g_gpu = L.unflatten(grad.cpu().numpy().astype(np.float64))
    capi.chns_learned_destroy(net)
    for k in G:
        assert relerr(g_gpu[k], G[k]) < 2e-2, (k, relerr(g_gpu[k], G[k]))


def test_adam_matches_oracle(capi):
    import torch
    net, flat = _randomised_net(capi, 8, 5)
    rng = np.random.default_rng(6)
    P = L.unflatten(flat.astype(np.float64))
    opt = L.Adam(P, lr=1e-3)
    for step in range(3):
        g = rng.standard_normal(len(flat)).astype(np.float32)
        capi.chns_learned_adam(net, dev(g, torch.float32), 1e-3)
        opt.step(P, L.unflatten(g.astype(np.float64)))
    torch.cuda.synchronize()
    got = capi.chns_learned_get_params(net)
    capi.chns_learned_destroy(net)
    assert relerr(got, L.flatten(P)) < 1e-6


@pytest.mark.parametrize("name", ["random0_box", "drop_l3_5"])
def test_grid_transfer_matches_oracle(capi, name):
    import torch
    om, gm = meshes(name)
    D = 16
    net = capi.chns_learned_create(D, 0, 0)
    rng = np.random.default_rng(7)
    n = om.n_nodes
    phi = 1.2 * np.tanh(2.0 * rng.standard_normal(n))
    r = rng.standard_normal(n)
    prm = capi.make_params(PRM)
    coef = capi.make_coef(dev(phi))
    x = torch.zeros(2 * D ** 3, device="cuda", dtype=torch.float32)
    s = capi.chns_learned_inputs(net, gm.handle, prm, coef, dev(r), x)
    grid = rng.standard_normal(D ** 3).astype(np.float32)
    y = torch.zeros(n, device="cuda", dtype=torch.float64)
    capi.chns_learned_prolong(net, gm.handle, dev(grid, torch.float32), y)
    torch.cuda.synchronize()
    Pg = L.grid_prolongation(om.node_int, om.extent, D)
    lr = L.cell_mean(Pg, L.log_inv_rho(fem.Coeffs(PRM), phi), D)
    xr, sr = L.restrict_inputs(Pg, r, lr, D)
    capi.chns_learned_destroy(net)
    assert abs(s - sr) <= 1e-12 * sr
    xg = x.cpu().numpy().reshape(2, D, D, D)
    assert relerr(xg[0], xr[0]) < 1e-5
    assert relerr(xg[1], xr[1]) < 1e-5
    assert relerr(y.cpu().numpy(), Pg @ grid.astype(np.float64)) < 1e-6


def test_energy_loss_matches_oracle(capi):
    """One pair through the C ABI (projection, r = A e, inputs, stored e and bfloat16
    coefficients) and the first training loss against the oracle's energy loss."""
    import torch
    om, gm = meshes("drop_l3_5")
    D = 16
    net, flat = _randomised_net(capi, D, 13)
    net2 = capi.chns_learned_create(D, 4, 13)
    capi.chns_learned_set_params(net2, flat)
    capi.chns_learned_destroy(net)
    capi.chns_learned_set_output_scale(net2, 0.05)
    rng = np.random.default_rng(14)
    n = om.n_nodes
    phi = np.tanh(2.0 * rng.standard_normal(n))
    e = rng.standard_normal(n) + 3.0
    prm = capi.make_params(PRM)
    capi.chns_learned_add_sample(net2, gm.handle, prm, capi.make_coef(dev(phi)), dev(e))
    loss = capi.chns_learned_train(net2, gm.handle, prm, 1, 1e-9, 0)
    capi.chns_learned_destroy(net2)
    co = fem.Coeffs(PRM)
    ep = e - e.mean()
    A64 = fem.poisson(fem.Elem(om), co, phi)
    r = A64 @ ep
    Pg = L.grid_prolongation(om.node_int, om.extent, D)
    x, s = L.restrict_inputs(Pg, r, L.cell_mean(Pg, L.log_inv_rho(co, phi), D), D)
    A16 = fem.poisson(fem.Elem(om), co, L.bf16_round(1.0 + phi) - 1.0)   # the loss's operator
    ref, _, _ = L.energy_loss_and_grad(_oracle_params(flat), Pg, A16, ep, x, s, D, 0.05,
                                       round_act=L.bf16_round)
    assert abs(loss[0] - ref) <= 2e-2 * ref, (loss[0], ref)


def _poisson_system(om, seed):
    rng = np.random.default_rng(seed)
    n = om.n_nodes
    phi = np.tanh(3.0 * rng.standard_normal(n))
    A = fem.poisson(fem.Elem(om), fem.Coeffs(PRM), phi)
    b = A @ rng.standard_normal(n)
    return phi, A, b


def test_fcg_with_jacobi_equals_pcg(capi):
    """Flexible CG with a fixed SPD preconditioner generates the PCG iterates."""
    om, gm = meshes("random1")
    phi, A, b = _poisson_system(om, 8)
    prm = capi.make_params(PRM)
    coef = capi.make_coef(dev(phi))
    its = {}
    for ksp in (capi.KSP_CG, capi.KSP_FCG):
        x = dev(np.zeros(om.n_nodes))
        st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, prm, coef, dev(b), x,
                                    capi.make_solver(ksp, capi.PC_JACOBI, 1e-10, 5000))
        its[ksp] = st.iterations
    assert abs(its[capi.KSP_CG] - its[capi.KSP_FCG]) <= 1, its


@pytest.mark.parametrize("inner", ["FP64", "FP32"])
def test_fcg_learned_solution_matches_oracle(capi, inner):
    """Whatever the network, FCG with the learned correction converges to the oracle's solution
    (convergence is decided by the unchanged residual tolerance)."""
    import scipy.sparse.linalg as spl
    om, gm = meshes("drop_l3_5")
    phi, A, b = _poisson_system(om, 9)
    prm = capi.make_params(PRM)
    coef = capi.make_coef(dev(phi))
    net = capi.chns_learned_create(16, 0, 11)
    capi.chns_learned_set_output_scale(net, 1e-2)
    x = dev(np.zeros(om.n_nodes))
    prec = getattr(capi, inner)
    st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, prm, coef, dev(b), x,
                                capi.make_solver(capi.KSP_FCG, capi.PC_LEARNED, 1e-11, 5000, 30,
                                                 prec, 1e-4, 40, check_every=4, learned=net))
    xg = x.cpu().numpy()
    capi.chns_learned_destroy(net)
    bm = b - b.mean()
    n = om.n_nodes
    # pure Neumann: pin the mean through a bordered system
    import scipy.sparse as sp
    K = sp.bmat([[A, np.ones((n, 1))], [np.ones((1, n)), None]]).tocsc()
    xr = spl.spsolve(K, np.concatenate([bm, [0.0]]))[:n]
    assert st.rel_residual <= 1e-11
    assert relerr(xg, xr) < 1e-8


def test_trained_network_reduces_iterations(capi):
    """Train on pairs from Jacobi-PCG solves of seeded right-hand sides on a drop octree, then
    compare FCG + learned correction with Jacobi-PCG on unseen right-hand sides."""
    import torch
    w = configs.many_drops(seed=3, n=4, lmin=3, lmax=6, Cn=0.02)
    from paper_2107_05123_gb300.session import Mesh
    gm = Mesh(w.anchors, w.levels)
    init = w.init(gm.node_xyz)
    prm_d = w.params.as_dict()
    prm = capi.make_params(prm_d)
    phi = dev(init["phi"])
    coef = capi.make_coef(phi)
    n = gm.n_nodes
    D = 32
    net = capi.chns_learned_create(D, 512, 5)
    rng = np.random.default_rng(12)

    def rhs():
        # smooth random right-hand sides: low Fourier modes at the nodes, mean-free
        xyz = gm.node_xyz
        f = np.zeros(n)
        for _ in range(6):
            k = rng.integers(1, 4, size=3)
            f += rng.standard_normal() * np.cos(np.pi * (k * xyz).sum(axis=1) + rng.uniform(0, 6.3))
        return f - f.mean()

    for _ in range(16):
        capi.chns_learned_collect(net, gm.handle, prm, coef, dev(rhs()), 4, 32)
    assert capi.chns_learned_num_samples(net) >= 64
    loss = capi.chns_learned_train(net, gm.handle, prm, 1500, 1e-3, 1)
    # the energy loss starts at 1 (zero output layer: c = 0)
    assert np.mean(loss[-100:]) < 0.7 * np.mean(loss[:20]), (loss[:20].mean(), loss[-100:].mean())
    its_j, its_l = [], []
    for _ in range(3):
        b = dev(rhs())
        for pc, lst, ksp in ((capi.PC_JACOBI, its_j, capi.KSP_CG),
                             (capi.PC_LEARNED, its_l, capi.KSP_FCG)):
            x = torch.zeros(n, device="cuda", dtype=torch.float64)
            st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, prm, coef, b, x,
                                        capi.make_solver(ksp, pc, 1e-8, 20000, 30, capi.FP64,
                                                         check_every=1, learned=net))
            assert st.rel_residual <= 1e-8
            lst.append(st.iterations)
    capi.chns_learned_destroy(net)
    print("Jacobi-PCG", its_j, "FCG + learned", its_l)
    assert np.mean(its_l) < 0.8 * np.mean(its_j), (its_j, its_l)


def test_step_collection_adds_pairs_and_leaves_the_step_unchanged(capi):
    """chns_step with chns_step_params.collect: every pressure solve adds its pairs, and the
    fields after the step equal those of the same step without collection."""
    from paper_2107_05123_gb300.session import DeviceState, default_step_params
    w = configs.rising_drop(3, 5, Cn=0.04)
    om, gm = meshes("drop_l3_5")
    f0 = w.init(gm.node_xyz)
    prm = capi.make_params(w.params.as_dict())
    net = capi.chns_learned_create(16, 64, 2)
    out = {}
    for collect in (False, True):
        ds = DeviceState(dict(phi=f0["phi"], mu=f0["mu"], u=f0["u"], p=f0["p"]))
        sp = default_step_params(1e-10, capi.FP64, 8)
        if collect:
            sp.collect, sp.collect_every, sp.collect_max = net, 4, 5
        capi.chns_step(gm.handle, ds.c, prm, sp)
        out[collect] = ds.host()
    n_pairs = capi.chns_learned_num_samples(net)
    capi.chns_learned_destroy(net)
    assert 2 <= n_pairs <= 10, n_pairs
    for k in ("phi", "mu", "u", "p"):
        assert relerr(out[True][k], out[False][k]) < 1e-9, k
