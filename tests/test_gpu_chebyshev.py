"""GPU check of the Chebyshev polynomial preconditioner: solutions of the Poisson system equal
the oracle's (bordered sparse LU) within 1e-8, in fewer iterations than Jacobi-PCG."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import fem
from tests.gpu_common import PRM, dev, meshes, relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("inner", ["FP64", "FP32"])
@pytest.mark.parametrize("degree", [2, 4])
def test_chebyshev_pcg_solves_poisson(inner, degree):
    from paper_2107_05123_gb300 import capi
    om, gm = meshes("drop_l3_5")
    rng = np.random.default_rng(21)
    n = om.n_nodes
    phi = np.tanh(3.0 * rng.standard_normal(n))
    A = fem.poisson(fem.Elem(om), fem.Coeffs(PRM), phi)
    b = A @ rng.standard_normal(n)
    prm = capi.make_params(PRM)
    coef = capi.make_coef(dev(phi))
    prec = getattr(capi, inner)
    its = {}
    for pc in (capi.PC_JACOBI, capi.PC_CHEBYSHEV):
        x = dev(np.zeros(n))
        st = capi.chns_krylov_solve(gm.handle, capi.OP_POISSON, prm, coef, dev(b), x,
                                    capi.make_solver(capi.KSP_CG, pc, 1e-11, 20000, degree,
                                                     prec, 1e-4, 40, check_every=4))
        assert st.rel_residual <= 1e-11
        its[pc] = st.iterations
        xg = x.cpu().numpy()
    K = sp.bmat([[A, np.ones((n, 1))], [np.ones((1, n)), None]]).tocsc()
    xr = spl.spsolve(K, np.concatenate([b - b.mean(), [0.0]]))[:n]
    assert relerr(xg, xr) < 1e-8
    assert its[capi.PC_CHEBYSHEV] < its[capi.PC_JACOBI], its
