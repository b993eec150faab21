"""GPU parity of a time step with velocity Dirichlet data (the walls move; the breakup workload's
shear): the step lifts the data into the velocity-prediction and velocity-update right-hand sides
(b - A g on the interior rows, g on the boundary rows) and matches the oracle's step, which
eliminates the boundary columns of its assembled matrices with the same data (1e-8 per field,
FP64). Zero data reproduces the no-slip step."""
import numpy as np
import pytest

from gpu_common import relerr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs  # noqa: E402
from oracle import step as ostep  # noqa: E402
from oracle.mesh import Mesh as OMesh  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import (DeviceState, Mesh, VelocityBC,  # noqa: E402
                                             default_step_params)

# a divergence-free linear field (trace zero) with all three components non-zero on the walls
A_LIN = np.array([[0.3, 1.0, 0.2], [0.1, -0.5, 0.4], [-0.3, 0.2, 0.2]])


def _linear(x, t=0.0):
    return A_LIN @ (x - 0.5).T


def _gpu_step(w, gm, f, prm, g=None, inner=capi.FP64):
    ds = DeviceState(dict(phi=f["phi"], mu=f["mu"], u=f["u"], p=f["p"]))
    sp = default_step_params(rtol=1e-12, newton_rtol=1e-13, inner=inner)
    bc = None
    if g is not None:
        bc = VelocityBC(g)
        bc.attach(sp)
    st = capi.chns_step(gm.handle, ds.c, capi.make_params(prm), sp)
    torch.cuda.synchronize()
    return ds.host(), st


@pytest.mark.parametrize("field", ["linear", "shear"])
def test_step_with_velocity_dirichlet_data_matches_oracle(field):
    w = configs.rising_drop(3, 5)
    om = OMesh(w.anchors, w.levels, w.extent)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(om.node_xyz)
    bc_fn = _linear if field == "linear" else (lambda x, t: configs.shear_velocity(x))
    f["u"] = bc_fn(om.node_xyz, 0.0)
    prm = w.params.as_dict()
    ref = ostep.chns_step(om, prm, ostep.State(phi=f["phi"], mu=f["mu"], u=f["u"], u_old=f["u"],
                                               p=f["p"]), newton_rtol=1e-13, velocity_bc=bc_fn)
    got, st = _gpu_step(w, gm, f, prm, g=bc_fn(om.node_xyz, prm["dt"]))
    for k in ("phi", "mu", "u"):
        assert relerr(got[k], getattr(ref, k)) < 1e-8, k
    assert relerr(got["p"] - got["p"].mean(), ref.p - ref.p.mean()) < 1e-8
    # the data holds on the boundary exactly
    b = gm.boundary
    g = bc_fn(om.node_xyz, prm["dt"])
    assert np.array_equal(got["u"][:, b], g[:, b])


def test_zero_velocity_data_is_no_slip():
    w = configs.rising_drop(3, 5)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(gm.node_xyz)
    prm = w.params.as_dict()
    a, _ = _gpu_step(w, gm, f, prm)
    b, _ = _gpu_step(w, gm, f, prm, g=np.zeros((3, gm.n_nodes)))
    for k in ("phi", "mu", "u", "p"):
        assert relerr(b[k], a[k]) < 1e-12, k


def test_mixed_precision_step_with_shear_data():
    """The FP32 inner solves with FP64 refinement under the shear reach the FP64 step's fields
    within the refinement tolerance."""
    w = configs.rising_drop(3, 5)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(gm.node_xyz)
    f["u"] = configs.shear_velocity(gm.node_xyz)
    prm = w.params.as_dict()
    g = configs.shear_velocity(gm.node_xyz)
    a, _ = _gpu_step(w, gm, f, prm, g=g)
    b, st = _gpu_step(w, gm, f, prm, g=g, inner=capi.FP32)
    assert max(st.vp[1].refinements, st.vu[1].refinements) >= 1
    for k in ("phi", "mu", "u"):
        assert relerr(b[k], a[k]) < 1e-8, k


def test_partial_velocity_data_is_rejected():
    w = configs.rising_drop(3, 5)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(gm.node_xyz)
    ds = DeviceState(dict(phi=f["phi"], mu=f["mu"], u=f["u"], p=f["p"]))
    sp = default_step_params()
    g = torch.zeros(gm.n_nodes, dtype=torch.float64, device="cuda")
    sp.u_bc = (capi.C.c_void_p * 3)(g.data_ptr(), None, None)
    with pytest.raises(capi.ChnsError):
        capi.chns_step(gm.handle, ds.c, capi.make_params(w.params.as_dict()), sp)
