"""GPU parity of the full time step (chns_step) against the oracle's two-block step, and the
invariants the paper states for it (mass conservation, Prop. mass_conservation)."""
import numpy as np
import pytest

from gpu_common import relerr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs  # noqa: E402
from oracle import fem, step  # noqa: E402
from oracle.mesh import Mesh as OMesh  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import DeviceState, Mesh, default_step_params  # noqa: E402


def _run(w, nsteps, rtol=1e-12, inner=capi.FP64, newton_rtol=1e-13):
    om = OMesh(w.anchors, w.levels, w.extent)
    gm = Mesh(w.anchors, w.levels, w.extent)
    f = w.init(om.node_xyz)
    st = step.State(phi=f["phi"], mu=f["mu"], u=f["u"], u_old=f["u"], p=f["p"])
    ds = DeviceState(dict(phi=f["phi"], mu=f["mu"], u=f["u"], p=f["p"]))
    prm = w.params.as_dict()
    sp = default_step_params(rtol=rtol, inner=inner, newton_rtol=newton_rtol)
    stats = []
    for _ in range(nsteps):
        st = step.chns_step(om, prm, st, newton_rtol=newton_rtol)
        stats.append(capi.chns_step(gm.handle, ds.c, capi.make_params(prm), sp))
    return om, gm, st, ds.host(), stats


@pytest.mark.parametrize("level", [3, 4])
def test_step_smooth_uniform_matches_oracle(level):
    w = configs.smooth_uniform(level, seed=0)
    om, gm, ref, got, stats = _run(w, 1)
    assert relerr(got["phi"], ref.phi) < 1e-8
    assert relerr(got["mu"], ref.mu) < 1e-8
    assert relerr(got["u"], ref.u) < 1e-8
    assert relerr(got["u_old"], ref.u_old) == 0.0
    assert relerr(got["p"] - got["p"].mean(), ref.p - ref.p.mean()) < 1e-8
    s = stats[0]
    assert abs(s.phi_mass_after - s.phi_mass_before) < 1e-11
    # inexact Newton (first linear solve to 1e-3) needs one more step than the oracle's exact one
    assert all(s.newton_its[i] <= 4 for i in range(2))


def test_step_adaptive_drop_matches_oracle():
    w = configs.rising_drop(3, 5, Cn=0.04)
    om, gm, ref, got, stats = _run(w, 2)
    assert om.n_hanging > 0
    for k in ("phi", "mu", "u"):
        assert relerr(got[k], getattr(ref, k)) < 1e-8, k
    assert relerr(got["p"] - got["p"].mean(), ref.p - ref.p.mean()) < 1e-8
    for s in stats:
        assert abs(s.phi_mass_after - s.phi_mass_before) < 1e-11


def test_step_mixed_precision_error_per_field():
    """FP32 inner solves with FP64 refinement to 1e-10: the step stays within 1e-6 of the oracle
    per field (the solves' residual tolerance times the conditioning of each sub-problem)."""
    w = configs.rising_drop(3, 5, Cn=0.04)
    om, gm, ref, got, stats = _run(w, 1, rtol=1e-10, inner=capi.FP32, newton_rtol=1e-10)
    for k in ("phi", "mu", "u"):
        assert relerr(got[k], getattr(ref, k)) < 1e-6, k
    assert relerr(got["p"] - got["p"].mean(), ref.p - ref.p.mean()) < 1e-6
