"""The phi integral through chns_phi_mass_noalloc, the entry point for callers that cannot
allocate while they run (code that must not call cudaMalloc, or applications whose memory is all
reserved up front by their own pool), on two calls in a row: it agrees with chns_phi_mass on the
same mesh and field, and with the oracle's FP64 integral 1^T M phi on an adaptive mesh with
hanging nodes. This file is collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs  # noqa: E402
from oracle import fem  # noqa: E402
from oracle.mesh import Mesh as OMesh  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import Mesh  # noqa: E402


def test_phi_mass_noalloc_matches_phi_mass_and_oracle():
    w = configs.rising_drop(3, 5, Cn=0.04)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    om = OMesh(w.anchors, w.levels, w.extent)
    assert mesh.n_hanging > 0
    el = fem.Elem(om)
    rng = np.random.default_rng(7)
    for call in range(2):
        phi_h = np.tanh(2.0 * rng.standard_normal(mesh.n_nodes))
        phi = torch.as_tensor(phi_h, device="cuda")
        ref = capi.chns_phi_mass(mesh.handle, phi)
        oracle = fem.phi_mass(el, phi_h)
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        capi.chns_phi_mass_noalloc(mesh.handle, phi, out)
        torch.cuda.synchronize()
        got = float(out.cpu()[0])
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (call, got, ref)
        assert abs(got - oracle) <= 1e-12 * max(1.0, abs(oracle)), (call, got, oracle)


def test_phi_mass_noalloc_inside_a_captured_graph():
    """After one call outside any capture, the call is recorded into a CUDA graph on a side
    stream; replaying the graph after phi was overwritten in place gives the oracle's integral of
    the new field each time."""
    w = configs.rising_drop(3, 5, Cn=0.04)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    el = fem.Elem(OMesh(w.anchors, w.levels, w.extent))
    rng = np.random.default_rng(11)
    phi = torch.as_tensor(np.tanh(rng.standard_normal(mesh.n_nodes)), device="cuda")
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    capi.chns_phi_mass_noalloc(mesh.handle, phi, out)  # the first call, outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        capi.chns_phi_mass_noalloc(mesh.handle, phi, out, stream=s)
    for rep in range(2):
        phi_h = np.tanh(2.0 * rng.standard_normal(mesh.n_nodes))
        phi.copy_(torch.as_tensor(phi_h, device="cuda"))
        out.fill_(np.nan)
        g.replay()
        torch.cuda.synchronize()
        got = float(out.cpu()[0])
        ref = fem.phi_mass(el, phi_h)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (rep, got, ref)
