"""The phi integral through chns_phi_mass_noalloc, the entry point for callers that cannot
allocate while they run (inside a stream capture, or under a fixed memory budget), agrees with
chns_phi_mass on the same mesh and field, on two calls in a row. This file is collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from chns_workloads import configs  # noqa: E402
from paper_2107_05123_gb300 import capi  # noqa: E402
from paper_2107_05123_gb300.session import Mesh  # noqa: E402


def test_phi_mass_noalloc_matches_phi_mass():
    w = configs.rising_drop(3, 5, Cn=0.04)
    mesh = Mesh(w.anchors, w.levels, w.extent)
    rng = np.random.default_rng(7)
    for call in range(2):
        phi = torch.as_tensor(np.tanh(2.0 * rng.standard_normal(mesh.n_nodes)), device="cuda")
        ref = capi.chns_phi_mass(mesh.handle, phi)
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        capi.chns_phi_mass_noalloc(mesh.handle, phi, out)
        torch.cuda.synchronize()
        got = float(out.cpu()[0])
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (call, got, ref)
