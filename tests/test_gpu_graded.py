"""The solver path on a frequency-adapted graded mesh (Section 5.3's spacing rules on a Kuhn
grid: spacings from ~25 m near the source to a few hundred metres in the boundary layers, with
conforming material interfaces) against the CPU oracle: FP64 true residual <= 1e-8 (also under the
oracle's matrix), edge DOFs and receiver fields within 1e-6 of the oracle's solution."""
import numpy as np
import pytest

import oracle
from paper_1808_00186_gb300 import api, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_00186_gb300 import build
    build.build()
    oracle.build()
    api.load()
    torch.cuda.set_device(0)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.fixture(scope="module")
def graded():
    m = synth.graded_marine_model(8.0, L_s=400.0, r_xy=1.5, r_z=1.0, r_b=0.5)
    m.receivers = np.stack([np.linspace(-300.0, 300.0, 21), np.zeros(21), np.zeros(21)], axis=1)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    xr, _, st = ref.solve(tol=1e-8)
    assert st == oracle.OK
    return m, ref, xr


@pytest.mark.parametrize("method", [api.METHOD_GMRES, api.METHOD_COCG])
def test_graded_mesh_parity(graded, method):
    m, ref, xr = graded
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        x, info, st = ctx.solve(precision=api.PREC_MIXED, tol=1e-8, method=method)
        assert st == api.OK and info[0]["true_rel_residual"] <= 1e-8
        rcv, _ = ctx.receivers(m.receivers, x)
    x = x.cpu().numpy()
    _, _, _, b = ref.system()
    assert np.linalg.norm(b[0] - ref.spmv(x[0])) / np.linalg.norm(b[0]) <= 1.0001e-8
    assert rel(x[0], xr[0]) <= 1e-6
    rr, _ = ref.receivers(xr, m.receivers)
    assert rel(rcv.cpu().numpy(), rr) <= 1e-6
    print("\ngraded %s: %d edges, %d iterations" % ("GMRES" if method == api.METHOD_GMRES else "COCG",
                                                   x.shape[1], info[0]["iters"]))
