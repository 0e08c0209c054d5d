"""The SELL-32 layout on a mesh whose node numbering is not a lattice's: the same cube model with
its node ids shuffled, so that the differences hi - lo of the edges take many values and the
layout keeps the original row order (no grouping by edge kind).  GMRES and COCG must still meet the
oracle bars on it (1e-8 residual, 1e-6 DOFs and receivers), and the lattice-numbered and shuffled
meshes must give the same solution (the same edges, renumbered)."""
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


@pytest.mark.parametrize("method", [api.METHOD_GMRES, api.METHOD_COCG])
def test_shuffled_node_numbering(method):
    m = synth.cube_block_model(12)
    rng = np.random.default_rng(11)
    new_id = rng.permutation(m.mesh.n_nodes)          # old node i becomes new_id[i]
    nodes = np.empty_like(m.mesh.nodes)
    nodes[new_id] = m.mesh.nodes
    tets = new_id[m.mesh.tets].astype(np.int32)
    ref = oracle.System(nodes, tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    xr, _, st = ref.solve(tol=1e-8)
    assert st == oracle.OK
    with api.Context(0) as ctx:
        ctx.mesh(nodes, tets)
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
    # the receiver fields do not depend on the numbering: same as the lattice-numbered mesh
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        x2, _, st2 = ctx.solve(precision=api.PREC_MIXED, tol=1e-8, method=method)
        rcv2, _ = ctx.receivers(m.receivers, x2)
    assert st2 == api.OK
    assert rel(rcv.cpu().numpy(), rcv2.cpu().numpy()) <= 1e-6
