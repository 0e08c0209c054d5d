"""Frequency reuse (petgem_assemble_frequency): A(w) = K + i w mu0 M_sigma from the real matrices
the first assembly keeps (eq. 9 is linear in w).

petgem_assemble forms A the same way, so a system re-assembled for a new frequency must be
bit-identical to a fresh assembly at that frequency; it must also match the oracle's system at
that frequency (normwise 1e-12, the element-matrix bar) and solve to the oracle's solution.
"""
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


def system_np(ctx):
    return [t.cpu().numpy() for t in ctx.system()]


@pytest.mark.parametrize("freqs", [(1.0, 0.25, 3.0), (2.0, 7.5)])
def test_frequency_reuse_equals_fresh_assembly_and_oracle(freqs):
    m = synth.marine_model(10, n_src=3)
    srcs2 = m.sources[:2]
    with api.Context(0) as a, api.Context(0) as f:
        a.mesh(m.mesh.nodes, m.mesh.tets)
        f.mesh(m.mesh.nodes, m.mesh.tets)
        a.assemble(freqs[0], m.sigma, m.sigma_p, m.sources)
        for k, fr in enumerate(freqs[1:]):
            src = srcs2 if k % 2 == 0 else m.sources
            a.assemble_frequency(fr, src)
            f.assemble(fr, m.sigma, m.sigma_p, src)
            sa, sf = system_np(a), system_np(f)
            for x, y in zip(sa, sf):  # row_ptr, col, val, b, diag
                assert np.array_equal(x, y)
            ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, fr, synth.sources_array(src))
            rp, col, val, b = ref.system()
            assert np.array_equal(sa[0], rp) and np.array_equal(sa[1], col)
            assert rel(sa[2], val) <= 1e-12
            assert rel(sa[3], b) <= 1e-12
            x, info, st = a.solve(precision=api.PREC_MIXED, tol=1e-8)
            assert st == api.OK
            xr, _, st_r = ref.solve(tol=1e-8)
            assert st_r == oracle.OK
            assert rel(x.cpu().numpy(), xr) <= 1e-6


def test_frequency_reuse_errors():
    m = synth.cube_block_model(4)
    with api.Context(0) as c:
        c.mesh(m.mesh.nodes, m.mesh.tets)
        with pytest.raises(api.PetgemError) as e:
            c.assemble_frequency(1.0, m.sources)
        assert e.value.status == api.ERR_INVALID_ARG
        c.assemble(2.0, m.sigma, m.sigma_p, m.sources)
        for fr, src in ((0.0, m.sources), (-1.0, m.sources), (1.0, [])):
            with pytest.raises(api.PetgemError) as e:
                c.assemble_frequency(fr, src)
            assert e.value.status == api.ERR_INVALID_ARG
