"""Parity of the SQMR solver (petgem_solve with method SQMR) with the CPU oracles.

Bars as for GMRES and COCG: the FP64 true residual <= 1e-8, judged again with the oracle's own
matrix; relative L2 <= 1e-6 on edge DOFs against the oracle's 1e-8 solution and on receiver
fields.  The FP64 variant also follows the FP64 SQMR oracle (oracle/sqmr.py, Jacobi split
symmetrically) in its number of iterations.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.sqmr import sqmr
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


MODELS = {
    "cube_block_n16": lambda: synth.cube_block_model(16),
    "marine_n12_3src": lambda: synth.marine_model(12, n_src=3),
    "cube_block_n24": lambda: synth.cube_block_model(24),
}
_REF = {}


def reference(name):
    if name not in _REF:
        m = MODELS[name]()
        ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
        xr, _, st = ref.solve(tol=1e-8)
        assert st == oracle.OK
        _REF[name] = (m, ref, xr)
    return _REF[name]


def gpu_sqmr(m, precision, **opts):
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        x, info, st = ctx.solve(precision=precision, method=api.METHOD_SQMR, **opts)
        rcv, _ = ctx.receivers(m.receivers, x)
        return x.cpu().numpy(), info, st, rcv.cpu().numpy()


@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
@pytest.mark.parametrize("name", list(MODELS))
def test_sqmr_solution_and_receivers(name, precision):
    m, ref, xr = reference(name)
    x, info, st, rcv = gpu_sqmr(m, precision, tol=1e-8, batch=0)  # batch is ignored: one by one
    assert st == api.OK
    _, _, _, b = ref.system()
    for s in range(len(m.sources)):
        assert info[s]["status"] == api.OK and info[s]["true_rel_residual"] <= 1e-8
        res = np.linalg.norm(b[s] - ref.spmv(x[s])) / np.linalg.norm(b[s])
        assert res <= 1.0001e-8, res
        assert rel(x[s], xr[s]) <= 1e-6
        assert info[s]["iters"] <= 4 * len(b[s]) ** (1.0 / 3.0) * 20
    rr, _ = ref.receivers(xr, m.receivers)
    assert rel(rcv, rr) <= 1e-6
    print("\n%s %s: SQMR iterations %s, inner solves %s" % (name, "c128" if precision == api.PREC_C128 else "mixed",
                                                          [i["iters"] for i in info], [i["restarts"] for i in info]))


def test_sqmr_fp64_iterations_follow_the_oracle():
    m, ref, _ = reference("cube_block_n16")
    rp, col, val, b = ref.system()
    n = len(rp) - 1
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    _, it_ref, rel_ref, _ = sqmr(A, b[0], tol=1e-8)
    assert rel_ref <= 1e-8
    _, info, st, _ = gpu_sqmr(m, api.PREC_C128, tol=1e-8)
    assert st == api.OK
    it = info[0]["iters"]
    # the device stops an inner solve on the quasi-residual tau (an estimate within sqrt(n + 1) of
    # the smoothed residual) and checks the true residual after; the oracle checks it every step
    assert abs(it - it_ref) <= 0.15 * it_ref + 10, (it, it_ref)


def test_sqmr_zero_rhs_and_unsupported_options():
    m = synth.cube_block_model(6)
    m.sigma = np.full_like(m.sigma, m.sigma_p)  # no anomaly: b = 0
    x, info, st, _ = gpu_sqmr(m, api.PREC_MIXED)
    assert st == api.OK and info[0]["iters"] == 0 and not np.any(x)
    m = synth.cube_block_model(6)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        with pytest.raises(api.PetgemError) as e:
            ctx.solve(method=api.METHOD_SQMR, precond=api.PRECOND_LEARNED)
        assert e.value.status == api.ERR_UNSUPPORTED
