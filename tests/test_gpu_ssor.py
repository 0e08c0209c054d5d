"""Parity of the multicolour SSOR preconditioner and the SSOR-preconditioned SQMR solver with the
CPU oracles (oracle/ssor.py, oracle/sqmr.py).

* Colouring: integer work, bit-exact against the oracle's Jones-Plassmann colouring on the
  oracle's own pattern (n = 16 cube, n = 12 marine); at the 64^3 marine size, checked row by row
  against its defining property (each row's colour is the smallest one absent from its
  higher-priority neighbours, and no entry joins two rows of one colour).
* z = M^{-1} r: FP64, within 1e-12 (norm-relative) of the oracle's sweeps on the same colouring.
* Solves: FP64 true residual <= 1e-8 judged with the oracle's matrix, edge DOFs and receiver
  fields within 1e-6 of the oracle's 1e-8 solution, iteration counts close to the FP64 SSOR-SQMR
  oracle's.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.sqmr import sqmr
from oracle.ssor import SSOR, jp_colouring, priority_rank
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
}
_REF = {}


def reference(name):
    if name not in _REF:
        m = MODELS[name]()
        ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
        xr, _, st = ref.solve(tol=1e-8)
        assert st == oracle.OK
        rp, col, val, b = ref.system()
        n = len(rp) - 1
        A = sp.csr_matrix((val, col, rp), shape=(n, n))
        colour, rounds = jp_colouring(rp, col)
        _REF[name] = (m, ref, xr, A, b, colour, rounds)
    return _REF[name]


@pytest.mark.parametrize("name", list(MODELS))
def test_colouring_bit_exact(name):
    m, _, _, A, _, colour_ref, rounds_ref = reference(name)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        colour, nc, nr = ctx.colouring()
        colour = colour.cpu().numpy()
    assert np.array_equal(colour, colour_ref)
    assert nc == colour_ref.max() + 1 and nr == rounds_ref


def test_colouring_property_at_full_size():
    m = synth.marine_model(64, n_src=1)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        colour, nc, nr = ctx.colouring()
        colour = colour.cpu().numpy().astype(np.int64)
        rp, col, _, _, _ = ctx.system()
        rp, col = rp.cpu().numpy(), col.cpu().numpy().astype(np.int64)
    n = len(rp) - 1
    assert n == 1872064 and colour.min() == 0 and colour.max() == nc - 1 and nc <= 64
    rank = priority_rank(n)
    rows = np.repeat(np.arange(n), np.diff(rp))
    off = rows != col
    rows, cols = rows[off], col[off]
    assert not np.any(colour[rows] == colour[cols])
    hi = rank[cols] > rank[rows]
    used = np.zeros(n, dtype=np.uint64)
    np.bitwise_or.at(used, rows[hi], np.left_shift(np.uint64(1), colour[cols[hi]].astype(np.uint64)))
    mex = np.log2((~used & (used + np.uint64(1))).astype(np.float64)).astype(np.int64)
    assert np.array_equal(colour, mex)
    print("\nmarine 64^3: %d colours in %d rounds" % (nc, nr))


@pytest.mark.parametrize("omega", [1.0, 1.3])
@pytest.mark.parametrize("name", list(MODELS))
def test_ssor_apply_matches_oracle(name, omega):
    m, _, _, A, b, colour_ref, _ = reference(name)
    rng = np.random.default_rng(5)
    r = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    want = SSOR(A, colour_ref, omega).minv(r)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        z = ctx.ssor_apply(torch.as_tensor(r, device="cuda"), omega=omega).cpu().numpy()
    assert rel(z, want) <= 1e-12
    assert np.max(np.abs(z - want)) <= 1e-11 * np.max(np.abs(want))


def gpu_ssor(m, precision=api.PREC_C128, **opts):
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        x, info, st = ctx.solve(precision=precision, method=api.METHOD_SQMR, precond=api.PRECOND_SSOR, **opts)
        rcv, _ = ctx.receivers(m.receivers, x)
        return x.cpu().numpy(), info, st, rcv.cpu().numpy()


@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
@pytest.mark.parametrize("name", list(MODELS))
def test_ssor_sqmr_solution_and_receivers(name, precision):
    m, ref, xr, A, b, colour_ref, _ = reference(name)
    x, info, st, rcv = gpu_ssor(m, precision, tol=1e-8)
    assert st == api.OK
    P = SSOR(A, colour_ref, 1.0)
    for s in range(len(m.sources)):
        assert info[s]["status"] == api.OK and info[s]["true_rel_residual"] <= 1e-8
        res = np.linalg.norm(b[s] - ref.spmv(x[s])) / np.linalg.norm(b[s])
        assert res <= 1.0001e-8, res
        assert rel(x[s], xr[s]) <= 1e-6
        _, it_ref, rel_ref, _ = sqmr(A, b[s], tol=1e-8, precond=P)
        assert rel_ref <= 1e-8
        # the device stops on the quasi-residual tau and checks the true residual after; the
        # oracle checks the true residual at every step.  Complex64 inner solves restart from the
        # FP64 residual, which costs a few tens of iterations more.
        slack = 0.15 if precision == api.PREC_C128 else 0.5
        assert abs(info[s]["iters"] - it_ref) <= slack * it_ref + 10, (info[s]["iters"], it_ref)
    rr, _ = ref.receivers(xr, m.receivers)
    assert rel(rcv, rr) <= 1e-6
    print("\n%s %s: SSOR-SQMR iterations %s, inner solves %s" % (
        name, "c128" if precision == api.PREC_C128 else "mixed", [i["iters"] for i in info],
        [i["restarts"] for i in info]))


def test_ssor_omega_and_unsupported_options():
    m, ref, xr, _, b, _, _ = reference("cube_block_n16")
    x, info, st, _ = gpu_ssor(m, tol=1e-8, omega=1.4)
    assert st == api.OK and info[0]["true_rel_residual"] <= 1e-8 and rel(x[0], xr[0]) <= 1e-6
    m6 = synth.cube_block_model(6)
    with api.Context(0) as ctx:
        ctx.mesh(m6.mesh.nodes, m6.mesh.tets)
        ctx.assemble(m6.freq, m6.sigma, m6.sigma_p, m6.sources)
        for kw, code in ((dict(method=api.METHOD_COCG), api.ERR_UNSUPPORTED),
                         (dict(method=api.METHOD_GMRES), api.ERR_UNSUPPORTED),
                         (dict(method=api.METHOD_SQMR, omega=2.5), api.ERR_INVALID_ARG),
                         (dict(method=api.METHOD_SQMR, omega=-0.5), api.ERR_INVALID_ARG)):
            with pytest.raises(api.PetgemError) as e:
                ctx.solve(precond=api.PRECOND_SSOR, **kw)
            assert e.value.status == code


@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
def test_ssor_zero_rhs(precision):
    m = synth.cube_block_model(6)
    m.sigma = np.full_like(m.sigma, m.sigma_p)  # no anomaly: b = 0
    x, info, st, _ = gpu_ssor(m, precision)
    assert st == api.OK and info[0]["iters"] == 0 and not np.any(x)
