"""Batch of meshes (petgem_solve_batch): the systems of several contexts, of different sizes and
with one or more sources each, solved together by COCG in one persistent launch per refinement
round.

Each system must meet the bars of a single solve against its own oracle: FP64 true residual
<= 1e-8 (judged again with the oracle's matrix), edge DOFs and receiver fields within 1e-6 of the
oracle's solution.  With the lane count fixed the batch is deterministic, so the graph-replayed
refinement rounds must give bit-identical results to direct launches.
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


MODELS = [lambda: synth.cube_block_model(8), lambda: synth.marine_model(12, n_src=2), lambda: synth.cube_block_model(16)]
_REF = {}


def reference(i):
    if i not in _REF:
        m = MODELS[i]()
        ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
        xr, _, st = ref.solve(tol=1e-8)
        assert st == oracle.OK
        _REF[i] = (m, ref, xr)
    return _REF[i]


def contexts(models):
    out = []
    for m in models:
        c = api.Context(0)
        c.mesh(m.mesh.nodes, m.mesh.tets)
        c.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        out.append(c)
    return out


def check_against_oracle(m, ref, xr, x, info, ctx):
    _, _, _, b = ref.system()
    for s in range(len(m.sources)):
        assert info[s]["status"] == api.OK and info[s]["true_rel_residual"] <= 1e-8, info[s]
        res = np.linalg.norm(b[s] - ref.spmv(x[s])) / np.linalg.norm(b[s])
        assert res <= 1.0001e-8, res
        assert rel(x[s], xr[s]) <= 1e-6
    rcv, _ = ctx.receivers(m.receivers, torch.as_tensor(x, device="cuda:0"))
    rr, _ = ref.receivers(xr, m.receivers)
    assert rel(rcv.cpu().numpy(), rr) <= 1e-6


@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
def test_batch_matches_oracle(precision):
    refs = [reference(i) for i in range(len(MODELS))]
    ctxs = contexts([r[0] for r in refs])
    try:
        xs, info, st = api.solve_batch(ctxs, precision=precision, tol=1e-8, use_graphs=1)
        assert st == api.OK
        k = 0
        for (m, ref, xr), c, x in zip(refs, ctxs, xs):
            ns = len(m.sources)
            check_against_oracle(m, ref, xr, x.cpu().numpy(), info[k:k + ns], c)
            k += ns
        assert k == len(info) == 4
        assert all(i["spmv_lanes"] in (1, 2, 4, 8) for i in info)  # the autotuner's pick
        print("\nbatch %s: iterations %s, inner solves %s, lanes %d" % (
            "c128" if precision == api.PREC_C128 else "mixed", [i["iters"] for i in info],
            [i["restarts"] for i in info], info[0]["spmv_lanes"]))
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_batch_graph_replay_is_bit_identical(lanes):
    refs = [reference(i) for i in (0, 1)]
    ctxs = contexts([r[0] for r in refs])
    try:
        out = []
        for g in (0, 1):
            xs, info, st = api.solve_batch(ctxs, precision=api.PREC_MIXED, tol=1e-8, use_graphs=g, spmv_lanes=lanes)
            assert st == api.OK
            out.append(([x.cpu().numpy() for x in xs], info))
        for a, b in zip(out[0][0], out[1][0]):
            assert np.array_equal(a, b)
        assert out[0][1] == out[1][1]
        assert all(i["spmv_lanes"] == lanes for i in out[0][1])
        k = 0
        for (m, ref, xr), c, x in zip(refs, ctxs, out[0][0]):
            ns = len(m.sources)
            check_against_oracle(m, ref, xr, x, out[0][1][k:k + ns], c)
            k += ns
    finally:
        for c in ctxs:
            c.close()


def test_batch_of_one_follows_the_single_solver():
    m, ref, xr = reference(2)
    (c,) = contexts([m])
    try:
        xs, info, st = api.solve_batch([c], precision=api.PREC_MIXED, tol=1e-8, spmv_lanes=4)
        x1, info1, st1 = c.solve(precision=api.PREC_MIXED, tol=1e-8, method=api.METHOD_COCG)
        assert st == st1 == api.OK
        # same iteration, same lanes; the block partition differs, so sums round differently
        assert abs(info[0]["iters"] - info1[0]["iters"]) <= 0.1 * info1[0]["iters"] + 10
        assert rel(xs[0].cpu().numpy(), x1.cpu().numpy()) <= 1e-6
    finally:
        c.close()


def test_batch_zero_rhs_and_errors():
    mz = synth.cube_block_model(6)
    mz.sigma = np.full_like(mz.sigma, mz.sigma_p)  # no anomaly: b = 0
    m, ref, xr = reference(0)
    ctxs = contexts([mz, m])
    try:
        xs, info, st = api.solve_batch(ctxs, precision=api.PREC_MIXED, tol=1e-8)
        assert st == api.OK
        assert info[0]["iters"] == 0 and not np.any(xs[0].cpu().numpy())
        check_against_oracle(m, ref, xr, xs[1].cpu().numpy(), info[1:], ctxs[1])
        for bad, code in ((dict(method=api.METHOD_GMRES), api.ERR_UNSUPPORTED), (dict(spmv_lanes=3), api.ERR_UNSUPPORTED),
                          (dict(precond=api.PRECOND_LEARNED), api.ERR_UNSUPPORTED), (dict(tol=0.0), api.ERR_INVALID_ARG)):
            with pytest.raises(api.PetgemError) as e:
                api.solve_batch(ctxs, **bad)
            assert e.value.status == code, bad
        with pytest.raises(api.PetgemError) as e:
            api.solve_batch([ctxs[1], ctxs[1]])
        assert e.value.status == api.ERR_INVALID_ARG
        fresh = api.Context(0)
        try:
            fresh.n_src, fresh.n_edges, fresh.nodes = 1, 1, ctxs[0].nodes
            with pytest.raises(api.PetgemError) as e:
                api.solve_batch([ctxs[1], fresh])
            assert e.value.status == api.ERR_INVALID_ARG
        finally:
            fresh.close()
        assert api.petgem_solve_batch([], [], [])[0] == api.OK
    finally:
        for c in ctxs:
            c.close()
