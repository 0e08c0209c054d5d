"""Parity at the workloads' full sizes (the oracle cannot solve these in test time, but it builds
their topology and system in seconds).

* marine 64^3 (1.57 M tets, 1.87 M edges), the bench's workload in the bench's launch
  configuration: one source, mixed-precision GMRES(50), SELL-32 products, CUDA-graph cycles.
* bathymetry 96^3 (5.31 M tets, 6.28 M edges), the largest case, two of its sources, mixed COCG.

Checks, against the FP64 oracle run on the same inputs:
* topology and CSR pattern bit-exact, whole arrays;
* matrix within 1e-12 of its largest entry, right-hand sides within 1e-12 (relative L2),
  Dirichlet rows with zero right-hand side, element matrices on 20,000 sampled tets within 1e-12;
* the solution judged by the oracle's matrix and right-hand side: ||b_o - A_o x|| is at most the
  device's own 1e-8 ||b|| plus the exact effect of the (1e-12-level) difference between the two
  systems, ||b_o - b|| + ||(A_o - A) x||;
* the receivers kernel on seeded edge DOFs within 1e-12 of the oracle's interpolation of them.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


def host_memory_gb():
    try:
        with open("/proc/meminfo") as f:
            return next(int(l.split()[1]) for l in f if l.startswith("MemAvailable:")) / 2 ** 20
    except (OSError, StopIteration):
        return 0.0


def unpack21(K21):
    K = np.zeros((K21.shape[1], 6, 6))
    k = 0
    for i in range(6):
        for j in range(i, 6):
            K[:, i, j] = K21[k]
            K[:, j, i] = K21[k]
            k += 1
    return K


def gpu_run(m, n_sample, **solve_opts):
    """Topology, system, sampled element matrices, solution and receivers from the device."""
    T = m.mesh.n_tets
    idx = np.sort(np.random.default_rng(0).choice(T, min(T, n_sample), replace=False))
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        g = dict(zip(("edges", "tet_edges", "signs", "boundary"), (t.cpu().numpy() for t in ctx.topology())))
        g.update(zip(("rp", "col", "val", "b", "diag"), (t.cpu().numpy() for t in ctx.system())))
        K21, M21, vol = ctx.elements()
        it = torch.as_tensor(idx, device=K21.device)
        g.update(idx=idx, K=unpack21(K21[:, it].cpu().numpy()), M=unpack21(M21[:, it].cpu().numpy()),
                 vol=vol[it].cpu().numpy())
        del K21, M21, vol
        x, info, st = ctx.solve(**solve_opts)
        g.update(x=x.cpu().numpy(), info=info, status=st)
        # the receivers kernel on seeded edge DOFs (not the solver's), so that the oracle's expected
        # fields depend on the inputs alone
        rng = np.random.default_rng(7)
        xs = rng.normal(size=g["x"].shape) + 1j * rng.normal(size=g["x"].shape)
        rcv, _ = ctx.receivers(m.receivers, torch.as_tensor(xs, device=x.device))
        g.update(x_syn=xs, rcv_syn=rcv.cpu().numpy())
    return g


def check_against_oracle(m, g):
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    e, te, sg, bd = ref.topology()
    assert np.array_equal(g["edges"], e) and np.array_equal(g["tet_edges"], te)
    assert np.array_equal(g["signs"], sg) and np.array_equal(g["boundary"], bd)
    worst = 0.0
    for k, t in enumerate(g["idx"]):
        Kr, Mr, vr = oracle.element(m.mesh.nodes[m.mesh.tets[t]], sg[t])
        worst = max(worst, np.abs(g["K"][k] - Kr).max() / np.abs(Kr).max(),
                    np.abs(g["M"][k] - Mr).max() / np.abs(Mr).max(), abs(g["vol"][k] - vr) / vr)
    assert worst <= 1e-12, worst
    rp, col, val, b = ref.system()
    assert np.array_equal(g["rp"], rp) and np.array_equal(g["col"], col)
    assert np.abs(g["val"] - val).max() <= 1e-12 * np.abs(val).max()
    n = len(rp) - 1
    dA = sp.csr_matrix((val - g["val"], col, rp), shape=(n, n))
    for s in range(b.shape[0]):
        bn = np.linalg.norm(b[s])
        db = np.linalg.norm(b[s] - g["b"][s])
        assert db <= 1e-12 * bn
        assert np.all(g["b"][s][bd == 1] == 0)
        inf = g["info"][s]
        assert inf["status"] == api.OK and inf["true_rel_residual"] <= 1e-8, inf
        x = g["x"][s]
        res = np.linalg.norm(b[s] - ref.spmv(x))
        bound = 1e-8 * np.linalg.norm(g["b"][s]) + db + np.linalg.norm(dA @ x) + 1e-14 * bn
        assert res <= bound, (res / bn, bound / bn)
    rr, st = ref.receivers(g["x_syn"], m.receivers)
    assert st == oracle.OK
    assert np.linalg.norm(np.ravel(g["rcv_syn"] - rr)) <= 1e-12 * np.linalg.norm(np.ravel(rr))
    return [i["iters"] for i in g["info"]]


def test_marine_n64_bench_configuration():
    if host_memory_gb() < 24:
        pytest.skip("needs ~8 GB of host memory for the oracle and the copies")
    m = synth.marine_model(64, n_src=1)
    g = gpu_run(m, 20000, precision=api.PREC_MIXED, tol=1e-8, use_graphs=1)
    assert g["status"] == api.OK and len(g["edges"]) == 1872064
    iters = check_against_oracle(m, g)
    print("\nmarine 64^3, mixed GMRES(50) with graphs: %s iterations" % iters)


def test_bathymetry_n96_two_sources():
    if host_memory_gb() < 48:
        pytest.skip("needs ~16 GB of host memory for the oracle and the copies")
    m = synth.bathymetry_model(96, 2)
    g = gpu_run(m, 20000, precision=api.PREC_MIXED, method=api.METHOD_COCG, tol=1e-8, batch=1, max_iters=60000)
    assert g["status"] == api.OK and len(g["edges"]) == 6276384
    iters = check_against_oracle(m, g)
    print("\nbathymetry 96^3, mixed COCG: %s iterations" % iters)
