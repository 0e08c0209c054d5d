"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Bars: bit-exact for the integer work (edge numbering, signs, boundary, CSR pattern);
relative 1e-12 normwise per element for the FP64 element matrices and for the assembled
matrix and right-hand sides; relative L2 <= 1e-6 on edge DOFs and receiver fields after
solving to a relative residual of 1e-8.  Sizes span many thread blocks with ragged tails.
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


def relabelled(mesh, seed):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(mesh.n_nodes)
    nodes = np.empty_like(mesh.nodes)
    nodes[perm] = mesh.nodes
    return nodes, perm[mesh.tets].astype(np.int32)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def unpack21(K21):
    T = K21.shape[1]
    K = np.zeros((T, 6, 6))
    k = 0
    for i in range(6):
        for j in range(i, 6):
            K[:, i, j] = K21[k]
            K[:, j, i] = K21[k]
            k += 1
    return K


CASES = {
    "cube_n1": lambda: (synth.kuhn_mesh(1, (0, 0, 0), (1, 1, 1)), None),
    "cube_block_n16": lambda: (synth.cube_block_model(16).mesh, None),
    "relabelled_jitter_n7": lambda: (synth.kuhn_mesh(7, (0, 0, 0), (7, 5, 3), jitter=0.15, seed=11), 3),
    "bathymetry_n9": lambda: (synth.bathymetry_model(9, 2).mesh, 5),
}


@pytest.mark.parametrize("case", list(CASES))
def test_topology_bit_exact(case):
    mesh, seed = CASES[case]()
    nodes, tets = (mesh.nodes, mesh.tets) if seed is None else relabelled(mesh, seed)
    ref = oracle.System(nodes, tets, topology_only=True)
    e_r, te_r, sg_r, bd_r = ref.topology()
    with api.Context(0) as ctx:
        E = ctx.mesh(nodes, tets)
        e, te, sg, bd = (t.cpu().numpy() for t in ctx.topology())
    assert E == ref.n_edges
    assert np.array_equal(e, e_r)
    assert np.array_equal(te, te_r)
    assert np.array_equal(sg, sg_r)
    assert np.array_equal(bd, bd_r)


def model_case(name):
    if name == "cube_block_n16":
        return synth.cube_block_model(16)
    if name == "cube_block_n5":
        return synth.cube_block_model(5)
    if name == "cube_block_n24":
        return synth.cube_block_model(24)
    if name == "marine_n12":
        return synth.marine_model(12, n_src=3)
    if name == "bathymetry_n10":
        return synth.bathymetry_model(10, 4)
    raise KeyError(name)


_ORACLE = {}


def oracle_solution(name):
    """Oracle system and its 1e-8 solution for a named model, computed once per test session."""
    if name not in _ORACLE:
        m = model_case(name)
        ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
        xr, info_r, st_r = ref.solve(tol=1e-8)
        _ORACLE[name] = (m, ref, xr, st_r)
    return _ORACLE[name]


def gpu_forward(m, solve=True, **opts):
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        rp, col, val, b, dg = (t.cpu().numpy() for t in ctx.system())
        K21, M21, vol = (t.cpu().numpy() for t in ctx.elements())
        out = dict(rp=rp, col=col, val=val, b=b, diag=dg, K21=K21, M21=M21, vol=vol)
        if solve:
            x, info, st = ctx.solve(**opts)
            rcv, _ = ctx.receivers(m.receivers, x)
            out.update(x=x.cpu().numpy(), info=info, rcv=rcv.cpu().numpy())
    return out


@pytest.mark.parametrize("name", ["cube_block_n16", "marine_n12", "bathymetry_n10"])
def test_elements_and_system(name):
    m = model_case(name)
    src = synth.sources_array(m.sources)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, src)
    g = gpu_forward(m, solve=False)
    _, _, sg, _ = ref.topology()
    K = unpack21(g["K21"])
    M = unpack21(g["M21"])
    T = m.mesh.n_tets
    idx = np.arange(T) if T <= 30000 else np.random.default_rng(0).choice(T, 30000, replace=False)
    worst = 0.0
    for t in idx:
        Kr, Mr, vr = oracle.element(m.mesh.nodes[m.mesh.tets[t]], sg[t])
        worst = max(worst, np.abs(K[t] - Kr).max() / np.abs(Kr).max(), np.abs(M[t] - Mr).max() / np.abs(Mr).max(),
                    abs(g["vol"][t] - vr) / vr)
    assert worst <= 1e-12, worst
    rp, col, val, b = ref.system()
    assert np.array_equal(g["rp"], rp) and np.array_equal(g["col"], col)
    assert np.abs(g["val"] - val).max() <= 1e-12 * np.abs(val).max()
    for s in range(b.shape[0]):
        assert rel(g["b"][s], b[s]) <= 1e-12
    # Dirichlet rows are identity rows with zero right-hand side.
    _, _, _, bd = ref.topology()
    assert np.all(g["b"][:, bd == 1] == 0)


def test_assembly_is_deterministic():
    m = model_case("marine_n12")
    a = gpu_forward(m, solve=False)
    b = gpu_forward(m, solve=False)
    assert np.array_equal(a["val"], b["val"]) and np.array_equal(a["b"], b["b"])


def test_spmv_matches_oracle():
    m = model_case("cube_block_n16")
    src = synth.sources_array(m.sources)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, src)
    rng = np.random.default_rng(1)
    x = rng.normal(size=ref.n_edges) + 1j * rng.normal(size=ref.n_edges)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        xt = ctx.tensor(x)
        y = torch.empty_like(xt)
        api.petgem_spmv(ctx.h, xt, y)
        yg = y.cpu().numpy()
    assert rel(yg, ref.spmv(x)) <= 1e-14


@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
@pytest.mark.parametrize("name", ["cube_block_n16", "marine_n12", "cube_block_n24"])
def test_solve_and_receivers(name, precision):
    # cube_block_n24 has 102,024 edges: each persistent Gram-Schmidt block walks 3 (complex64) or
    # 6 (complex128) row tiles, so the double-buffered stages are reused.
    m, ref, xr, st_r = oracle_solution(name)
    assert st_r == oracle.OK
    g = gpu_forward(m, precision=precision, tol=1e-8)
    _, _, _, b = ref.system()
    for s in range(len(m.sources)):
        inf = g["info"][s]
        assert inf["status"] == api.OK and inf["true_rel_residual"] <= 1e-8
        # The oracle's own matrix and right-hand side judge the GPU solution.
        res = np.linalg.norm(b[s] - ref.spmv(g["x"][s])) / np.linalg.norm(b[s])
        assert res <= 1.0001e-8, res
        assert rel(g["x"][s], xr[s]) <= 1e-6
    rr, st = ref.receivers(xr, m.receivers)
    assert st == oracle.OK
    assert rel(g["rcv"], rr) <= 1e-6
    # Receivers alone, from the same DOFs: interpolation parity at FP64 level.
    rr_same, _ = ref.receivers(g["x"], m.receivers)
    assert rel(g["rcv"], rr_same) <= 1e-12


@pytest.mark.parametrize("orth", [api.ORTH_CGS2, api.ORTH_CGS_IFNEEDED])
@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
def test_orthogonalisation_variants(orth, precision):
    m, ref, xr, _ = oracle_solution("cube_block_n24")
    g = gpu_forward(m, precision=precision, tol=1e-8, orth=orth)
    _, _, _, b = ref.system()
    inf = g["info"][0]
    assert inf["status"] == api.OK and inf["true_rel_residual"] <= 1e-8
    assert np.linalg.norm(b[0] - ref.spmv(g["x"][0])) / np.linalg.norm(b[0]) <= 1.0001e-8
    assert rel(g["x"][0], xr[0]) <= 1e-6
    if orth == api.ORTH_CGS2:
        assert inf["reorth"] == inf["iters"]


def many_sources_model(n_src):
    m = synth.cube_block_model(8)
    rng = np.random.default_rng(n_src)
    m.sources = [synth.Dipole(float(x), float(y), float(z), int(a), 1.0)
                 for x, y, z, a in zip(rng.uniform(-300, 300, n_src), rng.uniform(-300, 300, n_src),
                                       rng.uniform(-100, 200, n_src), rng.integers(0, 3, n_src))]
    return m


@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
@pytest.mark.parametrize("n_src,batch", [(3, 0), (20, 0), (5, 2)])
def test_block_multi_source_solve(n_src, batch, precision):
    # All sources of one frequency iterate together (one SpMM per Arnoldi step); each source keeps
    # its own Krylov space and stopping test, so every source must match its own oracle solve.
    # 3 sources pad to a group of 4, 20 to 32, and batch=2 splits 5 sources into groups 2, 2, 1.
    m = model_case("marine_n12") if n_src == 3 else many_sources_model(n_src)
    src = synth.sources_array(m.sources)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, src)
    xr, info_r, st_r = ref.solve(tol=1e-8)
    assert st_r == oracle.OK
    _, _, _, b = ref.system()
    g = gpu_forward(m, precision=precision, tol=1e-8, batch=batch)
    for s in range(n_src):
        inf = g["info"][s]
        assert inf["status"] == api.OK and inf["true_rel_residual"] <= 1e-8, (s, inf)
        res = np.linalg.norm(b[s] - ref.spmv(g["x"][s])) / np.linalg.norm(b[s])
        assert res <= 1.0001e-8, (s, res)
        assert rel(g["x"][s], xr[s]) <= 1e-6
    rr, _ = ref.receivers(xr, m.receivers)
    assert rel(g["rcv"], rr) <= 1e-6


def test_precision_switch_in_one_context():
    # complex64 and complex128 Krylov vectors share one workspace with different layouts.
    m, ref, xr, _ = oracle_solution("cube_block_n24")
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        for prec in (api.PREC_C128, api.PREC_MIXED, api.PREC_C128, api.PREC_MIXED):
            x, info, st = ctx.solve(precision=prec)
            assert st == api.OK and info[0]["true_rel_residual"] <= 1e-8 and info[0]["reorth"] == 0
            assert rel(x.cpu().numpy()[0], xr[0]) <= 1e-6


def test_solve_tight_tolerance_agrees_closely():
    m = model_case("cube_block_n5")
    src = synth.sources_array(m.sources)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, src)
    xr, _, _ = ref.solve(tol=1e-13)
    g = gpu_forward(m, tol=1e-13)
    assert rel(g["x"][0], xr[0]) <= 1e-10


# ---------------------------------------------------------------- edge cases
def test_no_anomaly_gives_zero_field():
    m = synth.cube_block_model(4)
    sigma = np.full(m.mesh.n_tets, m.sigma_p)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, sigma, m.sigma_p, m.sources)
        x, info, st = ctx.solve()
        assert st == api.OK and info[0]["iters"] == 0
        assert torch.count_nonzero(x).item() == 0


def test_single_cube_has_one_unknown():
    mesh = synth.kuhn_mesh(1, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))
    src = [synth.Dipole(0.3, -0.2, 0.1, 2, 1.0)]
    sigma = np.full(6, 0.5)
    ref = oracle.System(mesh.nodes, mesh.tets, sigma, 1.0, 2.0, synth.sources_array(src))
    xr, _, _ = ref.solve(tol=1e-12)
    with api.Context(0) as ctx:
        assert ctx.mesh(mesh.nodes, mesh.tets) == 19
        ctx.assemble(2.0, sigma, 1.0, src)
        x, info, st = ctx.solve(tol=1e-12)
        xg = x.cpu().numpy()
    assert rel(xg, xr) <= 1e-10
    assert np.count_nonzero(xg) == 1


def test_bad_meshes_are_rejected():
    mesh = synth.kuhn_mesh(2, (0, 0, 0), (1, 1, 1))
    with api.Context(0) as ctx:
        bad = mesh.tets.copy()
        bad[3, 2] = mesh.n_nodes + 5
        with pytest.raises(api.PetgemError) as e:
            ctx.mesh(mesh.nodes, bad)
        assert e.value.status == api.ERR_BAD_MESH
        rep = mesh.tets.copy()
        rep[0, 1] = rep[0, 0]
        with pytest.raises(api.PetgemError) as e:
            ctx.mesh(mesh.nodes, rep)
        assert e.value.status == api.ERR_BAD_MESH
        # The context stays usable after a rejected mesh.
        assert ctx.mesh(mesh.nodes, mesh.tets) == synth.kuhn_counts(2)["edges"]
        flat = mesh.nodes.copy()
        flat[:, 2] = 0.0                       # every tet collapses to zero volume
        ctx.mesh(flat, mesh.tets)
        with pytest.raises(api.PetgemError) as e:
            ctx.assemble(1.0, np.ones(mesh.n_tets), 1.0, [synth.Dipole(5, 5, 5)])
        assert e.value.status == api.ERR_DEGENERATE_TET


def test_receiver_outside_and_iteration_cap():
    m = synth.cube_block_model(4)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        x, info, st = ctx.solve(max_iters=3, allow_not_converged=True)
        assert st == api.ERR_NOT_CONVERGED
        assert info[0]["iters"] == 3 and info[0]["true_rel_residual"] > 1e-8
        rx = np.array([[0.0, 0.0, -100.0], [5000.0, 0.0, 0.0]])
        out, st = ctx.receivers(rx, x, allow_outside=True)
        assert st == api.ERR_RECEIVER_OUTSIDE
        o = out.cpu().numpy()
        assert np.isfinite(o[0, 0]).all() and np.isnan(o[0, 1]).all()
