"""CUDA-graph replay of the GMRES restart cycle (solve option use_graphs).

The captured cycle launches the same kernels with the same arguments in the same order as the
direct path, and every cycle-dependent scalar lives in device memory, so the solution and the
iteration record must be bit-identical with and without graphs; the solution must also meet the
same oracle bars as every other solve.  Several solves in one context reuse the capture (the key
matches) and a second mesh in the same context re-captures it (the key changes).
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


def solve_both(ctx, precision, orth):
    out = {}
    for g in (0, 1, 1):  # the second graph solve replays the cached capture
        x, info, st = ctx.solve(precision=precision, tol=1e-8, orth=orth, use_graphs=g)
        assert st == api.OK
        out.setdefault(g, []).append((x.cpu().numpy(), info))
    return out


@pytest.mark.parametrize("precision", [api.PREC_C128, api.PREC_MIXED])
@pytest.mark.parametrize("orth", [api.ORTH_CGS, api.ORTH_CGS2])
def test_graph_cycles_are_bit_identical(precision, orth):
    m = synth.cube_block_model(12)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    xr, _, st_r = ref.solve(tol=1e-8)
    assert st_r == oracle.OK
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        out = solve_both(ctx, precision, orth)
    x0, info0 = out[0][0]
    for xg, infog in out[1]:
        assert np.array_equal(xg, x0)
        for a, b in zip(infog, info0):
            assert a == b
    assert info0[0]["restarts"] >= 2  # several cycles replayed
    assert rel(x0[0], xr[0]) <= 1e-6


def test_graph_recaptured_for_a_new_mesh():
    with api.Context(0) as ctx:
        for n in (8, 10):
            m = synth.cube_block_model(n)
            ctx.mesh(m.mesh.nodes, m.mesh.tets)
            ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
            xg, ig, sg = ctx.solve(precision=api.PREC_MIXED, tol=1e-8, use_graphs=1)
            xd, idr, sd = ctx.solve(precision=api.PREC_MIXED, tol=1e-8, use_graphs=0)
            assert sg == sd == api.OK
            assert np.array_equal(xg.cpu().numpy(), xd.cpu().numpy())
            assert ig == idr


def test_graph_replay_with_sources_of_different_norms_and_a_second_tolerance():
    """The stop tolerance of a cycle (tol ||b||, and the inner tolerance of the mixed solver) is
    set by the cycle's initialisation, which runs outside the captured graph: sources whose
    right-hand sides differ in norm by 10^6 and a second solve at another tol, all replaying one
    capture, must give the direct launches' results bit for bit and each meet its own tol."""
    m = synth.cube_block_model(10)
    srcs = [synth.Dipole(1.0, 1.0, 1.0, 0, 1.0), synth.Dipole(60.0, -40.0, 1.0, 1, 1e-3),
            synth.Dipole(-30.0, 20.0, 1.0, 2, 1e3)]
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(srcs))
    xr, _, st_r = ref.solve(tol=1e-10)
    assert st_r == oracle.OK
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, srcs)
        for precision in (api.PREC_MIXED, api.PREC_C128):
            for tol in (1e-8, 1e-6, 1e-9):
                xg, ig, sg = ctx.solve(precision=precision, tol=tol, use_graphs=1, batch=1)
                xd, idr, sd = ctx.solve(precision=precision, tol=tol, use_graphs=0, batch=1)
                assert sg == sd == api.OK
                assert np.array_equal(xg.cpu().numpy(), xd.cpu().numpy())
                assert ig == idr
                for s in range(3):
                    assert ig[s]["true_rel_residual"] <= tol
                    assert rel(xg.cpu().numpy()[s], xr[s]) <= 1e3 * tol
