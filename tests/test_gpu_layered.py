"""Layered-Earth primary field kernel (petgem_primary_layered) against the FP64 oracle
(oracle/layered.py), through the C ABI.

Both sides evaluate the same Hankel integrals with the same quadrature nodes, but solve each
wavenumber's TE/TM problem differently (the oracle a linear system over the layers, the kernel an
admittance recursion) and take Bessel functions from different libraries; the bar is relative
1e-10 per point (normwise over the three components).  Models: the canonical marine model of
Section 5.1 (seawater, sediment, 100 m resistor, sediment) with an x-dipole 50 m above the
seafloor, and a three-layer model with a y-dipole inside the middle layer.  Points in every layer,
on interfaces (seafloor receivers), within metres of an interface and right above the source.
"""
import numpy as np
import pytest

import oracle
from oracle import layered as LY
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


def points(z_if, rng, n=14):
    p = [[0.0, 0.0, 80.0], [500.0, 0.0, 0.0], [-2000.0, 300.0, 0.0], [1200.0, -400.0, z_if[-1] + 2.0],
         [800.0, 800.0, z_if[-1] - 2.0], [3500.0, 100.0, -300.0]]
    for _ in range(n - len(p)):
        p.append([rng.uniform(-3000, 3000), rng.uniform(-1500, 1500), rng.uniform(z_if[-1] - 600, 400)])
    return np.array(p)


@pytest.mark.parametrize("case", ["canonical_x", "three_layer_y"])
def test_layered_primary_field_matches_oracle(case):
    rng = np.random.default_rng(7)
    if case == "canonical_x":
        z_if, sig, src, f = [0.0, -1000.0, -1100.0], [3.3, 1.0, 0.01, 1.0], synth.Dipole(10.0, -5.0, 50.0, 0, 1.0), 1.0
    else:
        z_if, sig, src, f = [200.0, -400.0], [3.3, 0.8, 0.1], synth.Dipole(-30.0, 40.0, -150.0, 1, 2.5), 0.5
    pts = points(z_if, rng)
    ref = LY.primary_field(pts, (src.x, src.y, src.z, src.axis, src.moment), np.array(z_if), np.array(sig), f)
    p_t = torch.as_tensor(pts, device="cuda")
    out = torch.empty((len(pts), 3), dtype=torch.complex128, device="cuda")
    api.petgem_primary_layered(torch.cuda.current_stream().cuda_stream, z_if, sig, f, src, p_t, out)
    got = out.cpu().numpy()
    for i in range(len(pts)):
        err = np.linalg.norm(got[i] - ref[i]) / np.linalg.norm(ref[i])
        assert err <= 1e-10, (i, pts[i], got[i], ref[i], err)


def test_one_layer_is_appendix_a_and_empty_call():
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(-900, 900, 9), rng.uniform(-900, 900, 9), rng.uniform(-900, 900, 9)], 1)
    src = synth.Dipole(1.0, 1.0, 1.0, 0, 1.0)
    out = torch.empty((9, 3), dtype=torch.complex128, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    api.petgem_primary_layered(s, [], [1.3], 2.0, src, torch.as_tensor(pts, device="cuda"), out)
    ref = oracle.primary_field(pts, (1.0, 1.0, 1.0, 0, 1.0), 1.3, 2.0)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    api.petgem_primary_layered(s, [0.0], [3.3, 1.0], 1.0, src, None, None)  # no points: nothing launched


def layered_case():
    """Three-layer background (seawater 3.3 S/m above z = 0, sediment 1 S/m to -1000 m, 0.5 S/m
    below) with a 0.02 S/m block one cell thick in the sediment; interfaces on node planes; an x-
    and a y-dipole 60 m above the seafloor, 1 Hz."""
    mesh = synth.kuhn_mesh(8, (-2000.0, -2000.0, -1500.0), (2000.0, 2000.0, 500.0))
    z_if, sig_l = [0.0, -1000.0], [3.3, 1.0, 0.5]
    cen = mesh.centroids()
    sigma = np.where(cen[:, 2] > 0.0, 3.3, np.where(cen[:, 2] > -1000.0, 1.0, 0.5))
    block = (np.abs(cen[:, 0]) < 500.0) & (np.abs(cen[:, 1]) < 500.0) & (cen[:, 2] > -750.0) & (cen[:, 2] < -500.0)
    sigma[block] = 0.02
    srcs = [synth.Dipole(0.0, 0.0, 60.0, 0, 1.0), synth.Dipole(200.0, 100.0, 60.0, 1, 1.0)]
    rx = np.stack([np.linspace(-1500, 1500, 13), np.zeros(13), np.zeros(13)], 1)
    return mesh, sigma, z_if, sig_l, srcs, rx, 1.0


def test_layered_assembly_solve_and_receivers_match_oracle():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    mesh, sigma, z_if, sig_l, srcs, rx, f = layered_case()
    s5 = [(d.x, d.y, d.z, d.axis, d.moment) for d in srcs]
    ref = oracle.System(mesh.nodes, mesh.tets, sigma, 1.0, f, np.array(s5))
    edges, te, sg, bd = ref.topology()
    rp, col, val, _ = ref.system()
    b_ref = LY.rhs(mesh.nodes, mesh.tets, sigma, z_if, sig_l, f, s5, te, sg, bd, ref.n_edges)
    A = sp.csr_matrix((val, col, rp), shape=(ref.n_edges, ref.n_edges)).tocsc()
    x_ref = np.stack([spl.spsolve(A, b_ref[i]) for i in range(len(srcs))])
    with api.Context(0) as ctx:
        ctx.mesh(mesh.nodes, mesh.tets)
        ctx.assemble_layered(f, sigma, z_if, sig_l, srcs)
        E = ctx.n_edges
        b = torch.empty((len(srcs), E), dtype=torch.complex128, device="cuda")
        api.petgem_get_system(ctx.h, b=b)
        x, info, st = ctx.solve(precision=api.PREC_MIXED, tol=1e-10)
        out, _ = ctx.receivers(rx, x)
        b, x, out = b.cpu().numpy(), x.cpu().numpy(), out.cpu().numpy()
    assert np.abs(b_ref).max() > 0
    for i in range(len(srcs)):
        assert np.linalg.norm(b[i] - b_ref[i]) <= 1e-10 * np.linalg.norm(b_ref[i])
        assert info[i]["true_rel_residual"] <= 1e-10
        assert np.linalg.norm(x[i] - x_ref[i]) <= 1e-6 * np.linalg.norm(x_ref[i])
    ep_ref = np.stack([LY.primary_field(rx, s, z_if, sig_l, f) for s in s5])
    es_ref = ref.receivers(x_ref, rx)[0][:, :, 1, :]
    assert np.linalg.norm(out[:, :, 0, :] - ep_ref) <= 1e-10 * np.linalg.norm(ep_ref)
    assert np.linalg.norm(out[:, :, 1, :] - es_ref) <= 1e-6 * np.linalg.norm(es_ref)
    assert np.allclose(out[:, :, 2, :], out[:, :, 0, :] + out[:, :, 1, :])
    # the background matters: the secondary field is that of the block alone (small next to E_p)
    assert np.linalg.norm(es_ref) < 0.5 * np.linalg.norm(ep_ref)
