"""Parity of the learned preconditioner's tensor-core kernels and network with the FP64 oracle
(oracle/learned.py), through the C ABI.

BF16 operands are rounded the same way on both sides (the oracle works in FP64 on the rounded
values), so the convolution kernels differ from the oracle only by FP32 accumulation: bar 1e-4 of
the largest entry.  The whole network keeps its activations in BF16 between layers: bar 5e-2
normwise for its output, loss and gradients.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import learned as OL
from paper_1808_00186_gb300 import api, synth
from paper_1808_00186_gb300 import learned as PL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_00186_gb300 import build
    build.build()
    oracle.build()
    api.load()
    torch.cuda.set_device(0)


def bf16(a):
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t, t.to(torch.float64).numpy()


def rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def to_zyx(a, grid, c):
    gx, gy, gz = grid
    return a.reshape(gz, gy, gx, c)


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 16), (32, 32)])
@pytest.mark.parametrize("grid", [(9, 7, 5), (13, 11, 6)])
def test_conv3d_matches_oracle(cin, cout, grid):
    rng = np.random.default_rng(cin + cout + grid[0])
    V = grid[0] * grid[1] * grid[2]
    xt, x = bf16(rng.normal(size=(V, cin)))
    wt, w = bf16(rng.normal(size=(27, cout, cin)) * 0.2)
    bias = rng.normal(size=cout).astype(np.float32)
    dev = "cuda"
    xg, wg, bg = xt.to(dev), wt.to(dev), torch.as_tensor(bias).to(dev)
    y32 = torch.empty((V, cout), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    api.petgem_nn_conv3d(stream, grid, cin, cout, xg, wg, bg, False, y32, True)
    ref = OL.conv3d(to_zyx(x, grid, cin), w, bias.astype(np.float64)).reshape(V, cout)
    assert rel_max(y32.cpu().numpy(), ref) <= 1e-4
    ybf = torch.empty((V, cout), dtype=torch.bfloat16, device=dev)
    api.petgem_nn_conv3d(stream, grid, cin, cout, xg, wg, bg, True, ybf, False)
    assert rel_max(ybf.float().cpu().numpy(), np.maximum(ref, 0.0)) <= 1e-2


@pytest.mark.parametrize("cin,cout,grid", [
    ((16, 16, (1, 1, 1))),      # one voxel: the brick is all halo
    ((16, 16, (8, 16, 3))),     # exactly one 8 x 16 tile per plane
    ((32, 32, (17, 33, 5))),    # several tiles in x and y, each with a one-voxel tail
    ((16, 16, (65, 65, 23))),   # two planes per CTA on a 152-SM GPU, the last group with one
    ((16, 32, (65, 65, 41))),   # four planes per CTA, the last group with one
    ((32, 16, (66, 50, 41))),
])
def test_conv3d_tiles_ragged_tails_and_plane_groups_match_oracle(cin, cout, grid):
    """The convolution's tiles are 8 x 16 voxels of a plane, 1, 2 or 4 planes per CTA (by grid
    size); every boundary of that tiling, and the grid's own, must give the oracle's result."""
    rng = np.random.default_rng(7 * cin + cout + grid[2])
    V = grid[0] * grid[1] * grid[2]
    xt, x = bf16(rng.normal(size=(V, cin)))
    wt, w = bf16(rng.normal(size=(27, cout, cin)) * 0.2)
    bias = rng.normal(size=cout).astype(np.float32)
    xg, wg, bg = xt.to("cuda"), wt.to("cuda"), torch.as_tensor(bias).to("cuda")
    y32 = torch.full((V, cout), float("nan"), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    api.petgem_nn_conv3d(stream, grid, cin, cout, xg, wg, bg, False, y32, True)
    ref = OL.conv3d(to_zyx(x, grid, cin), w, bias.astype(np.float64)).reshape(V, cout)
    got = y32.cpu().numpy()
    assert np.isfinite(got).all()  # every voxel written
    assert rel_max(got, ref) <= 1e-4


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 16), (32, 32)])
def test_conv3d_weight_gradient_matches_oracle(cin, cout):
    grid = (11, 9, 7)
    rng = np.random.default_rng(7 + cin * cout)
    V = grid[0] * grid[1] * grid[2]
    xt, x = bf16(rng.normal(size=(V, cin)))
    dyt, dy = bf16(rng.normal(size=(V, cout)))
    dw = torch.empty((27, cout, cin), dtype=torch.float32, device="cuda")
    api.petgem_nn_conv3d_wgrad(torch.cuda.current_stream().cuda_stream, grid, cin, cout, xt.cuda(), dyt.cuda(), dw)
    _, ref, _ = OL.conv3d_backward(to_zyx(x, grid, cin), np.zeros((27, cout, cin)), to_zyx(dy, grid, cout))
    assert rel_max(dw.cpu().numpy(), ref) <= 1e-4


def lattice_case(n, seed):
    m = PL.random_block_model(n, seed)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    return m, ref


def oracle_maps(m, ref, cells):
    """The auxiliary-space maps, scales, features and the system matrix of the oracle's assembly
    on a lattice of cells = (nx, ny, nz)."""
    import scipy.sparse as sp
    nx, ny, nz = (cells, cells, cells) if np.isscalar(cells) else cells
    rp, col, val, b = ref.system()
    edges, _, _, _ = ref.topology()
    A = sp.csr_matrix((val, col, rp), shape=(ref.n_edges, ref.n_edges))
    G, Pi = OL.aux_operators(edges, m.mesh.nodes, (nx, ny, nz))
    sg, sp_ = OL.aux_scales(G, Pi, A)
    nd = m.mesh.nodes
    h = (abs(nd[1, 0] - nd[0, 0]) * abs(nd[nx + 1, 1] - nd[0, 1]) * abs(nd[(nx + 1) * (ny + 1), 2] - nd[0, 2])) ** (1 / 3)
    feat = OL.node_features(m.sigma, (nx, ny, nz), m.sigma_p, m.freq, h)
    return A, b, G, Pi, sg, sp_, feat


def anisotropic_case(cells=(32, 4, 4), seed=3):
    """A jittered 32 x 4 x 4 lattice (five network levels along x, so c3 and c5 act on two levels
    each) with a resistive half and a conductive block, 1.5 Hz."""
    nx, ny, nz = cells
    xs = [np.linspace(-1000.0, 1000.0, nx + 1), np.linspace(-250.0, 250.0, ny + 1), np.linspace(-250.0, 250.0, nz + 1)]
    mesh = synth.kuhn_mesh_axes(xs, jitter=0.1, seed=seed)
    cen = mesh.centroids()
    sigma = np.where(cen[:, 0] > 300.0, 0.05, 1.0)
    sigma[(cen[:, 0] < -400.0) & (cen[:, 2] < 0.0)] = 4.0
    m = synth.Model("aniso", mesh, sigma, 1.0, 1.5, [synth.Dipole(1.0, 1.0, 1.0, 0, 1.0)], np.zeros((1, 3)))
    ref = oracle.System(mesh.nodes, mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    return m, ref

def perturbed_iterate(xstar, seed):
    rng = np.random.default_rng(seed)
    return xstar * (1 + 0.3 * rng.normal(size=xstar.shape)) + 1e-3 * np.abs(xstar).max() * rng.normal(size=xstar.shape)


def test_auxiliary_space_maps_match_oracle():
    """With all weights zero the network's output is its last bias b at every node, so
    z = D^-1 r + G phi + Pi w is a fixed function of the auxiliary maps, their diagonal scales and
    the residual's scale s: the kernels must reproduce the oracle's z to FP32 rounding."""
    n = 7
    m, ref = lattice_case(n, 21)
    A, b, G, Pi, sg, sp_, feat = oracle_maps(m, ref, n)
    xstar = ref.solve(tol=1e-10)[0][0]
    x = perturbed_iterate(xstar, 2)
    r = b[0] - ref.spmv(x)
    lay, n_par = PL.layout()
    p = np.zeros(n_par, np.float32)
    bias = np.random.default_rng(4).normal(size=16).astype(np.float32)
    bias[8:] = 0.0
    p[lay[-1][2]:lay[-1][2] + 16] = bias
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        api.petgem_learned_create(ctx.h, n, n, n)
        api.petgem_learned_params(ctx.h, set_params=p)
        r_t = ctx.tensor(r)
        z_t = torch.empty_like(r_t)
        api.petgem_learned_apply(ctx.h, r_t, z_t)
        z = z_t.cpu().numpy()
    _, s = OL.hx_input(r, G, Pi, sg, sp_, feat)
    y = np.tile(bias.astype(np.float64), (G.shape[1], 1))
    zr = OL.hx_direction(y, r, s, G, Pi, sg, sp_, A.diagonal())
    assert np.linalg.norm(z - zr) <= 1e-5 * np.linalg.norm(zr)
    # the correction is a real part of z (not just the Jacobi term)
    assert np.linalg.norm(zr - r / A.diagonal()) >= 1e-2 * np.linalg.norm(zr)


def test_network_forward_loss_and_gradients_match_oracle():
    cells = (32, 4, 4)
    m, ref = anisotropic_case(cells)
    A, b, G, Pi, sg, sp_, feat = oracle_maps(m, ref, cells)
    assert OL.levels((cells[2] + 1, cells[1] + 1, cells[0] + 1)) == 5
    rng = np.random.default_rng(1)
    x = (rng.normal(size=ref.n_edges) + 1j * rng.normal(size=ref.n_edges)) * 1e-9
    x[ref.topology()[3] == 1] = 0.0
    p = PL.init_params(5)
    lay, _ = PL.layout()
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        api.petgem_learned_create(ctx.h, *cells)
        api.petgem_learned_params(ctx.h, set_params=p)
        loss = api.petgem_learned_train_step(ctx.h, ctx.tensor(x[None, :]), 1e-12)
        g_gpu = api.petgem_learned_params(ctx.h, grad=True)
        r_t = ctx.tensor(b[0] - ref.spmv(x))
        z_t = torch.empty_like(r_t)
        api.petgem_learned_apply(ctx.h, r_t, z_t)
        z = z_t.cpu().numpy()
    r = b[0] - ref.spmv(x)
    xin, s = OL.hx_input(r, G, Pi, sg, sp_, feat)
    P = PL.unflatten(p)
    shape = (cells[2] + 1, cells[1] + 1, cells[0] + 1)
    # the oracle rounds weights, activations and gradients to bfloat16 where the kernels store
    # them, so both sides take the same rounding steps; what remains is FP32 against FP64
    # accumulation, which can flip single roundings
    y, cache = OL.forward(P, xin.reshape(*shape, 16), round_bf16=True)
    L, gy = OL.hx_angle_loss(y.reshape(-1, 16), r, s, G, Pi, sg, sp_, A.diagonal(), ref.spmv)
    gref = OL.backward(P, cache, gy.reshape(*shape, 16))
    assert abs(loss - L) <= 1e-3 * L
    for name, w, bb, ci, co in lay:
        for got, ref_ in ((g_gpu[w:w + 27 * co * ci].reshape(27, co, ci), gref[name + ".W"]),
                          (g_gpu[bb:bb + co], gref[name + ".b"])):
            got, ref_ = got.reshape(-1).astype(np.float64), ref_.reshape(-1)
            err = np.linalg.norm(got - ref_) / max(np.linalg.norm(ref_), 1e-30)
            cos = got @ ref_ / max(np.linalg.norm(got) * np.linalg.norm(ref_), 1e-300)
            print("%s: normwise %.3f cosine %.5f" % (name, err, cos))
            assert err <= 2e-2 and cos >= 0.9998, name
    # apply: z = D^-1 r + G phi + Pi w from the network's output
    zr = OL.hx_direction(y.reshape(-1, 16), r, s, G, Pi, sg, sp_, A.diagonal())
    assert np.linalg.norm(z - zr) <= 1e-3 * np.linalg.norm(zr - r / A.diagonal())


def test_learned_fgmres_gains_over_jacobi_on_unseen_models():
    """A network trained on the GPU (the library's own forward and backward kernels) on residuals
    of the plain solver over random block models lowers the FGMRES iteration count against plain
    Jacobi GMRES(50) on models it has not seen, without falling back, and the answer is the
    oracle's (the FP64 true residual decides convergence)."""
    n = 12
    params, hist = PL.train(n=n, models=32, epochs=8, lr=2e-3, seed=1, samples_per_model=8)
    assert hist["loss"][-1] < hist["loss"][0]
    res = PL.evaluate(params, n, [10000, 10001, 10002])
    for rec in res:
        assert rec["status_learned"] == api.OK and rec["fell_back"] == 0
        assert rec["relres_learned"] <= 1e-8
    ratio = np.mean([r["iters_learned"] / r["iters_jacobi"] for r in res])
    print("\nlearned FGMRES / Jacobi GMRES iterations on unseen n=%d models: %s (mean ratio %.2f)"
          % (n, [(r["iters_learned"], r["iters_jacobi"]) for r in res], ratio))
    assert ratio <= 0.75
    m, ref = lattice_case(n, 10000)
    xr = ref.solve(tol=1e-10)[0][0]
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        api.petgem_learned_create(ctx.h, n, n, n)
        api.petgem_learned_params(ctx.h, set_params=params)
        xl, info_l, st = ctx.solve(precision=api.PREC_MIXED, precond=api.PRECOND_LEARNED)
        xl = xl.cpu().numpy()[0]
    assert st == api.OK and info_l[0]["fell_back"] == 0
    assert np.linalg.norm(xl - xr) <= 1e-6 * np.linalg.norm(xr)


def test_learned_cycles_replayed_as_cuda_graphs_are_bit_identical():
    """Learned FGMRES cycles captured once as a CUDA graph and replayed give the direct launches'
    solution and iteration record bit for bit, in both precisions, with the committed weights
    (cycles that stop early skip the remaining network applications in both modes)."""
    n = 10
    m, ref = lattice_case(n, 10003)
    p = np.load(PL.WEIGHTS)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        api.petgem_learned_create(ctx.h, n, n, n)
        api.petgem_learned_params(ctx.h, set_params=p)
        for prec in (api.PREC_MIXED, api.PREC_C128):
            out = []
            for g in (0, 1, 1):
                x, info, st = ctx.solve(precision=prec, precond=api.PRECOND_LEARNED, use_graphs=g)
                assert st == api.OK and info[0]["true_rel_residual"] <= 1e-8
                out.append((x.cpu().numpy(), info))
            for x, info in out[1:]:
                assert np.array_equal(x, out[0][0]) and info == out[0][1]


@pytest.mark.parametrize("precision", [api.PREC_MIXED, api.PREC_C128])
def test_learned_block_fgmres_matches_oracle_and_single_source_solves(precision):
    """Several sources of one frequency in one learned block solve (flexible GMRES on interleaved
    block vectors, the network applied to every source's column, one SpMM per step): every
    source meets the FP64 residual bar, matches its own oracle solution and receivers, and takes
    about the iterations of its single-source learned solve (the SpMM sums in another order)."""
    n = 12
    m = PL.random_block_model(n, 10004)
    rng = np.random.default_rng(5)
    m.sources = [synth.Dipole(float(x), float(y), float(z), 0, 1.0)
                 for x, y, z in zip(rng.uniform(-300, 300, 5), rng.uniform(-300, 300, 5), rng.uniform(-200, 200, 5))]
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    xr, _, st_r = ref.solve(tol=1e-8)
    assert st_r == oracle.OK
    _, _, _, b = ref.system()
    rr, _ = ref.receivers(xr, m.receivers)
    p = np.load(PL.WEIGHTS)
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        api.petgem_learned_create(ctx.h, n, n, n)
        api.petgem_learned_params(ctx.h, set_params=p)
        xb, ib, st = ctx.solve(precision=precision, precond=api.PRECOND_LEARNED, batch=0, tol=1e-8)
        assert st == api.OK
        xs, isg, st = ctx.solve(precision=precision, precond=api.PRECOND_LEARNED, batch=1, tol=1e-8)
        assert st == api.OK
        rcv = torch.empty((len(m.sources), len(m.receivers), 3, 3), dtype=torch.complex128, device="cuda")
        api.petgem_receivers(ctx.h, torch.as_tensor(m.receivers, device="cuda"), xb, rcv)
    xb = xb.cpu().numpy()
    for s in range(len(m.sources)):
        assert ib[s]["status"] == api.OK and ib[s]["true_rel_residual"] <= 1e-8, (s, ib[s])
        assert np.linalg.norm(b[s] - ref.spmv(xb[s])) / np.linalg.norm(b[s]) <= 1.0001e-8
        assert np.linalg.norm(xb[s] - xr[s]) / np.linalg.norm(xr[s]) <= 1e-6
        assert ib[s]["fell_back"] == isg[s]["fell_back"]
        assert abs(ib[s]["iters"] - isg[s]["iters"]) <= 0.1 * isg[s]["iters"] + 5, (s, ib[s], isg[s])
    assert np.linalg.norm(rcv.cpu().numpy() - rr) / np.linalg.norm(rr) <= 1e-6
    print("\nlearned block / single-source iterations:", [(i["iters"], j["iters"]) for i, j in zip(ib, isg)])


def test_learned_cycle_graph_replayed_for_another_model_of_the_same_size():
    """A captured learned cycle is kept when a new mesh and assembly of the same sizes move none
    of its buffers: the second model's solve replays the first model's graph and must equal its
    own direct launches bit for bit."""
    n = 10
    p = np.load(PL.WEIGHTS)
    models = [PL.random_block_model(n, seed) for seed in (10005, 10006)]
    out = {}
    with api.Context(0) as ctx:
        for g in (1, 0):
            for k, m in enumerate(models):
                ctx.mesh(m.mesh.nodes, m.mesh.tets)
                ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
                api.petgem_learned_create(ctx.h, n, n, n)
                if not out:
                    api.petgem_learned_params(ctx.h, set_params=p)
                x, info, st = ctx.solve(precision=api.PREC_MIXED, precond=api.PRECOND_LEARNED, use_graphs=g)
                assert st == api.OK and info[0]["true_rel_residual"] <= 1e-8
                out[(g, k)] = (x.cpu().numpy(), info)
    for k in range(2):
        assert np.array_equal(out[(1, k)][0], out[(0, k)][0]) and out[(1, k)][1] == out[(0, k)][1]
