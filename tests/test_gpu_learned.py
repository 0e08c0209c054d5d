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


def oracle_input(m, ref, x, n):
    """The network input grid defined in the library's documentation, built from the oracle's
    assembled system: residual r = b - A x scaled by 1 / RMS(r), plus the two node features."""
    rp, col, val, b = ref.system()
    edges, _, _, _ = ref.topology()
    r = b[0] - ref.spmv(x)
    diag = np.array([val[rp[i]:rp[i + 1]][col[rp[i]:rp[i + 1]] == i][0] for i in range(ref.n_edges)])
    s = math.sqrt(np.mean(np.abs(r) ** 2))
    slot = OL.edge_grid_index(edges, n)
    grid = OL.edges_to_grid(r, slot, (n + 1) ** 3, 1.0 / s)
    # node features: cell whose lowest corner is the node (clamped), log10(sigma/sigma_p), log10(w mu0 sigma h^2)
    sig_cell = m.sigma.reshape(n, n, n, 6).mean(axis=3)        # [k][j][i]
    idx = np.minimum(np.arange(n + 1), n - 1)
    sc = sig_cell[np.ix_(idx, idx, idx)].reshape(-1)
    h = 2000.0 / n
    w = 2 * math.pi * m.freq * 4e-7 * math.pi
    grid[:, 14] = np.log10(sc / m.sigma_p)
    grid[:, 15] = np.log10(w * sc * h * h)
    return grid, r, s, slot, diag


def test_network_forward_loss_and_gradients_match_oracle():
    n = 6
    m, ref = lattice_case(n, 11)
    xstar = ref.solve(tol=1e-12)[0][0]
    rng = np.random.default_rng(1)
    x = xstar * (1 + 0.3 * rng.normal(size=xstar.shape)) + 1e-3 * np.abs(xstar).max() * rng.normal(size=xstar.shape)
    p = PL.init_params(5)
    lay, _ = PL.layout()
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        api.petgem_learned_create(ctx.h, n, n, n)
        api.petgem_learned_params(ctx.h, set_params=p)
        loss = api.petgem_learned_train_step(ctx.h, ctx.tensor(x[None, :]), 1e-12)
        g_gpu = api.petgem_learned_params(ctx.h, grad=True)
        r_t = ctx.tensor(ref.system()[3][0] - ref.spmv(x))
        z_t = torch.empty_like(r_t)
        api.petgem_learned_apply(ctx.h, r_t, z_t)
        z = z_t.cpu().numpy()
    grid, r, s, slot, diag = oracle_input(m, ref, x, n)
    P = PL.unflatten(p)
    shape = (n + 1, n + 1, n + 1)
    y, cache = OL.forward(P, grid.reshape(*shape, 16))
    L, gy = OL.angle_loss(y.reshape(-1, 16), r, slot, ref.spmv, diag)
    gref = OL.backward(P, cache, gy.reshape(*shape, 16))
    assert abs(loss - L) <= 5e-2 * L
    for name, w, b, ci, co in lay:
        gw = g_gpu[w:w + 27 * co * ci].reshape(27, co, ci)
        assert np.linalg.norm(gw - gref[name + ".W"]) <= 5e-2 * np.linalg.norm(gref[name + ".W"]) + 1e-12, name
        gb = g_gpu[b:b + co]
        assert np.linalg.norm(gb - gref[name + ".b"]) <= 5e-2 * np.linalg.norm(gref[name + ".b"]) + 1e-12, name
    # apply: z = s N(r / s) on the edges
    corr = s * OL.grid_to_edges(y.reshape(-1, 16), slot)
    assert np.linalg.norm(z - corr) <= 5e-2 * np.linalg.norm(corr)


def test_learned_fgmres_converges_and_is_compared_with_jacobi():
    n = 12
    params, hist = PL.train(n=n, models=6, epochs=3, lr=2e-3, seed=1)
    assert hist["loss"][-1] < hist["loss"][0]
    m, ref = lattice_case(n, 999)
    xr = ref.solve(tol=1e-10)[0][0]
    with api.Context(0) as ctx:
        ctx.mesh(m.mesh.nodes, m.mesh.tets)
        ctx.assemble(m.freq, m.sigma, m.sigma_p, m.sources)
        api.petgem_learned_create(ctx.h, n, n, n)
        api.petgem_learned_params(ctx.h, set_params=params)
        xj, info_j, _ = ctx.solve(precision=api.PREC_MIXED)
        xl, info_l, st = ctx.solve(precision=api.PREC_MIXED, precond=api.PRECOND_LEARNED)
        xl = xl.cpu().numpy()[0]
    assert st == api.OK and info_l[0]["true_rel_residual"] <= 1e-8
    assert np.linalg.norm(xl - xr) <= 1e-6 * np.linalg.norm(xr)
    print("\nlearned FGMRES: %d iterations (fell back: %d), Jacobi GMRES: %d iterations"
          % (info_l[0]["iters"], info_l[0]["fell_back"], info_j[0]["iters"]))
