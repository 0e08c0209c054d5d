"""Pins for the learned-preconditioner oracle (oracle/learned.py).

The paper has no learned part, so these pins check the oracle against mathematics only:
a brute-force convolution loop, adjointness of pooling / upsampling and of the convolution's
input gradient, central finite differences of the whole network's loss, and the bijectivity of
the edge <-> grid map on Kuhn lattices.  The network is "parity unpinned" against the paper.
"""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_1808_00186_gb300 import synth


def brute_conv(x, W, b):
    Z, Y, X, Ci = x.shape
    Co = W.shape[1]
    y = np.zeros((Z, Y, X, Co))
    for z in range(Z):
        for yy in range(Y):
            for xx in range(X):
                acc = b.copy()
                for t, (dx, dy, dz) in enumerate(L.OFFS):
                    a, bb, c = xx + dx, yy + dy, z + dz
                    if 0 <= a < X and 0 <= bb < Y and 0 <= c < Z:
                        acc = acc + W[t] @ x[c, bb, a]
                y[z, yy, xx] = acc
    return y


def test_conv3d_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 4, 5, 3))
    W = rng.normal(size=(27, 2, 3))
    b = rng.normal(size=2)
    assert np.allclose(L.conv3d(x, W, b), brute_conv(x, W, b), rtol=1e-12, atol=1e-12)
    # The tap order is (dx fastest): tap 14 = (+1, 0, 0) reads the +x neighbour.
    assert L.OFFS[14] == (1, 0, 0) and L.OFFS[13] == (0, 0, 0) and L.OFFS[22] == (0, 0, 1)


def test_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(5, 3, 6, 2))
    yc = rng.normal(size=(3, 2, 3, 2))
    assert np.isclose(np.sum(L.pool(x) * yc), np.sum(x * L.pool_backward(yc, x.shape)))
    assert np.isclose(np.sum(L.upsample(yc, x.shape) * x), np.sum(yc * L.upsample_backward(x, yc.shape)))
    W = rng.normal(size=(27, 4, 2))
    dy = rng.normal(size=(5, 3, 6, 4))
    dx, dW, db = L.conv3d_backward(x, W, dy)
    assert np.isclose(np.sum(L.conv3d(x, W, np.zeros(4)) * dy), np.sum(x * dx))
    # pooled values are averages: constants are preserved
    assert np.allclose(L.pool(np.ones((5, 5, 5, 1))), 1.0)


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    p = L.init_params(seed=3)
    x = rng.normal(size=(5, 6, 7, L.N_IN))
    t = rng.normal(size=(5, 6, 7, 16))
    _, dy, cache = L.loss(p, x, t)
    g = L.backward(p, cache, dy)
    for name in ["c1.W", "c2.W", "c4.W", "c5.b", "c7.W", "c3.b"]:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, 3, replace=False):
            if name == "c7.W" and np.unravel_index(idx, p[name].shape)[1] >= L.N_OUT:
                continue
            old = flat[idx]
            eps = 1e-5 * max(1.0, abs(old))
            flat[idx] = old + eps
            lp, _, _ = L.loss(p, x, t)
            flat[idx] = old - eps
            lm, _, _ = L.loss(p, x, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-8, abs(fd)) + 1e-10, (name, idx, fd, an)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_edge_grid_map_is_injective(n):
    m = synth.kuhn_mesh(n, (0, 0, 0), (1, 1, 1), jitter=0.1 if n > 2 else 0.0)
    s = oracle.System(m.nodes, m.tets, topology_only=True)
    edges, _, _, _ = s.topology()
    g = L.edge_grid_index(edges, n)
    assert np.all(g >= 0) and len(np.unique(g)) == len(g)
    assert g.max() < (n + 1) ** 3 * 7
    # every lattice direction appears, and axis edges number 3 n (n+1)^2
    cls = g % 7
    assert np.sum(cls < 3) == 3 * n * (n + 1) ** 2


def test_angle_loss_gradient_by_finite_differences():
    from paper_1808_00186_gb300 import synth as S
    m = S.cube_block_model(3)
    sysm = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, S.sources_array(m.sources))
    edges, _, _, _ = sysm.topology()
    rp, col, val, b = sysm.system()
    diag = np.array([val[rp[i]:rp[i + 1]][col[rp[i]:rp[i + 1]] == i][0] for i in range(sysm.n_edges)])
    slot = L.edge_grid_index(edges, 3)
    rng = np.random.default_rng(0)
    y = rng.normal(size=(4 ** 3, 16))
    r = rng.normal(size=sysm.n_edges) + 1j * rng.normal(size=sysm.n_edges)
    loss, gy = L.angle_loss(y, r, slot, sysm.spmv, diag)
    assert 0.0 <= loss <= 1.0
    for idx in rng.choice(y.size, 12, replace=False):
        i, c = np.unravel_index(idx, y.shape)
        old = y[i, c]
        y[i, c] = old + 1e-6
        lp, _ = L.angle_loss(y, r, slot, sysm.spmv, diag)
        y[i, c] = old - 1e-6
        lm, _ = L.angle_loss(y, r, slot, sysm.spmv, diag)
        y[i, c] = old
        assert abs((lp - lm) / 2e-6 - gy[i, c]) <= 1e-6 * max(1.0, abs(gy[i, c])), (i, c)
    # the exact correction direction z = D A^{-1} r has zero loss
    A = np.zeros((sysm.n_edges, sysm.n_edges), complex)
    for i in range(sysm.n_edges):
        A[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    z = diag * np.linalg.solve(A, r)
    yz = L.edges_to_grid(z, slot, 4 ** 3)
    l0, _ = L.angle_loss(yz, r, slot, sysm.spmv, diag)
    assert l0 < 1e-10


# ---------------------------------------------------------------- auxiliary-space preconditioner
def hx_case(n, seed=3, jitter=0.15):
    """A jittered Kuhn lattice with a random block model, its oracle system as a scipy matrix."""
    import scipy.sparse as sp
    from paper_1808_00186_gb300 import learned as PL
    m = PL.random_block_model(n, seed)
    mesh = synth.kuhn_mesh(n, (-1000.0,) * 3, (1000.0,) * 3, jitter=jitter)
    ref = oracle.System(mesh.nodes, mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    rp, col, val, b = ref.system()
    A = sp.csr_matrix((val, col, rp), shape=(ref.n_edges, ref.n_edges))
    edges, _, _, bd = ref.topology()
    return m, mesh, ref, A, edges, bd


def test_gradient_and_vector_maps_reproduce_fields_they_represent_exactly():
    """The degrees of freedom of the edge basis are tangential components (a constant field E0
    has DOFs E0 . t_e / |t_e|, as the element pins fix): G of the nodal values of a linear function
    a . x is the DOF vector of its gradient a, and Pi of a constant vector field v is the DOF vector
    of v, exactly, on every edge whose two nodes are interior."""
    n = 5
    _, mesh, ref, A, edges, bd = hx_case(n)
    G, Pi = L.aux_operators(edges, mesh.nodes, n)
    inner = L.interior_nodes(n)
    both = inner[edges[:, 0]] & inner[edges[:, 1]]
    assert both.sum() > 0 and inner.sum() == (n - 1) ** 3
    a = np.array([0.3, -1.7, 2.2])
    t = mesh.nodes[edges[:, 1]] - mesh.nodes[edges[:, 0]]
    t = t / np.linalg.norm(t, axis=1)[:, None]
    phi = np.where(inner, mesh.nodes @ a, 0.0)
    assert np.allclose((G @ phi)[both], (t @ a)[both], rtol=1e-13, atol=1e-9)
    v = np.array([1.1, 0.4, -0.8])
    w = np.where(inner[:, None], v[None, :], 0.0).reshape(-1)
    assert np.allclose((Pi @ w)[both], (t @ v)[both], rtol=1e-13, atol=1e-9)
    # boundary edges (Dirichlet rows) receive nothing from either space
    assert np.all((abs(G) @ np.ones(G.shape[1]))[bd == 1] == 0)
    assert np.all((abs(Pi) @ np.ones(Pi.shape[1]))[bd == 1] == 0)


def test_gradient_space_diagonal_is_the_nodal_stiffness_times_i_omega_mu0():
    """K annihilates discrete gradients, so diag(G^T A G) = i w mu0 diag(G^T M_sigma G), and
    G^T M_sigma G is the P1 nodal stiffness with coefficient sigma: its diagonal is
    sum over the node's tets of sigma V |grad lambda_i|^2 (barycentric gradients, closed form)."""
    n = 4
    m, mesh, ref, A, edges, bd = hx_case(n, seed=5)
    G, Pi = L.aux_operators(edges, mesh.nodes, n)
    dg = (G.T @ A @ G).diagonal()
    inner = L.interior_nodes(n)
    wmu0 = 2.0 * np.pi * m.freq * 4e-7 * np.pi
    stiff = np.zeros(mesh.nodes.shape[0])
    for t, tet in enumerate(mesh.tets):
        _, grad, _, vol = oracle.geometry(mesh.nodes[tet])
        for k in range(4):
            stiff[tet[k]] += m.sigma[t] * vol * grad[k] @ grad[k]
    assert np.all(np.abs(dg.real[inner]) <= 1e-9 * np.abs(dg.imag[inner]))
    assert np.allclose(dg.imag[inner], wmu0 * stiff[inner], rtol=1e-10)
    sg, sp_ = L.aux_scales(G, Pi, A)
    assert np.allclose(sg[inner], 1.0 / np.sqrt(wmu0 * stiff[inner]), rtol=1e-10)
    assert np.all(sg[~inner] == 0) and np.all(sp_[~inner] == 0) and np.all(sp_[inner] > 0)
    # the vector space's diagonal is the diagonal of the explicit Galerkin product, node by node
    dp = np.abs((Pi.T @ A @ Pi).diagonal()).reshape(-1, 3)
    assert np.allclose(sp_[inner], 1.0 / np.sqrt(dp[inner]), rtol=1e-12)


def test_hx_loss_gradient_by_finite_differences_and_exact_auxiliary_solves():
    n = 3
    m, mesh, ref, A, edges, bd = hx_case(n, seed=2, jitter=0.1)
    G, Pi = L.aux_operators(edges, mesh.nodes, n)
    sg, sp_ = L.aux_scales(G, Pi, A)
    diag = A.diagonal()
    feat = L.node_features(m.sigma, (n, n, n), m.sigma_p, m.freq, 2000.0 / n)
    rng = np.random.default_rng(0)
    r = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    r[bd == 1] = 0.0
    x, s = L.hx_input(r, G, Pi, sg, sp_, feat)
    # the input is normalised: RMS over the interior nodes' four complex channels is one
    inner = L.interior_nodes(n)
    assert np.isclose((x[inner, :8] ** 2).sum() / (4 * inner.sum()), 1.0)
    assert np.all(x[~inner, :8] == 0)
    y = rng.normal(size=x.shape)
    loss, gy = L.hx_angle_loss(y, r, s, G, Pi, sg, sp_, diag, ref.spmv)
    assert 0.0 <= loss <= 1.0
    for idx in rng.choice(np.nonzero(inner)[0], 6, replace=False):
        for c in (0, 1, 3, 7):
            old = y[idx, c]
            y[idx, c] = old + 1e-6
            lp, _ = L.hx_angle_loss(y, r, s, G, Pi, sg, sp_, diag, ref.spmv)
            y[idx, c] = old - 1e-6
            lm, _ = L.hx_angle_loss(y, r, s, G, Pi, sg, sp_, diag, ref.spmv)
            y[idx, c] = old
            assert abs((lp - lm) / 2e-6 - gy[idx, c]) <= 1e-6 * max(1.0, abs(gy[idx, c])), (idx, c)
    assert np.all(gy[:, 8:] == 0)
    # with the exact auxiliary solutions encoded in y, the direction is the additive
    # auxiliary-space preconditioner D^-1 r + G (G^T A G)^-1 G^T r + Pi (Pi^T A Pi)^-1 Pi^T r
    import scipy.sparse.linalg as spl
    ig, ip = np.nonzero(sg)[0], np.nonzero(sp_.reshape(-1))[0]
    phi = np.zeros(G.shape[1], complex)
    phi[ig] = spl.spsolve((G.T @ A @ G)[ig][:, ig].tocsc(), (G.T @ r)[ig])
    w = np.zeros(Pi.shape[1], complex)
    w[ip] = spl.spsolve((Pi.T @ A @ Pi)[ip][:, ip].tocsc(), (Pi.T @ r)[ip])
    ye = np.zeros_like(y)
    ye[ig, 0], ye[ig, 1] = (phi[ig] / (s * sg[ig])).real, (phi[ig] / (s * sg[ig])).imag
    wn, spn = w.reshape(-1, 3), sp_
    ok = spn > 0
    ye[:, 2:5] = np.where(ok, (wn / np.where(ok, s * spn, 1)).real, 0)
    ye[:, 5:8] = np.where(ok, (wn / np.where(ok, s * spn, 1)).imag, 0)
    z = L.hx_direction(ye, r, s, G, Pi, sg, sp_, diag)
    assert np.allclose(z, r / diag + G @ phi + Pi @ w, rtol=1e-10, atol=1e-14 * np.abs(z).max())
    # and that preconditioner lowers the one-step residual angle below Jacobi's on this residual
    zj = r / diag
    ang = lambda zz: 1 - abs(np.vdot(r, A @ zz)) ** 2 / (np.vdot(A @ zz, A @ zz).real * np.vdot(r, r).real)
    assert ang(z) < ang(zj)


def test_depth_grows_with_the_grid_and_shared_weights_get_every_levels_gradient():
    """Poolings continue until the coarsest grid has at most 3 nodes per axis: 33 nodes a side gives
    33, 17, 9, 5, 3 (five levels), 65 gives six.  On a five-level grid c3 and c5 act on two levels
    each; central finite differences of the whole network's loss check that their gradients
    collect both uses."""
    assert [L.levels((g, g, g)) for g in (5, 7, 13, 33, 65, 97)] == [3, 3, 4, 5, 6, 7]
    assert L.levels((65, 9, 5)) == 6
    rng = np.random.default_rng(7)
    p = L.init_params(seed=4)
    x = rng.normal(size=(5, 6, 33, L.N_IN))
    t = rng.normal(size=(5, 6, 33, 16))
    _, dy, cache = L.loss(p, x, t)
    assert cache["L"] == 5
    g = L.backward(p, cache, dy)
    for name in ["c3.W", "c5.W", "c4.W", "c3.b", "c5.b", "c1.W"]:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, 3, replace=False):
            old = flat[idx]
            eps = 1e-5 * max(1.0, abs(old))
            flat[idx] = old + eps
            lp, _, _ = L.loss(p, x, t)
            flat[idx] = old - eps
            lm, _, _ = L.loss(p, x, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-8, abs(fd)) + 1e-10, (name, idx, fd, an)


def test_bf16_rounding_is_round_to_nearest_even():
    """Values of the bfloat16 grid (8 significand bits) stay, halfway cases go to the even
    neighbour, others to the nearest; the rounding matches torch's float -> bfloat16 conversion."""
    eps = 2.0 ** -7                         # spacing of bfloat16 in [1, 2)
    v = np.array([1.0, 1.0 + eps, 1.0 + eps / 2, 1.0 + 3 * eps / 2, 1.0 + 0.3 * eps, -2.5, 3.0e38, 1e-39])
    out = L.bf16(v)
    assert out[0] == 1.0 and out[1] == 1.0 + eps
    assert out[2] == 1.0                    # tie -> even (1.0)
    assert out[3] == 1.0 + 2 * eps          # tie -> even (1 + 2 eps)
    assert out[4] == 1.0 and out[5] == -2.5
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = rng.normal(size=1000) * 10.0 ** rng.uniform(-20, 20, 1000)
    ref = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16(x), ref)
