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
