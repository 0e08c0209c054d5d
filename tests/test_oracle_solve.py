"""Pins for the oracle's assembly, Dirichlet rows, GMRES, receivers and dense LU.

* Global matrix: brute-force dense assembly of the (separately pinned) element matrices.
* Right-hand side: an independent high-order quadrature (Duffy-collapsed tensor Gauss-Legendre)
  of -i w mu0 dsigma int N_k . E_p, built from the expanded basis of Appendix B eqs. B.8-B.13.
* The 4-point rule integrates every polynomial of degree <= 2 exactly.
* GMRES against dense solves; dense LU against numpy.
* Whole space (Section 2 eq. 6 with uniform sigma != sigma_p): with the exact field as boundary data,
  E_s converges at first order in h to the closed form E_p(sigma) - E_p(sigma_p).
* Receivers (Section 3 eq. 7): fields of the form a + b x x lie in the Nedelec space and are
  reproduced exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1808_00186_gb300 import synth
from tests.golden.tables import local_edge_table

MU0 = 4e-7 * math.pi


def dense(sys_):
    rp, col, val, b = sys_.system()
    n = sys_.n_edges
    A = np.zeros((n, n), np.complex128)
    for r in range(n):
        A[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
    return A, b


def small_model(n=2, seed=0):
    m = synth.kuhn_mesh(n, (0.0, 0.0, 0.0), (100.0, 100.0, 100.0), jitter=0.15, seed=seed)
    rng = np.random.default_rng(seed)
    sigma = rng.choice([0.3, 1.0, 2.0], size=m.n_tets)
    src = np.array([[-500.0, 30.0, 40.0, 0, 1.0], [600.0, -200.0, 300.0, 2, 2.0]])
    return m, sigma, 1.0, 1.0, src


def duffy_rule(n):
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1), 0.5 * w
    pts, wts = [], []
    for a, wa in zip(x, w):
        for b, wb in zip(x, w):
            for c, wc in zip(x, w):
                pts.append([a, b * (1 - a), c * (1 - a) * (1 - b)])
                wts.append(wa * wb * wc * (1 - a) ** 2 * (1 - b))
    return np.array(pts), np.array(wts)   # unit tet, total weight 1/6


def expanded_basis(P, x):
    """Eqs. B.7-B.13: lambda_i = (a_i + b_i x + c_i y + d_i z) / (6V) from cofactors; returns [6][3]."""
    C = np.hstack([np.ones((4, 1)), P])
    Ci = np.linalg.inv(C)
    lam = Ci[0] + x @ Ci[1:]
    grad = Ci[1:].T
    out = []
    for a, b in local_edge_table():
        ln = np.linalg.norm(P[b] - P[a])
        out.append(ln * (lam[a] * grad[b] - lam[b] * grad[a]))
    return np.array(out)


def test_global_matrix_brute_force():
    m, sigma, sp, f, src = small_model()
    s = oracle.System(m.nodes, m.tets, sigma, sp, f, src)
    A, b = dense(s)
    edges, te, sg, bd = s.topology()
    n = s.n_edges
    Aref = np.zeros((n, n), np.complex128)
    w = 2 * math.pi * f
    for t in range(m.n_tets):
        K, M, _ = oracle.element(m.nodes[m.tets[t]], sg[t])
        Ae = K + 1j * w * MU0 * sigma[t] * M
        Aref[np.ix_(te[t], te[t])] += Ae
    inner = bd == 0
    Aref[~inner, :] = 0
    Aref[:, ~inner] = 0
    Aref[~inner, ~inner] = 1
    assert np.abs(A - Aref).max() <= 1e-13 * np.abs(Aref).max()
    assert np.allclose(A, A.T, rtol=0, atol=1e-13 * np.abs(A).max())   # complex symmetric
    assert np.all(b[:, ~inner] == 0)


def test_rhs_against_high_order_quadrature():
    m, sigma, sp, f, src = small_model()
    s = oracle.System(m.nodes, m.tets, sigma, sp, f, src)
    _, b = dense(s)
    edges, te, sg, bd = s.topology()
    ref = np.zeros_like(b)
    qp, qw = duffy_rule(7)
    w = 2 * math.pi * f
    for t in range(m.n_tets):
        ds = sigma[t] - sp
        if ds == 0:
            continue
        P = m.nodes[m.tets[t]]
        J = (P[1:] - P[0]).T
        x = P[0] + qp @ J.T
        vol6 = abs(np.linalg.det(J))
        for sc in range(src.shape[0]):
            Ep = oracle.primary_field(x, src[sc], sp, f)
            R = np.zeros(6, np.complex128)
            for xq, wq, e in zip(x, qw, Ep):
                R += wq * vol6 * (expanded_basis(P, xq) @ e)
            for i in range(6):
                if not bd[te[t, i]]:
                    ref[sc, te[t, i]] += -1j * w * MU0 * ds * sg[t, i] * R[i]
    for sc in range(src.shape[0]):
        err = np.linalg.norm(b[sc] - ref[sc]) / np.linalg.norm(ref[sc])
        assert err < 5e-3, err     # the degree-2 rule on 50 m tets, 500 m from the source


def test_four_point_rule_is_degree_two():
    q = oracle.quadrature()
    assert np.allclose(q.sum(axis=1), 1.0, atol=1e-15)
    P = np.array([[0.3, -1.0, 2.0], [2.0, 0.5, 1.0], [-0.5, 2.0, 0.0], [1.0, 1.0, 3.5]])
    vol = abs(np.linalg.det(P[1:] - P[0])) / 6
    x = q @ P
    qp, qw = duffy_rule(4)
    xr = P[0] + qp @ (P[1:] - P[0])
    for ex in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (0, 1, 1), (1, 0, 1), (0, 0, 2)]:
        f = lambda p: np.prod(p ** np.array(ex), axis=1)
        exact = 6 * vol * np.sum(qw * f(xr))
        assert np.sum(vol / 4 * f(x)) == pytest.approx(exact, rel=1e-12, abs=1e-12)


def test_dense_lu_matches_numpy():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(40, 40)) + 1j * rng.normal(size=(40, 40))
    b = rng.normal(size=40) + 1j * rng.normal(size=40)
    assert np.allclose(oracle.dense_solve(A, b), np.linalg.solve(A, b), rtol=1e-11, atol=0)


@pytest.mark.parametrize("n", [2, 3])
def test_gmres_matches_dense_solve(n):
    m = synth.cube_block_model(n)
    src = synth.sources_array(m.sources)
    s = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, src)
    A, b = dense(s)
    xd = oracle.dense_solve(A, b[0])
    assert np.allclose(xd, np.linalg.solve(A, b[0]), rtol=1e-10, atol=1e-10 * np.abs(xd).max())
    x, info, st = s.solve(restart=50, tol=1e-12)
    assert st == oracle.OK and info[0, 2] <= 1e-12
    assert np.linalg.norm(x[0] - xd) <= 1e-9 * np.linalg.norm(xd)
    # GMRES with a restart length >= n converges within one cycle.
    x2, info2, st2 = s.solve(restart=s.n_edges, tol=1e-12)
    assert st2 == oracle.OK and info2[0, 1] <= 2 and info2[0, 0] <= s.n_edges


def test_gmres_reports_non_convergence():
    m = synth.cube_block_model(4)
    s = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    x, info, st = s.solve(restart=10, tol=1e-12, maxit=15)
    assert st == oracle.NOT_CONVERGED and info[0, 0] == 15 and info[0, 2] > 1e-12


def exact_whole_space(m, x):
    src = synth.sources_array(m.sources)[0]
    return oracle.primary_field(x, src, 0.5, m.freq) - oracle.primary_field(x, src, 1.0, m.freq)


def whole_space_error(n):
    m = synth.whole_space_model(n)
    top = oracle.System(m.mesh.nodes, m.mesh.tets, topology_only=True)
    edges, te, sg, bd = top.topology()
    pa, pb = m.mesh.nodes[edges[:, 0]], m.mesh.nodes[edges[:, 1]]
    ln = np.linalg.norm(pb - pa, axis=1)
    t = (pb - pa) / ln[:, None]
    g = np.zeros(edges.shape[0], np.complex128)
    for sgl, w in [(-math.sqrt(0.6), 5 / 9), (0.0, 8 / 9), (math.sqrt(0.6), 5 / 9)]:   # Gauss-Legendre on each edge
        x = pa + 0.5 * (1 + sgl) * (pb - pa)
        g += 0.5 * w * np.einsum("ij,ij->i", exact_whole_space(m, x), t)
    g = np.where(bd == 1, g, 0)
    s = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources),
                      g=g[None, :])
    x, info, st = s.solve(tol=1e-12)
    assert st == oracle.OK
    out, st = s.receivers(x, m.receivers)
    assert st == oracle.OK
    ex = exact_whole_space(m, m.receivers)
    return np.abs(out[0, :, 1, :] - ex).max() / np.abs(ex).max()


@pytest.mark.slow
def test_whole_space_first_order_convergence():
    errs = [whole_space_error(n) for n in (4, 8, 16)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.8 <= r <= 1.3 for r in rates), (errs, rates)
    assert errs[-1] < 0.2


def test_receivers_reproduce_nedelec_fields():
    m = synth.kuhn_mesh(3, (-50.0, -50.0, -50.0), (50.0, 70.0, 40.0), jitter=0.15, seed=2)
    s = oracle.System(m.nodes, m.tets, np.ones(m.n_tets), 1.0, 1.0, np.array([[0.0, 0, 500, 0, 1]]))
    edges, te, sg, bd = s.topology()
    a = np.array([1.0 + 2j, -0.5, 0.25j])
    bv = np.array([0.01, -0.02j, 0.03])
    F = lambda p: a + np.cross(np.broadcast_to(bv, p.shape), p)
    pa, pb = m.nodes[edges[:, 0]], m.nodes[edges[:, 1]]
    x = np.einsum("ij,ij->i", F(0.5 * (pa + pb)), (pb - pa)) / np.linalg.norm(pb - pa, axis=1)
    rng = np.random.default_rng(4)
    rx = rng.uniform([-45, -45, -45], [45, 65, 35], size=(25, 3))
    out, st = s.receivers(x[None, :], rx)
    assert st == oracle.OK
    assert np.allclose(out[0, :, 1, :], F(rx), rtol=0, atol=1e-12 * np.abs(F(rx)).max())
    assert np.allclose(out[0, :, 2, :], out[0, :, 0, :] + out[0, :, 1, :])
    out2, st2 = s.receivers(x[None, :], np.array([[0.0, 0.0, 500.0]]))
    assert st2 == oracle.OUTSIDE and np.isnan(out2).all()
