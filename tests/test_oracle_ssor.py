"""Pins for the multicolour SSOR oracle (oracle/ssor.py) and its use in the SQMR oracle.

* splitmix64 against the generator's published outputs for seed 0.
* The Jones-Plassmann colouring is proper and equals the sequential greedy colouring that visits
  the rows in decreasing priority (networkx's greedy_color with that order), the identity that
  characterises it: a row's neighbours coloured before it are exactly those of higher priority.
* M^{-1} r, M1^{-1} v and M2^{-1} t against dense solves with M = (D + w L) D^{-1} (D + w U)
  built from the colour-permuted matrix's triangles (np.tril / np.triu), and the forward sweep
  with one colour per row in natural order against scipy's triangular solve.
* omega = 0 reduces SSOR to Jacobi: SQMR's iterates equal those of the Jacobi-split SQMR.
* The preconditioned Lanczos residuals are M^{-1}-orthogonal in the bilinear form, and the
  SSOR-preconditioned SQMR solves the FEM system of a small Kuhn mesh.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle
from oracle.ssor import SSOR, jp_colouring, priority_rank, splitmix64
from oracle.sqmr import sqmr
from paper_1808_00186_gb300 import synth


def test_splitmix64_published_outputs():
    gamma = 0x9E3779B97F4A7C15
    states = np.array([0, gamma, (2 * gamma) % 2 ** 64], dtype=np.uint64)
    out = [int(v) for v in splitmix64(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def random_pattern(n, deg, seed):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, n * deg // 2)
    j = rng.integers(0, n, n * deg // 2)
    S = sp.coo_matrix((np.ones(len(i)), (i, j)), shape=(n, n))
    S = ((S + S.T) + sp.eye(n)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return S


def fem_system(n=5):
    m = synth.cube_block_model(n)
    ref = oracle.System(m.mesh.nodes, m.mesh.tets, m.sigma, m.sigma_p, m.freq, synth.sources_array(m.sources))
    rp, col, val, b = ref.system()
    E = len(rp) - 1
    return sp.csr_matrix((val, col, rp), shape=(E, E)), b[0]


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def greedy_reference(indptr, indices):
    nx = pytest.importorskip("networkx")
    n = len(indptr) - 1
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for i in range(n):
        for j in indices[indptr[i]:indptr[i + 1]]:
            if j != i:
                G.add_edge(i, int(j))
    order = list(np.argsort(-priority_rank(n)))
    col = nx.greedy_color(G, strategy=lambda g, c: iter(int(v) for v in order))
    return np.array([col[i] for i in range(n)])


@pytest.mark.parametrize("case", ["random_300_6", "random_500_12", "fem_n4"])
def test_colouring_is_proper_and_greedy_in_priority_order(case):
    if case == "fem_n4":
        A, _ = fem_system(4)
        indptr, indices = A.indptr, A.indices
    else:
        _, n, deg = case.split("_")
        S = random_pattern(int(n), int(deg), seed=int(n))
        indptr, indices = S.indptr, S.indices
    colour, rounds = jp_colouring(indptr, indices)
    n = len(indptr) - 1
    rows = np.repeat(np.arange(n), np.diff(indptr))
    off = rows != indices
    assert not np.any(colour[rows[off]] == colour[indices[off]])
    assert np.array_equal(colour, greedy_reference(indptr, indices))
    assert 1 <= rounds <= n
    assert colour.max() <= np.diff(indptr).max()  # at most (neighbours + 1) colours


def dense_ssor(A, colours, omega):
    perm = np.argsort(colours, kind="stable")
    Ap = A.toarray()[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    L, U = np.tril(Ap, -1), np.triu(Ap, 1)
    M1 = (D + omega * L) @ np.diag(1.0 / np.sqrt(np.diag(Ap)))
    M = (D + omega * L) @ np.linalg.inv(D) @ (D + omega * U)
    return perm, M, M1


@pytest.mark.parametrize("omega", [1.0, 0.6, 1.5])
def test_ssor_matches_dense_factors(omega):
    A, _ = fem_system(4)
    colour, _ = jp_colouring(A.indptr, A.indices)
    P = SSOR(A, colour, omega)
    perm, M, M1 = dense_ssor(A, colour, omega)
    assert np.allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())  # complex symmetric
    rng = np.random.default_rng(7)
    r = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    for got, Mat in ((P.minv(r), M), (P.m1inv(r), M1), (P.m2inv(r), M1.T)):
        want = np.empty_like(r)
        want[perm] = np.linalg.solve(Mat, r[perm])
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_natural_order_forward_sweep_is_a_triangular_solve():
    A, _ = fem_system(3)
    n = A.shape[0]
    P = SSOR(A, np.arange(n), 1.3)
    rng = np.random.default_rng(3)
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    T = (sp.diags(A.diagonal()) + 1.3 * sp.tril(A, -1)).tocsr()
    want = spl.spsolve_triangular(T, v, lower=True)
    assert np.linalg.norm(P.forward(v) - want) <= 1e-12 * np.linalg.norm(want)


def test_omega_zero_is_jacobi():
    A, b = fem_system(4)
    colour, _ = jp_colouring(A.indptr, A.indices)
    P = SSOR(A, colour, 0.0)
    r = b + 0.3
    assert np.allclose(P.minv(r), r / A.diagonal(), rtol=1e-14, atol=0)
    xj_end, it_j, _, rec_j = sqmr(A, b, tol=1e-9, record=True)
    xs_end, it_s, _, rec_s = sqmr(A, b, tol=1e-9, record=True, precond=P)
    # identical up to rounding (the two apply D^{-1/2} as D^{1/2} D^{-1} and as 1 / D^{1/2}); the
    # Lanczos recurrences amplify rounding differences only after a few tens of steps
    for xj, xs in zip(rec_j["x"][:30], rec_s["x"][:30]):
        assert np.linalg.norm(xj - xs) <= 1e-12 * max(np.linalg.norm(xj), 1e-300)
    assert abs(it_j - it_s) <= 2
    assert np.linalg.norm(xj_end - xs_end) <= 1e-8 * np.linalg.norm(xj_end)


def test_lanczos_residuals_are_minv_orthogonal():
    rng = np.random.default_rng(11)
    n = 80
    S = random_pattern(n, 6, seed=5)
    vals = rng.normal(size=S.nnz) + 1j * rng.normal(size=S.nnz)
    A = sp.csr_matrix((vals, S.indices, S.indptr), shape=(n, n))
    A = (0.5 * (A + A.T) + sp.diags(8.0 + 2.0j + rng.uniform(0, 1, n))).tocsr()
    colour, _ = jp_colouring(A.indptr, A.indices)
    P = SSOR(A, colour, 1.0)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    _, _, _, rec = sqmr(A, b, tol=1e-13, record=True, precond=P)
    R = rec["r"][:8]
    Z = [P.minv(r) for r in R]
    for i in range(len(R)):
        for j in range(i):
            assert abs(np.dot(R[i], Z[j])) <= 1e-9 * np.linalg.norm(R[i]) * np.linalg.norm(Z[j])


def test_ssor_sqmr_solves_the_fem_system_in_fewer_steps():
    A, b = fem_system(6)
    colour, _ = jp_colouring(A.indptr, A.indices)
    x_ref = spl.spsolve(A.tocsc(), b)
    x, it, rel, _ = sqmr(A, b, tol=1e-10, precond=SSOR(A, colour, 1.0))
    assert rel <= 1e-10
    assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    _, it_j, _, _ = sqmr(A, b, tol=1e-10)
    assert it < it_j, (it, it_j)
