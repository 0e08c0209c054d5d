"""Pins for the COCG oracle (oracle/cocg.py), none of which asks the oracle for its own answer.

* Real symmetric positive definite systems: COCG is Jacobi-preconditioned CG there, so its
  residual history equals that of the library CG (scipy.sparse.linalg.cg, same preconditioner).
* Complex symmetric systems: the solution equals a dense solve; the preconditioned residuals are
  orthogonal in the bilinear form (r_i^T M^{-1} r_k = 0, i != k), which is what the method rests
  on; in exact arithmetic it terminates within n steps.
* The assembled FEM system of a small Kuhn mesh: the solution equals the dense LU of the oracle's
  matrix (numpy), at the solver's tolerance.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle.cocg import cocg
from paper_1808_00186_gb300 import synth


def spd(n, seed):
    rng = np.random.default_rng(seed)
    B = sp.random(n, n, density=0.05, random_state=seed) + sp.eye(n)
    A = (B @ B.T + sp.diags(rng.uniform(0.5, 2.0, n))).tocsr()
    return A, rng.normal(size=n)


def complex_symmetric(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    R = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = 0.5 * (R + R.T) / np.sqrt(n) + np.diag(shift * (1.0 + 0.3j) + rng.uniform(0, 1, n))
    assert np.allclose(A, A.T)
    return sp.csr_matrix(A), rng.normal(size=n) + 1j * rng.normal(size=n)


def test_equals_preconditioned_cg_on_real_spd():
    A, b = spd(300, 1)
    x, it, rel, hist = cocg(A, b, tol=1e-10, record=True)
    ours = [np.linalg.norm(r) for r in hist]
    ref = [np.linalg.norm(b)]
    M = sp.diags(1.0 / A.diagonal())
    spla.cg(A, b, rtol=1e-10, atol=0.0, M=M, callback=lambda xk: ref.append(np.linalg.norm(b - A @ xk)))
    # the first steps agree to rounding (later ones drift apart as rounding amplifies in CG);
    # the step count is the same
    assert np.allclose(ours[:10], ref[:10], rtol=1e-8, atol=0.0)
    assert abs(len(ours) - len(ref)) <= 1
    assert np.linalg.norm(x - spla.spsolve(A.tocsc(), b)) <= 1e-8 * np.linalg.norm(x)


def test_complex_symmetric_solution_orthogonality_and_termination():
    A, b = complex_symmetric(40, 3)
    x, it, rel, hist = cocg(A, b, tol=1e-12, record=True)
    xd = np.linalg.solve(A.toarray(), b)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert it <= 40 + 5  # n steps in exact arithmetic
    d = A.diagonal()
    for i in range(6):
        for k in range(i + 1, 6):
            g = np.dot(hist[i], hist[k] / d)
            scale = np.linalg.norm(hist[i]) * np.linalg.norm(hist[k] / d)
            assert abs(g) <= 1e-9 * scale
    # the Hermitian inner product does not make them orthogonal (the form matters)
    herm = abs(np.vdot(hist[0], hist[1] / d)) / (np.linalg.norm(hist[0]) * np.linalg.norm(hist[1] / d))
    assert herm > 1e-3


def test_fem_system_matches_dense_lu():
    m = synth.kuhn_mesh(3, (0.0, 0.0, 0.0), (300.0, 300.0, 300.0), jitter=0.1, seed=5)
    rng = np.random.default_rng(5)
    sigma = rng.choice([0.5, 1.0, 3.0], size=m.n_tets)
    src = np.array([[-400.0, 30.0, 40.0, 0, 1.0]])
    ref = oracle.System(m.nodes, m.tets, sigma, 1.0, 2.0, src)
    rp, col, val, b = ref.system()
    n = len(rp) - 1
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    x, it, rel, _ = cocg(A, b[0], tol=1e-12, maxit=20000)
    xd = np.linalg.solve(A.toarray(), b[0])
    assert rel <= 1e-11
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_zero_rhs_and_initial_guess():
    A, b = complex_symmetric(20, 7)
    x, it, rel, _ = cocg(A, np.zeros(20, complex))
    assert it == 0 and not np.any(x)
    xd = np.linalg.solve(A.toarray(), b)
    x, it, rel, _ = cocg(A, b, tol=1e-12, x0=xd)
    assert it == 0 and rel <= 1e-12
