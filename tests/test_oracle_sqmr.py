"""Pins for the SQMR oracle (oracle/sqmr.py), none of which asks the oracle for its own answer.

* The Lanczos part: SQMR's residuals r_n are COCG's (same bilinear Lanczos recurrences, Jacobi
  preconditioning), so they must equal the independent COCG oracle's residual history.
* The QMR part: the SQMR iterate is the quasi-minimal-residual smoothing of the COCG iterates
  (Zhou and Walker's residual smoothing): with s_n = ||D^{-1/2} r_n||,
  1/tau_n^2 = 1/tau_{n-1}^2 + 1/s_n^2 and x^Q_n = (1 - eta) x^Q_{n-1} + eta x^C_n,
  eta = tau_n^2 / s_n^2, where x^C_n is obtained from COCG's residual by a dense solve.
* The quasi-residual bound ||D^{-1/2} (b - A x_n)|| <= sqrt(n + 1) tau_n at every step.
* Exactness: the solution equals a dense solve (complex symmetric and the FEM system of a small
  Kuhn mesh); in exact arithmetic the method terminates within n steps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.cocg import cocg
from oracle.sqmr import sqmr
from paper_1808_00186_gb300 import synth


def complex_symmetric(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    R = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = 0.5 * (R + R.T) / np.sqrt(n) + np.diag(shift * (1.0 + 0.3j) + rng.uniform(0, 1, n))
    assert np.allclose(A, A.T)
    return sp.csr_matrix(A), rng.normal(size=n) + 1j * rng.normal(size=n)


@pytest.mark.parametrize("seed,shift", [(1, 4.0), (2, 1.5)])
def test_lanczos_residuals_equal_cocg_and_iterates_are_its_qmr_smoothing(seed, shift):
    A, b = complex_symmetric(60, seed, shift)
    Ad = A.toarray()
    d = A.diagonal()
    w = 1.0 / np.abs(d)  # |D^{-1/2} v|^2 = sum |v_i|^2 / |d_i|
    _, _, _, hist = cocg(A, b, tol=1e-13, record=True)
    _, _, _, rec = sqmr(A, b, tol=1e-13, record=True)
    steps = min(12, len(hist) - 1, len(rec["r"]) - 1)
    assert steps >= 10
    for n in range(steps + 1):
        assert np.allclose(rec["r"][n], hist[n], rtol=0, atol=1e-9 * np.linalg.norm(b))
    tau = np.sqrt(np.sum(w * np.abs(b) ** 2))
    assert np.isclose(rec["tau"][0], tau, rtol=1e-12)
    xq = np.zeros_like(b)
    for n in range(1, steps + 1):
        s2 = np.sum(w * np.abs(hist[n]) ** 2)
        tau2 = 1.0 / (1.0 / tau ** 2 + 1.0 / s2)
        eta = tau2 / s2
        xc = np.linalg.solve(Ad, b - hist[n])  # the COCG iterate with residual hist[n]
        xq = (1.0 - eta) * xq + eta * xc
        tau = np.sqrt(tau2)
        assert np.isclose(rec["tau"][n], tau, rtol=1e-9)
        assert np.linalg.norm(rec["x"][n] - xq) <= 1e-8 * np.linalg.norm(xq)


def test_quasi_residual_bound_solution_and_termination():
    A, b = complex_symmetric(40, 3)
    s = 1.0 / np.sqrt(np.abs(A.diagonal()))
    x, it, rel, rec = sqmr(A, b, tol=1e-12, record=True)
    for n, (xn, tn) in enumerate(zip(rec["x"], rec["tau"])):
        rn = np.linalg.norm(s * (b - A @ xn))
        assert rn <= np.sqrt(n + 1) * tn * (1 + 1e-10) + 1e-14
    assert rel <= 1e-12
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert it <= 40 + 5


def test_fem_system_matches_dense_lu():
    m = synth.kuhn_mesh(3, (0.0, 0.0, 0.0), (300.0, 300.0, 300.0), jitter=0.1, seed=5)
    rng = np.random.default_rng(5)
    sigma = rng.choice([0.5, 1.0, 3.0], size=m.n_tets)
    src = np.array([[-400.0, 30.0, 40.0, 0, 1.0]])
    ref = oracle.System(m.nodes, m.tets, sigma, 1.0, 2.0, src)
    rp, col, val, b = ref.system()
    n = len(rp) - 1
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    x, it, rel, _ = sqmr(A, b[0], tol=1e-12, maxit=20000)
    xd = np.linalg.solve(A.toarray(), b[0])
    assert rel <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_zero_rhs_and_exact_initial_guess():
    A, b = complex_symmetric(20, 7)
    x, it, rel, _ = sqmr(A, np.zeros(20, complex))
    assert it == 0 and not np.any(x)
    xd = np.linalg.solve(A.toarray(), b)
    x, it, rel, _ = sqmr(A, b, tol=1e-12, x0=xd)
    assert it == 0 and rel <= 1e-12
