"""FP64 CPU oracle of the symmetric QMR method (SQMR; Freund and Nachtigal, 1994) for the
complex-symmetric system of the paper's eq. 9: the solver of the paper's mesh-adaptation study
(Section 5.3).

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/, __graft_entry__.smoke() and bench.py's
CPU legs may use it; the CUDA library never does.

SQMR runs the symmetric Lanczos recurrences in the bilinear form u^T v (the same residuals r_n,
directions q_n and scalars alpha, beta as COCG) and takes as iterate the quasi-minimal-residual
combination of them, which smooths COCG's erratic residual history.  Preconditioner: the Jacobi
diagonal split symmetrically, M = M1 M2 with M1 = M2 = D^{1/2} (D = diag(A)); only
M1^{-1} v = D^{-1/2} v (principal complex square root) and M^{-1} v = D^{-1} v are applied.  The
symmetric SOR split of oracle/ssor.py (the paper's SQMR + SOR runs) can be passed instead.

Steps, in the method's order (x0 given; r0 = b - A x0; t = M1^{-1} r0; tau0 = ||t||_2;
q0 = M2^{-1} t; theta0 = 0; rho0 = r0^T q0; d0 = 0):
    t = A q;  sigma = q^T t;  alpha = rho / sigma;  r -= alpha t
    t = M1^{-1} r;  theta' = ||t|| / tau;  c = 1 / sqrt(1 + theta'^2);  tau' = tau theta' c
    d = c^2 theta^2 d + c^2 alpha q;  x += d;  stop when ||b - A x||_2 <= tol ||b||_2
    u = M2^{-1} t;  rho' = r^T u;  beta = rho' / rho;  q = u + beta q.
A scipy sparse product is the only library step.  The stopping test recomputes the true residual
each step (the oracle's purpose is exactness, not speed).
"""
from __future__ import annotations

import numpy as np


def sqmr(A, b, tol: float = 1e-8, maxit: int = 100000, x0=None, record=False, precond=None):
    """Returns (x, iterations, relative residual ||b - A x|| / ||b|| recomputed at the end, record)
    where record (if asked) holds per step the iterate x_n, tau_n and the Lanczos residual r_n.
    precond: None for the Jacobi split, else an object whose m1inv / m2inv apply M1^{-1} and
    M2^{-1} of a symmetric split M = M1 M2, M2 = M1^T (oracle.ssor.SSOR)."""
    b = np.asarray(b, dtype=np.complex128)
    if precond is None:
        d = np.asarray(A.diagonal(), dtype=np.complex128)
        m1 = 1.0 / np.sqrt(d)  # M1^{-1} = M2^{-1} = D^{-1/2}, principal root
        m1inv = m2inv = lambda v: m1 * v
    else:
        m1inv, m2inv = precond.m1inv, precond.m2inv
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A @ x
    t = m1inv(r)
    tau = np.linalg.norm(t)
    q = m2inv(t)
    theta = 0.0
    rho = np.dot(r, q)  # bilinear: no conjugate
    dv = np.zeros_like(b)
    bn = np.linalg.norm(b)
    rec = {"x": [x.copy()], "tau": [tau], "r": [r.copy()]} if record else None
    it = 0
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0, rec
    while np.linalg.norm(b - A @ x) > tol * bn and it < maxit:
        t = A @ q
        sigma = np.dot(q, t)
        if sigma == 0.0 or rho == 0.0:
            break  # breakdown of the bilinear form
        alpha = rho / sigma
        r = r - alpha * t
        t = m1inv(r)
        theta_new = np.linalg.norm(t) / tau
        c2 = 1.0 / (1.0 + theta_new * theta_new)
        tau = tau * theta_new * np.sqrt(c2)
        dv = c2 * theta * theta * dv + c2 * alpha * q
        theta = theta_new
        x = x + dv
        it += 1
        if record:
            rec["x"].append(x.copy())
            rec["tau"].append(tau)
            rec["r"].append(r.copy())
        u = m2inv(t)
        rho_new = np.dot(r, u)
        beta = rho_new / rho
        rho = rho_new
        q = u + beta * q
    rel = np.linalg.norm(b - A @ x) / bn
    return x, it, rel, rec
