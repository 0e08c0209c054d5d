"""FP64 CPU oracle of the conjugate orthogonal conjugate gradient method (COCG; van der Vorst and
Melissen, IEEE Trans. Magn. 26, 1990) for the complex-symmetric system of the paper's eq. 9.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/, __graft_entry__.smoke() and bench.py's
CPU legs may use it; the CUDA library never does.

The paper's mesh-adaptation study (Section 5.3) solves the same system with a short-recurrence
Krylov method for complex-symmetric matrices (symmetric QMR).  COCG is the conjugate-gradient
member of that family: CG with the unconjugated bilinear form u^T v in place of the Hermitian
inner product, which A^T = A makes a valid orthogonality for the residuals.  Preconditioner: the
Jacobi diagonal M = diag(A) (complex symmetric, so z = M^{-1} r keeps the recurrences valid).

Steps, in the method's order (x0 given, r0 = b - A x0, z0 = M^{-1} r0, p0 = z0, rho0 = r0^T z0):
    q = A p;  alpha = rho / (p^T q);  x += alpha p;  r -= alpha q;  stop when ||r||_2 <= tol ||b||_2
    z = M^{-1} r;  rho' = r^T z;  beta = rho' / rho;  p = z + beta p.
A scipy sparse product is the only library step.
"""
from __future__ import annotations

import numpy as np


def cocg(A, b, tol: float = 1e-8, maxit: int = 100000, x0=None, record=False):
    """Returns (x, iterations, relative residual ||b - A x|| / ||b|| recomputed at the end,
    residual history if record)."""
    b = np.asarray(b, dtype=np.complex128)
    d = np.asarray(A.diagonal(), dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A @ x
    z = r / d
    p = z.copy()
    rho = np.dot(r, z)  # bilinear: no conjugate
    bn = np.linalg.norm(b)
    hist = [r.copy()] if record else None
    it = 0
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0, hist
    while np.linalg.norm(r) > tol * bn and it < maxit:
        q = A @ p
        pq = np.dot(p, q)
        if pq == 0.0 or rho == 0.0:
            break  # breakdown of the bilinear form
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if record:
            hist.append(r.copy())
        z = r / d
        rho_new = np.dot(r, z)
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    rel = np.linalg.norm(b - A @ x) / bn
    return x, it, rel, hist
