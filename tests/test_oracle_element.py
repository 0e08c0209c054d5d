"""Pins for the oracle's element matrices (Appendix B eqs. B.14-B.15 with eq. B.16 signs).

The reference values here are exact rational integrals: the basis of eqs. B.8-B.13 is built
symbolically from the exact inverse of [1 x y z], its curl is taken symbolically, and every
product is integrated exactly over the tet through the affine map to the unit tet with the
monomial formula  int xi^a eta^b zeta^c = a! b! c! / (a + b + c + 3)!.  None of that uses the
closed form int lambda_p lambda_q = V (1 + delta_pq) / 20 that the oracle is written with.
"""
import math

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

import oracle
from paper_1808_00186_gb300 import synth
from tests.golden.tables import local_edge_table

X, Y, Z = sympy.symbols("x y z")
XI, ETA, ZETA = sympy.symbols("xi eta zeta")


def exact_element(P):
    """Exact K^W, M^W (without edge lengths and signs) for integer vertices P [4][3]."""
    P = [[sympy.Integer(int(v)) for v in row] for row in P]
    C = sympy.Matrix([[1, *row] for row in P])
    Cinv = C.inv()
    lam = [Cinv[0, i] + Cinv[1, i] * X + Cinv[2, i] * Y + Cinv[3, i] * Z for i in range(4)]
    grad = [sympy.Matrix([sympy.diff(l, v) for v in (X, Y, Z)]) for l in lam]
    W = []
    for a, b in local_edge_table():
        W.append(lam[a] * grad[b] - lam[b] * grad[a])

    def curl(F):
        return sympy.Matrix([sympy.diff(F[2], Y) - sympy.diff(F[1], Z),
                             sympy.diff(F[0], Z) - sympy.diff(F[2], X),
                             sympy.diff(F[1], X) - sympy.diff(F[0], Y)])

    J = sympy.Matrix([[P[k][d] - P[0][d] for k in (1, 2, 3)] for d in range(3)])
    detJ = abs(J.det())
    sub = {X: P[0][0] + J[0, 0] * XI + J[0, 1] * ETA + J[0, 2] * ZETA,
           Y: P[0][1] + J[1, 0] * XI + J[1, 1] * ETA + J[1, 2] * ZETA,
           Z: P[0][2] + J[2, 0] * XI + J[2, 1] * ETA + J[2, 2] * ZETA}

    def integrate(expr):
        poly = sympy.Poly(sympy.expand(expr.subs(sub, simultaneous=True)), XI, ETA, ZETA)
        tot = sympy.Integer(0)
        for (a, b, c), coef in poly.terms():
            tot += coef * sympy.factorial(a) * sympy.factorial(b) * sympy.factorial(c) / sympy.factorial(a + b + c + 3)
        return tot * detJ

    curls = [curl(w) for w in W]
    K = np.zeros((6, 6))
    M = np.zeros((6, 6))
    for i in range(6):
        for j in range(i, 6):
            K[i, j] = K[j, i] = float(integrate(curls[i].dot(curls[j])))
            M[i, j] = M[j, i] = float(integrate(W[i].dot(W[j])))
    return K, M, float(detJ) / 6.0


TETS = [
    [[0, 0, 0], [2, 0, 1], [1, 3, 0], [0, 1, 4]],
    [[0, 0, 0], [1, 3, 0], [2, 0, 1], [0, 1, 4]],      # same tet, opposite orientation
    [[1, 1, 1], [2, 1, 1], [2, 2, 1], [2, 2, 2]],      # a Kuhn tet
    [[-3, 2, 5], [4, -1, 2], [0, 6, -2], [5, 5, 5]],
]


@pytest.mark.parametrize("P", TETS)
def test_element_matrices_exact(P):
    P = np.array(P, dtype=np.float64)
    table = local_edge_table()
    ln = np.array([np.linalg.norm(P[b] - P[a]) for a, b in table])
    for signs in (np.ones(6, np.int8), np.array([1, -1, 1, -1, -1, 1], np.int8)):
        K, M, vol = oracle.element(P, signs)
        Kw, Mw, vol_ex = exact_element(P)
        scale = np.outer(signs * ln, signs * ln)
        assert vol == pytest.approx(vol_ex, rel=1e-14)
        assert np.abs(K - scale * Kw).max() <= 1e-13 * np.abs(scale * Kw).max()
        assert np.abs(M - scale * Mw).max() <= 1e-13 * np.abs(scale * Mw).max()


def random_tets(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        P = rng.normal(size=(4, 3)) * rng.uniform(1, 300)
        v = abs(np.linalg.det(P[1:] - P[0])) / 6
        if v > 1e-2 * np.prod(np.ptp(P, axis=0)):
            out.append(P)
    return out


def global_dofs(P, signs, field_on_edge):
    """Edge DOFs in the element's global orientation: local direction a -> b times S_i."""
    table = local_edge_table()
    return np.array([signs[i] * field_on_edge(P[a], P[b]) for i, (a, b) in enumerate(table)])


@pytest.mark.parametrize("seed", range(4))
def test_gradient_null_space_and_constant_field(seed):
    rng = np.random.default_rng(100 + seed)
    for P in random_tets(5, seed):
        signs = rng.choice([-1, 1], size=6).astype(np.int8)
        K, M, vol = oracle.element(P, signs)
        assert np.allclose(K, K.T, rtol=0, atol=1e-14 * np.abs(K).max())
        assert np.allclose(M, M.T, rtol=0, atol=1e-14 * np.abs(M).max())
        assert np.all(np.linalg.eigvalsh(M) > 0)
        # Discrete gradient: DOF of grad phi on edge a -> b is (phi_b - phi_a) / l.  K annihilates it.
        phi = rng.normal(size=4)
        idx = {tuple(p): k for k, p in enumerate(map(tuple, P))}
        g = global_dofs(P, signs, lambda pa, pb: (phi[idx[tuple(pb)]] - phi[idx[tuple(pa)]]) / np.linalg.norm(pb - pa))
        assert np.abs(K @ g).max() <= 1e-12 * np.abs(K).max() * np.abs(g).max()
        # A constant field E0 has DOFs E0 . t; M reproduces its L2 norm, K its zero curl.
        E0 = rng.normal(size=3)
        e = global_dofs(P, signs, lambda pa, pb: E0 @ (pb - pa) / np.linalg.norm(pb - pa))
        assert e @ M @ e == pytest.approx(vol * (E0 @ E0), rel=1e-12)
        assert np.abs(K @ e).max() <= 1e-12 * np.abs(K).max() * np.abs(e).max()


def test_volumes_tile_the_box():
    m = synth.kuhn_mesh(3, (-1, -2, 0), (2, 1, 4), jitter=0.15, seed=3)
    total = 0.0
    for t in m.tets:
        _, _, v = oracle.element(m.nodes[t], np.ones(6, np.int8))
        total += v
    assert total == pytest.approx(3 * 3 * 4, rel=1e-13)
