"""Pins for the oracle's whole-space dipole primary field (Appendix A eqs. A.1-A.3).

The garbled x-dipole bracket is read as (d_a d_j / r^2)(-k^2 r^2 + 3ikr + 3) + delta_aj
(k^2 r^2 - ikr - 1).  These tests pin that reading, k and the sign convention without
retyping the formula: the field must satisfy the source-free curl-curl equation of eq. 6's
operator, curl curl E + i w mu0 sigma E = 0 (checked by finite differences), be
divergence-free, reduce to the textbook static dipole as w -> 0, and be the same field for
the x-, y- and z-dipoles up to a rotation of axes.
"""
import math

import numpy as np
import pytest

import oracle

MU0 = 4e-7 * math.pi


def field_fn(src, sigma, freq):
    return lambda x: oracle.primary_field(np.asarray(x).reshape(-1, 3), src, sigma, freq).reshape(-1, 3)


def jacobian(F, x, h):
    """dF_i/dx_j by 4th-order central differences, vectorised over the stencil."""
    pts = []
    for j in range(3):
        for s in (-2, -1, 1, 2):
            p = np.array(x, dtype=float)
            p[j] += s * h
            pts.append(p)
    v = F(np.array(pts)).reshape(3, 4, 3)
    Jm = (v[:, 0] - 8 * v[:, 1] + 8 * v[:, 2] - v[:, 3]) / (12 * h)   # [j][i]
    return Jm.T


def curl(F, h):
    def c(xs):
        xs = np.asarray(xs).reshape(-1, 3)
        out = []
        for x in xs:
            J = jacobian(F, x, h)
            out.append([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
        return np.array(out)
    return c


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sigma,freq", [(1.0, 2.0), (3.3, 0.25), (0.5, 5.0)])
def test_curl_curl_equation(axis, sigma, freq):
    src = np.array([10.0, -20.0, 5.0, axis, 1.0])
    F = field_fn(src, sigma, freq)
    skin = math.sqrt(2.0 / (2 * math.pi * freq * MU0 * sigma))
    rng = np.random.default_rng(axis)
    for _ in range(3):
        d = rng.normal(size=3)
        x = src[:3] + d / np.linalg.norm(d) * skin * rng.uniform(0.3, 2.0)
        h = 2e-3 * skin
        cc = curl(curl(F, h), h)(x)[0]
        E = F(x)[0]
        term = 1j * 2 * math.pi * freq * MU0 * sigma * E
        assert np.abs(cc + term).max() <= 2e-6 * np.abs(term).max()
        div = np.trace(jacobian(F, x, h))
        assert abs(div) <= 1e-7 * np.abs(E).max() / skin


def test_static_limit_is_dc_dipole():
    src = np.array([0.0, 0.0, 0.0, 0, 2.5])
    sigma = 0.7
    rng = np.random.default_rng(5)
    pts = rng.normal(size=(10, 3)) * 3.0
    E = oracle.primary_field(pts, src, sigma, 1e-14)
    for x, e in zip(pts, E):
        r = np.linalg.norm(x)
        n = x / r
        dc = 2.5 / (4 * math.pi * sigma * r ** 3) * (3 * n[0] * n - np.array([1.0, 0, 0]))
        assert np.allclose(e, dc, rtol=1e-9, atol=0)


def test_axis_rotation():
    rng = np.random.default_rng(9)
    x_src = rng.normal(size=3) * 10
    pts = x_src + rng.normal(size=(8, 3)) * 400
    Ex = oracle.primary_field(pts, np.r_[x_src, 0, 1.0], 1.3, 1.0)
    # Cyclic relabelling (x, y, z) -> (y, z, x) turns the x-dipole into the y-dipole.
    perm = [2, 0, 1]
    Ey = oracle.primary_field(x_src[perm] + (pts - x_src)[:, perm], np.r_[x_src[perm], 1, 1.0], 1.3, 1.0)
    assert np.allclose(Ey, Ex[:, perm], rtol=1e-13, atol=0)
    Ez = oracle.primary_field(x_src[[1, 2, 0]] + (pts - x_src)[:, [1, 2, 0]], np.r_[x_src[[1, 2, 0]], 2, 1.0], 1.3, 1.0)
    assert np.allclose(Ez, Ex[:, [1, 2, 0]], rtol=1e-13, atol=0)


def test_decay_and_linearity_in_moment():
    sigma, freq = 1.0, 1.0
    skin = math.sqrt(2.0 / (2 * math.pi * freq * MU0 * sigma))
    r = np.array([3.0, 6.0]) * skin
    pts = np.stack([r, 0 * r, 0 * r], axis=1)
    E = oracle.primary_field(pts, np.array([0, 0, 0, 1, 1.0]), sigma, freq)  # broadside of a y-dipole
    # Broadside |E| r^3 ~ |k^2 r^2 - ikr - 1| e^{-r/skin}: the ratio of the two is the pure decay.
    k = (1 - 1j) / skin
    ratio = (abs(E[1, 1]) * r[1] ** 3 / abs(k * k * r[1] ** 2 - 1j * k * r[1] - 1)) / \
            (abs(E[0, 1]) * r[0] ** 3 / abs(k * k * r[0] ** 2 - 1j * k * r[0] - 1))
    assert ratio == pytest.approx(math.exp(-3.0), rel=1e-12)
    E2 = oracle.primary_field(pts, np.array([0, 0, 0, 1, 3.0]), sigma, freq)
    assert np.allclose(E2, 3.0 * E, rtol=1e-15)
